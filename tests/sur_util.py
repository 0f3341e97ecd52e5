"""Test helper: the surrogate oracle run with every tensor operation in a
given floating-point type (BF16 rounding at the same points). Running it in
FP32 gives a second correct implementation whose distance from the FP64 oracle
measures the spread that accumulation precision alone causes on given inputs.

Reordered runs. Relabelling the hidden channels by a permutation (the rows and
columns of every weight, the biases and the projection's columns moved along)
leaves the network's function unchanged in exact arithmetic and rounds the
same activations to BF16, but every reduction over channels adds its terms in
another order. Each permutation therefore gives one more correct FP32
implementation; `fp32_runs` returns several, and the GPU parity bounds are
taken from the largest distance among them (see test_gpu_surrogate)."""
import contextlib

import numpy as np
import torch

from oracle import surrogate as S


@contextlib.contextmanager
def _dtype(dtype):
    old = S.DT
    S.DT = dtype
    try:
        yield
    finally:
        S.DT = old


def params_in(flat, dtype):
    P = S.Params(torch.as_tensor(flat, dtype=torch.float64))
    for k in ("w_lift", "b_lift", "w_proj", "b_proj"):
        setattr(P, k, getattr(P, k).to(dtype))
    P.w1, P.w2 = [w.to(dtype) for w in P.w1], [w.to(dtype) for w in P.w2]
    P.b1, P.b2 = [b.to(dtype) for b in P.b1], [b.to(dtype) for b in P.b2]
    return P


def channel_permutation(n_params, perm, blocks=4):
    """Index array fp such that flat[fp] is the parameter vector of the same
    network with hidden channel c renamed perm^-1(c) (new channel k is old
    channel perm[k])."""
    P = S.Params(np.arange(n_params, dtype=np.float64), len(perm), blocks)
    pi = torch.as_tensor(perm, dtype=torch.long)
    parts = [P.w_lift[pi], P.b_lift[pi]]
    for b in range(blocks):
        parts += [P.w1[b][:, :, :, pi][..., pi], P.b1[b][pi], P.w2[b][:, :, :, pi][..., pi], P.b2[b][pi]]
    parts += [P.w_proj[:, pi], P.b_proj]
    return torch.cat([t.reshape(-1) for t in parts]).long().numpy()


def oracle_in(dtype, frames, targets, flat, n, want_grad=True, perm=None):
    """(pred, grad, g_frames, loss) of the oracle with `dtype` arithmetic;
    frames (B, n^3, 8), targets (B, n^3, 3) or None. perm: run the network
    with its hidden channels relabelled (results are returned in the original
    labelling)."""
    def rnd(t):
        return torch.as_tensor(t).to(torch.float32).to(torch.bfloat16).to(dtype)

    flat = np.asarray(flat, dtype=np.float64)
    fp = None
    if perm is not None:
        fp = channel_permutation(flat.size, perm)
        flat = flat[fp]
    with _dtype(dtype):
        P = params_in(flat, dtype)
        f = torch.as_tensor(frames).to(dtype).reshape(-1, n, n, n, 8)
        pred = S.forward(f, P, n, rnd=rnd)["pred"].double().reshape(f.shape[0], -1, 3)
        if not want_grad:
            return pred, None, None, None
        L, g, gf = S.loss_and_grad(f, torch.as_tensor(targets).to(dtype), P, n, rnd=rnd)
    g = g.double()
    if fp is not None:
        out = torch.empty_like(g)
        out[torch.as_tensor(fp)] = g
        g = out
    return pred, g, gf.double(), L


def fp32_runs(frames, targets, flat, n, k=6, want_grad=True, seed=0, channels=32):
    """k correct FP32 implementations: the identity labelling and k - 1 seeded
    channel permutations; a list of oracle_in results."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        perm = None if i == 0 else rng.permutation(channels)
        out.append(oracle_in(torch.float32, frames, targets, flat, n, want_grad=want_grad, perm=perm))
    return out


def blocks_of(n_params, blocks=4):
    """(name, flat indices) of every parameter block."""
    P = S.Params(np.arange(n_params, dtype=np.float64), 32, blocks)
    out = [("w_lift", P.w_lift), ("b_lift", P.b_lift), ("w_proj", P.w_proj), ("b_proj", P.b_proj)]
    for bi in range(blocks):
        out += [(f"w1_{bi}", P.w1[bi]), (f"b1_{bi}", P.b1[bi]), (f"w2_{bi}", P.w2[bi]), (f"b2_{bi}", P.b2[bi])]
    return [(k, v.reshape(-1).long().numpy()) for k, v in out]
