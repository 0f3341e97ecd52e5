"""Test helper: the surrogate oracle run with every tensor operation in a
given floating-point type (BF16 rounding at the same points). Running it in
FP32 gives a second correct implementation whose distance from the FP64 oracle
measures the spread that accumulation precision alone causes on given inputs."""
import contextlib

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


def oracle_in(dtype, frames, targets, flat, n, want_grad=True):
    """(pred, grad, g_frames, loss) of the oracle with `dtype` arithmetic;
    frames (B, n^3, 8), targets (B, n^3, 3) or None."""
    def rnd(t):
        return torch.as_tensor(t).to(torch.float32).to(torch.bfloat16).to(dtype)

    with _dtype(dtype):
        P = params_in(flat, dtype)
        f = torch.as_tensor(frames).to(dtype).reshape(-1, n, n, n, 8)
        pred = S.forward(f, P, n, rnd=rnd)["pred"].double().reshape(f.shape[0], -1, 3)
        if not want_grad:
            return pred, None, None, None
        L, g, gf = S.loss_and_grad(f, torch.as_tensor(targets).to(dtype), P, n, rnd=rnd)
    return pred, g.double(), gf.double(), L


def blocks_of(n_params, blocks=4):
    """(name, flat indices) of every parameter block."""
    import numpy as np
    P = S.Params(np.arange(n_params, dtype=np.float64), 32, blocks)
    out = [("w_lift", P.w_lift), ("b_lift", P.b_lift), ("w_proj", P.w_proj), ("b_proj", P.b_proj)]
    for bi in range(blocks):
        out += [(f"w1_{bi}", P.w1[bi]), (f"b1_{bi}", P.b1[bi]), (f"w2_{bi}", P.w2[bi]), (f"b2_{bi}", P.b2[bi])]
    return [(k, v.reshape(-1).long().numpy()) for k, v in out]
