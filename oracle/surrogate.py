"""Oracle of the learned grid-space surrogate (test infrastructure only: the
product never imports it; tests, smoke() and bench.py's CPU legs do).

The paper names learned dynamics models only as a direction (Sec. 6). The
surrogate is a small 3D convolutional neural operator over the simulation grid:

  features f (8 channels per node): m, p_x, p_y, p_z, phi_0, phi_1, phi_2, 0
  h_0   = W_l f + b_l                                   (1x1x1 lift to C channels)
  r_b   = relu(conv3(h_{b-1}, W1_b) + b1_b)             b = 1..B
  h_b   = h_{b-1} + conv3(r_b, W2_b) + b2_b
  pred  = f[1:4] + W_p h_B + b_p                        (momentum, 10 steps later)

conv3 is the zero-padded 3x3x3 cross-correlation over nodes (i, j, k):
  conv3(h, W)[i,j,k,o] = sum_{a,b,c,q} W[a,b,c,o,q] h[i+a-1, j+b-1, k+c-1, q].

Precision: the CUDA kernels store weights and activations (and activation
gradients) in BF16 and accumulate in FP32. This oracle rounds at the same
points (argument `rnd`) and computes everything else in FP64, so both sides
agree up to accumulation order. With rnd = identity the backward pass is the
exact FP64 gradient, which the tests pin against torch.autograd and finite
differences.

Features (`grid_features`): with the quadratic B-spline weights W_ip of the
MLS-MPM transfer (Sec. 3.1), m_i = sum_p W_ip m_p and p_i = sum_p W_ip m_p
(v_p + C_p (x_i - x_p)) (the affine momentum transfer without the stress
impulse); phi_i^k = sum_{p of material k} W_ip m_p / m_i is the mass fraction
of material k (0 where m_i = 0). Mass is divided by m_ref, momentum by
m_ref * v_ref.

Loss: L = mean over frames, nodes and components of (pred - target)^2 with the
target the momentum features of the frame 10 steps later.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as Fn

from . import mpm

DT = torch.float64
CIN = 8


def bf16(t):
    """Round to the nearest BF16 value (ties to even); returned in FP64."""
    return torch.as_tensor(t, dtype=DT).to(torch.float32).to(torch.bfloat16).to(DT)


def identity(t):
    return torch.as_tensor(t, dtype=DT)


# ---------------------------------------------------------------------------
# grid features from a particle state
# ---------------------------------------------------------------------------
def _t(a):
    return a.to(DT) if isinstance(a, torch.Tensor) else torch.as_tensor(np.asarray(a), dtype=DT)


class _Grid:
    def __init__(self, n):
        self.n, self.dx, self.inv_dx = n, 1.0 / n, float(n)


def grid_features(x, v, C, mat, mass, n, m_ref, v_ref, n_materials=3):
    """(n^3, 8) FP64 features, node order (i, j, k) with k fastest.
    mass: per-particle mass (N,); mat: material index per particle."""
    x, v, C, mass = (_t(a) for a in (x, v, C, mass))
    mat = torch.as_tensor(np.asarray(mat), dtype=torch.long)
    W, dpos, lin = mpm.stencil(x, _Grid(n))
    n3 = n ** 3
    idx = lin.reshape(-1)
    wm = W * mass[:, None]                                     # (N, 27)
    m = torch.zeros(n3, dtype=DT).index_add(0, idx, wm.reshape(-1))
    vel = v[:, None, :] + torch.einsum("pab,pob->poa", C, dpos)  # v_p + C_p (x_i - x_p)
    p = torch.zeros(n3, 3, dtype=DT).index_add(0, idx, (wm[..., None] * vel).reshape(-1, 3))
    out = torch.zeros(n3, CIN, dtype=DT)
    out[:, 0] = m / m_ref
    out[:, 1:4] = p / (m_ref * v_ref)
    has = m > 0
    safe = torch.where(has, m, torch.ones_like(m))
    for k in range(n_materials):
        sel = (mat == k).to(DT)
        mk = torch.zeros(n3, dtype=DT).index_add(0, idx, (wm * sel[:, None]).reshape(-1))
        out[:, 4 + k] = torch.where(has, mk / safe, torch.zeros_like(m))
    return out


def features_vjp_v(x, mass, n, g_feat, m_ref, v_ref):
    """dL/dv_p for a cotangent g_feat (n^3, 8) on the features: only the
    momentum channels depend on v, linearly: dL/dv_p = m_p sum_i W_ip g_i / (m_ref v_ref)."""
    x, mass = _t(x), _t(mass)
    W, _, lin = mpm.stencil(x, _Grid(n))
    g = torch.as_tensor(g_feat, dtype=DT)[:, 1:4]
    return mass[:, None] * torch.einsum("po,poa->pa", W, g[lin]) / (m_ref * v_ref)


def features_vjp(x, v, C, mat, mass, n, g_feat, m_ref, v_ref, channels=(0, 1, 2, 3)):
    """(dL/dx, dL/dv, dL/dC) for a cotangent g_feat (n^3, 8) on the feature
    channels `channels` (mass and momentum by default; the material fractions
    are left out), by torch autograd through grid_features."""
    xt = _t(x).clone().requires_grad_(True)
    vt = _t(v).clone().requires_grad_(True)
    Ct = _t(C).clone().requires_grad_(True)
    f = grid_features(xt, vt, Ct, mat, mass, n, m_ref, v_ref)
    g = torch.as_tensor(g_feat, dtype=DT).clone()
    keep = torch.zeros(CIN, dtype=DT)
    keep[list(channels)] = 1.0
    gx, gv, gC = torch.autograd.grad((f * g * keep).sum(), (xt, vt, Ct))
    return gx, gv, gC


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------
def param_count(channels=32, blocks=4, cin=CIN):
    c = channels
    return c * cin + c + blocks * 2 * (27 * c * c + c) + 3 * c + 3


class Params:
    """Views into the flat parameter vector, in this order:
    w_lift (C, cin), b_lift (C), then per block w1 (3,3,3,C,C), b1 (C),
    w2 (3,3,3,C,C), b2 (C), then w_proj (3, C), b_proj (3).
    Convolution weights are indexed [a][b][c][out][in]."""

    def __init__(self, flat, channels=32, blocks=4, cin=CIN):
        self.c, self.b, self.cin = channels, blocks, cin
        flat = torch.as_tensor(flat, dtype=DT)
        want = param_count(channels, blocks, cin)
        if flat.numel() != want:
            raise ValueError(f"parameter vector has {flat.numel()} entries, expected {want}")
        self.flat = flat
        i = 0

        def take(*shape):
            nonlocal i
            k = int(np.prod(shape))
            t = flat[i:i + k].reshape(*shape)
            i += k
            return t

        c = channels
        self.w_lift, self.b_lift = take(c, cin), take(c)
        self.w1, self.b1, self.w2, self.b2 = [], [], [], []
        for _ in range(blocks):
            self.w1.append(take(3, 3, 3, c, c))
            self.b1.append(take(c))
            self.w2.append(take(3, 3, 3, c, c))
            self.b2.append(take(c))
        self.w_proj, self.b_proj = take(3, c), take(3)


def init_params(seed, channels=32, blocks=4, cin=CIN):
    """He-normal weights; the second convolution of each block and the
    projection are scaled by 0.1 so that the network starts near pred = f[1:4]."""
    rng = np.random.default_rng(seed)
    c = channels
    parts = [rng.normal(0, np.sqrt(2.0 / cin), (c, cin)), np.zeros(c)]
    for _ in range(blocks):
        parts += [rng.normal(0, np.sqrt(2.0 / (27 * c)), (3, 3, 3, c, c)), np.zeros(c),
                  rng.normal(0, 0.1 * np.sqrt(2.0 / (27 * c)), (3, 3, 3, c, c)), np.zeros(c)]
    parts += [rng.normal(0, 0.1 * np.sqrt(1.0 / c), (3, c)), np.zeros(3)]
    return np.concatenate([np.ravel(a) for a in parts])


# ---------------------------------------------------------------------------
# convolution and its two adjoints (library conv3d as the primitive)
# ---------------------------------------------------------------------------
def conv3(h, w, b=None):
    """h (B, n, n, n, q) -> (B, n, n, n, o); w (3, 3, 3, o, q)."""
    inp = h.permute(0, 4, 1, 2, 3)
    ker = w.permute(3, 4, 0, 1, 2)
    out = Fn.conv3d(inp, ker, bias=b, padding=1)
    return out.permute(0, 2, 3, 4, 1)


def conv3_input_grad(g, w):
    """Adjoint of conv3 w.r.t. its input: sum_{a,b,c,o} W[a,b,c,o,q] g[i-a+1, j-b+1, k-c+1, o]."""
    inp = g.permute(0, 4, 1, 2, 3)
    ker = w.permute(3, 4, 0, 1, 2)
    out = Fn.conv_transpose3d(inp, ker, padding=1)
    return out.permute(0, 2, 3, 4, 1)


def conv3_weight_grad(h, g):
    """dW[a,b,c,o,q] = sum over frames and nodes of g[v, o] h[v + (a-1, b-1, c-1), q]
    (h zero outside the grid)."""
    n = h.shape[1]
    hp = Fn.pad(h, (0, 0, 1, 1, 1, 1, 1, 1))
    out = torch.zeros(3, 3, 3, g.shape[-1], h.shape[-1], dtype=DT)
    for a in range(3):
        for b in range(3):
            for c in range(3):
                hs = hp[:, a:a + n, b:b + n, c:c + n, :]
                out[a, b, c] = torch.einsum("zijko,zijkq->oq", g, hs)
    return out


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
def _grid(frames, n):
    """(B, n, n, n, 8) view of frames given as (B, n^3, 8), (n^3, 8) or already
    as a (B, n1, n2, n3, 8) block of nodes."""
    f = torch.as_tensor(frames, dtype=DT)
    if f.dim() == 5:
        return f
    return f.reshape(-1, n, n, n, f.shape[-1])


def forward(frames, P, n, rnd=bf16):
    """frames (B, n^3, 8) or (n^3, 8). Returns a cache with every stored
    activation and pred (B, n, n, n, 3)."""
    f = rnd(_grid(frames, n))
    wl = rnd(P.w_lift)
    h = rnd(torch.einsum("zijkq,oq->zijko", f, wl) + P.b_lift)
    cache = {"f": f, "h": [h], "r": [], "a_pos": []}
    for bi in range(P.b):
        a = conv3(h, rnd(P.w1[bi]), P.b1[bi])
        r = rnd(torch.relu(a))
        h = rnd(h + conv3(r, rnd(P.w2[bi]), P.b2[bi]))
        cache["r"].append(r)
        cache["a_pos"].append(a > 0)
        cache["h"].append(h)
    cache["pred"] = f[..., 1:4] + torch.einsum("zijko,co->zijkc", h, rnd(P.w_proj)) + P.b_proj
    return cache


def predict(frames, P, n, rnd=bf16):
    """Predicted normalised momentum, (B, nodes, 3)."""
    pred = forward(frames, P, n, rnd)["pred"]
    return pred.reshape(pred.shape[0], -1, 3)


def backward_from(cache, g_pred, P, n, rnd=bf16):
    """Reverse pass of a forward cache for a cotangent g_pred on the prediction
    (same shape as cache["pred"]): gradient w.r.t. the flat parameters (FP64)
    and w.r.t. the (rounded) input frames; the stored activation gradients
    are rounded by `rnd` where the kernels store them in BF16."""
    g_pred = torch.as_tensor(g_pred, dtype=DT).reshape(cache["pred"].shape)
    hB = cache["h"][-1]
    wp = rnd(P.w_proj)
    grads = {"w_proj": torch.einsum("zijkc,zijko->co", g_pred, hB), "b_proj": g_pred.sum((0, 1, 2, 3))}
    g_h = rnd(torch.einsum("zijkc,co->zijko", g_pred, wp))
    gw1, gb1, gw2, gb2 = [None] * P.b, [None] * P.b, [None] * P.b, [None] * P.b
    for bi in reversed(range(P.b)):
        h_prev, r = cache["h"][bi], cache["r"][bi]
        gw2[bi] = conv3_weight_grad(r, g_h)
        gb2[bi] = g_h.sum((0, 1, 2, 3))
        g_a = rnd(conv3_input_grad(g_h, rnd(P.w2[bi])) * cache["a_pos"][bi])
        gw1[bi] = conv3_weight_grad(h_prev, g_a)
        gb1[bi] = g_a.sum((0, 1, 2, 3))
        g_h = rnd(g_h + conv3_input_grad(g_a, rnd(P.w1[bi])))
    f = cache["f"]
    grads["w_lift"] = torch.einsum("zijko,zijkq->oq", g_h, f)
    grads["b_lift"] = g_h.sum((0, 1, 2, 3))
    g_f = torch.einsum("zijko,oq->zijkq", g_h, rnd(P.w_lift))
    g_f[..., 1:4] += g_pred
    parts = [grads["w_lift"], grads["b_lift"]]
    for bi in range(P.b):
        parts += [gw1[bi], gb1[bi], gw2[bi], gb2[bi]]
    parts += [grads["w_proj"], grads["b_proj"]]
    flat = torch.cat([t.reshape(-1) for t in parts])
    return flat, g_f.reshape(g_f.shape[0], -1, CIN)


def loss_and_grad(frames, targets, P, n, rnd=bf16):
    """Loss, gradient w.r.t. the flat parameters (FP64), and the gradient
    w.r.t. the (rounded) input features, by the chain rule written out.
    targets: (B, n^3, 3)."""
    cache = forward(frames, P, n, rnd)
    pred = cache["pred"]
    tgt = torch.as_tensor(targets, dtype=DT).reshape(pred.shape)
    count = pred.numel()
    diff = pred - tgt
    L = float((diff ** 2).sum() / count)
    flat, g_f = backward_from(cache, 2.0 * diff / count, P, n, rnd)
    return L, flat, g_f


def input_vjp(frames, g_pred, P, n, rnd=bf16):
    """(d pred / d frame)^T g_pred, (B, nodes, 8)."""
    return backward_from(forward(frames, P, n, rnd), g_pred, P, n, rnd)[1]


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015, Algorithm 1) with bias
    correction, step index t >= 1; returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def relative_l2(pred, target):
    """||pred - target|| / ||target|| per frame."""
    pred = torch.as_tensor(pred, dtype=DT).reshape(pred.shape[0], -1)
    target = torch.as_tensor(target, dtype=DT).reshape(pred.shape)
    return (torch.linalg.norm(pred - target, dim=1) / torch.linalg.norm(target, dim=1)).numpy()
