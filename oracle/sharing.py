"""Oracle of gradient sharing within fluid bodies and its attraction-loss
approximation (Sec. 5.1, "Gradient Sharing within Fluid Bodies").

TEST INFRASTRUCTURE ONLY: the product never imports it; tests, smoke() and
bench.py's CPU legs do. Plain torch FP64 on the CPU, brute force over all
particle pairs of a scene (O(N^2): small cases only).

The paper shares per-particle gradients between neighbouring particles of a
fluid body, weighting neighbour j by a kernel w(L_j, d_ij) of its loss at the
previous iteration (a lower loss gets a higher weight) and of the distance
d_ij, and approximates the sharing in practice by an attraction loss
    L_att = sum_i sum_j w(L_j, d_ij) |p_i - p_j|.
The paper does not give w. Reading used here (also in the CUDA library):
    w(L_j, d) = c_j k(d / h),   c_j = exp(-L_j / tau),
    k(r) = (1 - r^2)^3 for 0 <= r < 1, else 0,
with a radius h (at most one grid spacing) and a loss scale tau. k is C^1 at
the edge of its support (k(1) = k'(1) = 0), so L_att is differentiable in the
positions. Particles interact only within their own scene. A particle's own
term (j = i) is zero in L_att (distance 0); the shared gradient includes it
(k(0) = 1).

With phi(d) = d k(d / h):
    L_att       = sum_a sum_{j != a} c_j phi(d_aj)
    dL_att/dp_a = sum_{j != a} (c_j + c_a) phi'(d_aj) (p_a - p_j) / d_aj,
    phi'(d)     = k(r) + r k'(r),  r = d / h,  k'(r) = -6 r (1 - r^2)^2,
(pairs at distance 0 are left out of both sums). The gradient formula is
pinned against torch.autograd of the loss in tests/test_oracle_sharing.py.
    shared g'_a = sum_j c_j k(d_aj / h) g_j   (j over a's scene, j = a included)
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64


def _t(a):
    if isinstance(a, torch.Tensor):
        return a.to(DT)
    return torch.tensor(np.asarray(a), dtype=DT)


def kernel_k(r):
    """k(r) = (1 - r^2)^3 on [0, 1), 0 beyond."""
    r = _t(r)
    inside = r < 1.0
    return torch.where(inside, (1.0 - r * r) ** 3, torch.zeros_like(r))


def kernel_dk(r):
    """k'(r) = -6 r (1 - r^2)^2 on [0, 1), 0 beyond."""
    r = _t(r)
    inside = r < 1.0
    return torch.where(inside, -6.0 * r * (1.0 - r * r) ** 2, torch.zeros_like(r))


def weights_c(ell, tau):
    """c_j = exp(-L_j / tau): neighbours with a lower loss weigh more."""
    return torch.exp(-_t(ell) / float(tau))


def _pairs(x, scene):
    """Pairwise differences p_a - p_j, distances and the same-scene mask."""
    x = _t(x)
    scene = torch.as_tensor(np.asarray(scene))
    diff = x[:, None, :] - x[None, :, :]
    d2 = (diff * diff).sum(-1)
    # sqrt only of positive squares, so that autograd stays finite at d = 0
    d = torch.where(d2 > 0.0, torch.sqrt(torch.where(d2 > 0.0, d2, torch.ones_like(d2))), torch.zeros_like(d2))
    same = scene[:, None] == scene[None, :]
    return diff, d, same


def attraction_loss(x, scene, ell, h, tau):
    """L_att = sum_a sum_{j != a, same scene} c_j phi(d_aj) as a differentiable
    torch expression of x (FP64)."""
    x = _t(x)
    c = weights_c(ell, tau)
    diff, d, same = _pairs(x, scene)
    mask = same & (d > 0.0) & (d < h)
    dd = torch.where(mask, d, torch.ones_like(d))  # keep sqrt's gradient finite off the mask
    phi = torch.where(mask, dd * kernel_k(dd / h), torch.zeros_like(d))
    return (phi * c[None, :]).sum()


def attraction_grad(x, scene, ell, h, tau):
    """dL_att/dp_a by the closed form in the module docstring, (N, 3) FP64."""
    x = _t(x)
    c = weights_c(ell, tau)
    diff, d, same = _pairs(x, scene)
    mask = same & (d > 0.0) & (d < h)
    dd = torch.where(mask, d, torch.ones_like(d))
    r = dd / h
    dphi = kernel_k(r) + r * kernel_dk(r)
    coef = torch.where(mask, (c[None, :] + c[:, None]) * dphi / dd, torch.zeros_like(d))
    return (coef[:, :, None] * diff).sum(1)


def share_gradients(x, scene, ell, h, tau, g):
    """g'_a = sum_{j in a's scene} c_j k(d_aj / h) g_j (j = a included), (N, 3)."""
    x = _t(x)
    g = _t(g)
    c = weights_c(ell, tau)
    _, d, same = _pairs(x, scene)
    w = torch.where(same, kernel_k(d / h), torch.zeros_like(d)) * c[None, :]
    return w @ g

