"""Pins of the gradient-sharing oracle (Sec. 5.1) against what the definition
and the mathematics fix: a two-particle closed form, brute force with Python
loops over pairs, torch.autograd of the loss, translation / rotation
invariance, zero net force, compact support, scene separation, linearity."""
import math

import numpy as np
import pytest
import torch

from oracle import sharing as S

H, TAU = 0.05, 0.5


def _cloud(seed, n=40, scenes=1):
    rng = np.random.default_rng(seed)
    x = 0.4 + 0.1 * rng.random((n, 3))
    scene = np.repeat(np.arange(scenes), n // scenes + 1)[:n]
    ell = rng.random(n)
    return x, scene, ell


def _loops(x, scene, ell, h, tau):
    total = 0.0
    for a in range(len(x)):
        for j in range(len(x)):
            if j == a or scene[a] != scene[j]:
                continue
            d = math.dist(x[a], x[j])
            if 0.0 < d < h:
                total += math.exp(-ell[j] / tau) * d * (1.0 - (d / h) ** 2) ** 3
    return total


def test_kernel_values_and_support():
    r = torch.tensor([0.0, 0.5, 0.999999, 1.0, 1.7], dtype=torch.float64)
    k = S.kernel_k(r)
    assert k[0] == 1.0 and abs(k[1] - 0.421875) < 1e-15 and k[3] == 0.0 and k[4] == 0.0
    assert abs(k[2]) < 1e-15
    # k is C^1 at r = 1 and k' is its derivative
    rr = torch.linspace(0.05, 0.95, 19, dtype=torch.float64)
    fd = (S.kernel_k(rr + 1e-6) - S.kernel_k(rr - 1e-6)) / 2e-6
    assert torch.allclose(fd, S.kernel_dk(rr), atol=1e-8)
    assert abs(S.kernel_dk(torch.tensor(0.9999999, dtype=torch.float64))) < 1e-10


def test_two_particles_closed_form():
    d = 0.03
    x = np.array([[0.5, 0.5, 0.5], [0.5 + d * 0.6, 0.5 + d * 0.8, 0.5]])
    ell = np.array([0.2, 1.3])
    c = np.exp(-ell / TAU)
    r = d / H
    phi = d * (1 - r * r) ** 3
    L = float(S.attraction_loss(x, [0, 0], ell, H, TAU))
    assert abs(L - (c[0] + c[1]) * phi) < 1e-14
    dphi = (1 - r * r) ** 3 - 6 * r * r * (1 - r * r) ** 2
    u = (x[0] - x[1]) / d
    g = S.attraction_grad(x, [0, 0], ell, H, TAU).numpy()
    assert np.allclose(g[0], (c[0] + c[1]) * dphi * u, atol=1e-13)
    assert np.allclose(g[1], -(c[0] + c[1]) * dphi * u, atol=1e-13)


def test_loss_matches_pairwise_loops():
    x, scene, ell = _cloud(1, n=30, scenes=2)
    L = float(S.attraction_loss(x, scene, ell, H, TAU))
    assert L > 0.0
    assert abs(L - _loops(x, scene, ell, H, TAU)) < 1e-12 * max(1.0, L)


def test_gradient_matches_autograd():
    x, scene, ell = _cloud(2, n=36, scenes=2)
    xt = torch.tensor(x, dtype=torch.float64, requires_grad=True)
    L = S.attraction_loss(xt, scene, ell, H, TAU)
    (g_auto,) = torch.autograd.grad(L, xt)
    g = S.attraction_grad(x, scene, ell, H, TAU)
    assert torch.allclose(g, g_auto, rtol=1e-10, atol=1e-12)


def test_gradient_matches_finite_differences():
    x, scene, ell = _cloud(3, n=20)
    g = S.attraction_grad(x, scene, ell, H, TAU).numpy()
    eps = 1e-7
    for a, k in [(0, 0), (3, 1), (7, 2), (11, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[a, k] += eps
        xm[a, k] -= eps
        fd = (float(S.attraction_loss(xp, scene, ell, H, TAU)) - float(S.attraction_loss(xm, scene, ell, H, TAU))) / (2 * eps)
        assert abs(fd - g[a, k]) < 1e-6 * max(1.0, abs(g[a, k]))


def test_invariances_and_zero_net_force():
    x, scene, ell = _cloud(4, n=32)
    L0 = float(S.attraction_loss(x, scene, ell, H, TAU))
    assert abs(float(S.attraction_loss(x + np.array([0.01, -0.02, 0.005]), scene, ell, H, TAU)) - L0) < 1e-12
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    assert abs(float(S.attraction_loss(x @ R.T, scene, ell, H, TAU)) - L0) < 1e-12
    g = S.attraction_grad(x, scene, ell, H, TAU)
    assert float(g.sum(0).abs().max()) < 1e-12  # depends on differences only


def test_scenes_do_not_interact_and_support_is_compact():
    x, _, ell = _cloud(5, n=24)
    both = S.attraction_loss(np.concatenate([x, x]), [0] * 24 + [1] * 24, np.concatenate([ell, ell]), H, TAU)
    one = S.attraction_loss(x, [0] * 24, ell, H, TAU)
    assert abs(float(both) - 2 * float(one)) < 1e-12
    far = np.array([[0.2, 0.2, 0.2], [0.2 + 1.001 * H, 0.2, 0.2], [0.2, 0.2 + 1.5 * H, 0.2]])
    assert float(S.attraction_loss(far, [0, 0, 0], [0.0, 0.0, 0.0], H, TAU)) == 0.0


def test_share_gradients_special_cases():
    x, scene, ell = _cloud(6, n=25, scenes=1)
    rng = np.random.default_rng(7)
    g = rng.normal(size=(25, 3))
    c = np.exp(-ell / TAU)
    # no neighbours within a tiny radius: each particle keeps c_a g_a
    assert np.allclose(S.share_gradients(x, scene, ell, 1e-9, TAU, g).numpy(), c[:, None] * g, atol=1e-14)
    # brute force with loops
    out = S.share_gradients(x, scene, ell, H, TAU, g).numpy()
    for a in (0, 9, 24):
        ref = np.zeros(3)
        for j in range(25):
            d = math.dist(x[a], x[j])
            if d < H:
                ref += c[j] * (1 - (d / H) ** 2) ** 3 * g[j]
        assert np.allclose(out[a], ref, atol=1e-13)
    # linear in g
    g2 = rng.normal(size=(25, 3))
    lhs = S.share_gradients(x, scene, ell, H, TAU, 2.0 * g - g2).numpy()
    assert np.allclose(lhs, 2.0 * out - S.share_gradients(x, scene, ell, H, TAU, g2).numpy(), atol=1e-13)
