"""Pins of the oracle's transfer stages (Sec. 3.2, MLS-MPM) to closed forms.

Each test checks a fact that the quadratic B-spline MLS-MPM scheme fixes
exactly, so a dropped term, a wrong sign or a transposed operand in the oracle
fails one of them.
"""
import numpy as np
import pytest
import torch

import scenes
from oracle import mpm

DT = torch.float64


def _model(n=16, dt=1e-4, bound=0, gravity=(0.0, 0.0, 0.0), kinds=(0,)):
    sc = scenes.small_block(0, n, list(kinds), gravity=gravity, bound=bound, dt=dt)
    return sc, mpm.Model(sc)


def _rand_x(rng, N, n):
    return torch.tensor(rng.uniform(0.3, 0.7, (N, 3)), dtype=DT)


def test_bspline_moments():
    """Sum W = 1, sum W (x_i - x_p) = 0, sum W (x_i - x_p)(x_i - x_p)^T = dx^2/4 I."""
    rng = np.random.default_rng(0)
    sc, model = _model()
    x = _rand_x(rng, 500, model.n)
    W, dpos, _ = mpm.stencil(x, model)
    assert torch.allclose(W.sum(1), torch.ones(500, dtype=DT), atol=1e-14)
    assert torch.allclose((W[..., None] * dpos).sum(1), torch.zeros(500, 3, dtype=DT), atol=1e-16)
    M2 = torch.einsum("po,poi,poj->pij", W, dpos, dpos)
    ref = (model.dx ** 2 / 4.0) * torch.eye(3, dtype=DT).expand(500, 3, 3)
    assert torch.allclose(M2, ref, atol=1e-17, rtol=1e-12)


def test_bspline_weights_closed_form():
    """At f = 1 (particle on a node) the 1D weights are (1/8, 3/4, 1/8)."""
    sc, model = _model()
    x = torch.tensor([[5.0, 6.0, 7.0]], dtype=DT) * model.dx
    W, dpos, lin = mpm.stencil(x, model)
    w1 = torch.tensor([0.125, 0.75, 0.125], dtype=DT)
    ref = (w1[:, None, None] * w1[None, :, None] * w1[None, None, :]).reshape(-1)
    assert torch.allclose(W[0], ref, atol=1e-15)
    # base node is (4, 5, 6)
    assert int(lin[0, 0]) == (4 * model.n + 5) * model.n + 6


def test_p2g_conserves_mass_and_momentum():
    """sum_i m_i = sum_p m_p and sum_i mv_i = sum_p m_p v_p: the affine and
    stress terms of MLS-MPM have zero sum by the first-moment identity."""
    rng = np.random.default_rng(1)
    sc, model = _model(kinds=(0, 1, 2))
    N = 300
    x = _rand_x(rng, N, model.n)
    v = torch.tensor(rng.normal(size=(N, 3)), dtype=DT)
    C = torch.tensor(rng.normal(size=(N, 3, 3)), dtype=DT)
    tau = torch.tensor(rng.normal(size=(N, 3, 3)) * 1e3, dtype=DT)
    tau = tau + tau.transpose(1, 2)
    mass = torch.tensor(rng.uniform(0.5, 2.0, N), dtype=DT)
    vol = torch.tensor(rng.uniform(0.5, 2.0, N), dtype=DT)
    m, mv = mpm.p2g(x, v, C, tau, mass, vol, model)
    assert abs(m.sum().item() - mass.sum().item()) <= 1e-14 * mass.sum().item()
    P = (mass[:, None] * v).sum(0)
    assert torch.allclose(mv.sum(0), P, atol=1e-12 * P.abs().max().item() + 1e-12)


def test_p2g_single_particle_nodes():
    """One particle on a node: node masses are m_p times the tensor weights and
    the node momentum carries the affine term A (x_i - x_p)."""
    sc, model = _model()
    x = torch.tensor([[8.0, 8.0, 8.0]], dtype=DT) * model.dx
    v = torch.tensor([[1.0, -2.0, 0.5]], dtype=DT)
    C = torch.zeros(1, 3, 3, dtype=DT)
    C[0, 0, 1] = 3.0
    tau = torch.zeros(1, 3, 3, dtype=DT)
    mass = torch.tensor([2.0], dtype=DT)
    vol = torch.tensor([1.0], dtype=DT)
    m, mv = mpm.p2g(x, v, C, tau, mass, vol, model)
    n = model.n
    lin = lambda i, j, k: (i * n + j) * n + k
    assert m[lin(8, 8, 8)].item() == pytest.approx(2.0 * 0.75 ** 3, rel=1e-14)
    # node (8, 9, 8): dpos = (0, dx, 0); momentum = W (m v + m C dpos), (C dpos)_x = 3 dx
    W = 0.75 * 0.125 * 0.75
    ref = W * 2.0 * (v[0] + torch.tensor([3.0 * model.dx, 0.0, 0.0], dtype=DT))
    assert torch.allclose(mv[lin(8, 9, 8)], ref, rtol=1e-13)


def test_p2g_stress_term_sign():
    """A compressed liquid particle (J < 1, tau = K J (J-1) I < 0) pushes its
    neighbour nodes outward: the +x node gets +x momentum."""
    sc, model = _model()
    x = torch.tensor([[8.0, 8.0, 8.0]], dtype=DT) * model.dx
    tau = -1e3 * torch.eye(3, dtype=DT)[None]
    z = torch.zeros(1, 3, dtype=DT)
    m, mv = mpm.p2g(x, z, torch.zeros(1, 3, 3, dtype=DT), tau, torch.ones(1, dtype=DT),
                    torch.ones(1, dtype=DT), model)
    n = model.n
    # A = -dt V 4/dx^2 tau = +dt 4/dx^2 1e3 I (positive), node at +dx in x
    assert mv[(9 * n + 8) * n + 8, 0].item() > 0.0
    assert mv[(7 * n + 8) * n + 8, 0].item() < 0.0


def test_g2p_affine_reproduction():
    """Grid velocity v_i = v0 + G x_i gives v_p = v0 + G x_p and C_p = G exactly."""
    rng = np.random.default_rng(2)
    sc, model = _model()
    n = model.n
    G = torch.tensor(rng.normal(size=(3, 3)), dtype=DT)
    v0 = torch.tensor(rng.normal(size=3), dtype=DT)
    idx = torch.arange(n ** 3)
    _, xi = mpm.node_positions(idx, model)
    vg = v0 + xi @ G.T
    x = _rand_x(rng, 200, n)
    Fp = torch.eye(3, dtype=DT).expand(200, 3, 3).clone()
    x1, v1, C1, F1 = mpm.g2p(x, Fp, vg, model)
    assert torch.allclose(v1, v0 + x @ G.T, atol=1e-13)
    assert torch.allclose(C1, G.expand(200, 3, 3), atol=1e-11)
    assert torch.allclose(x1, x + model.dt * v1, atol=1e-16)
    assert torch.allclose(F1, (torch.eye(3, dtype=DT) + model.dt * G).expand(200, 3, 3), atol=1e-14)


def test_rigid_rotation_keeps_F_orthogonal_to_second_order():
    """A rigid spin field (G skew) advances F by (I + dt G), which stays a
    rotation up to O(dt^2) per step: |F^T F - I| ~ (dt |G|)^2."""
    sc, model = _model()
    n = model.n
    w = 5.0
    G = torch.tensor([[0.0, -w, 0.0], [w, 0.0, 0.0], [0.0, 0.0, 0.0]], dtype=DT)
    _, xi = mpm.node_positions(torch.arange(n ** 3), model)
    vg = xi @ G.T
    x = torch.full((1, 3), 0.5, dtype=DT)
    F = torch.eye(3, dtype=DT)[None]
    _, _, _, F1 = mpm.g2p(x, F, vg, model)
    err = (F1[0].T @ F1[0] - torch.eye(3, dtype=DT)).abs().max().item()
    assert err == pytest.approx((model.dt * w) ** 2, rel=1e-6)


def test_domain_error():
    sc, model = _model()
    x = torch.tensor([[0.2 * model.dx, 0.5, 0.5]], dtype=DT)
    with pytest.raises(mpm.DomainError):
        mpm.stencil(x, model)
