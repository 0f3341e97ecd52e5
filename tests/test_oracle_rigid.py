"""Pins of the oracle's particle-represented rigid bodies (Sec. 3.2 "Rigid
body": elastic MLS-MPM, then an object-level rigid transformation fitted and
enforced): the polar factor against numpy's SVD and finite differences of it,
exact reproduction of a configuration that is already rigid, conservation of
the object's mass-weighted centroid and linear momentum, least-squares
optimality of the fitted rotation, exact free fall, a spinning block staying
rigid at the expected angle, and the gradient of a rollout with a rigid body
in liquid against finite differences."""
import numpy as np
import pytest
import torch

import scenes
from oracle import mpm
from oracle import rigid as rg

DT = torch.float64


def _rot(axis, angle):
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


def _polar_svd(A):
    U, _, Vt = np.linalg.svd(A)
    return U @ Vt


def test_polar_factor_matches_svd_and_is_a_rotation():
    rng = np.random.default_rng(0)
    for _ in range(20):
        A = rng.normal(size=(3, 3))
        if np.linalg.det(A) < 0:
            A[:, 0] *= -1.0
        R = rg.polar(torch.tensor(A, dtype=DT)).numpy()
        assert np.abs(R - _polar_svd(A)).max() < 1e-12
        assert np.abs(R.T @ R - np.eye(3)).max() < 1e-13
        assert abs(np.linalg.det(R) - 1.0) < 1e-13
        S = R.T @ A
        assert np.abs(S - S.T).max() < 1e-12 * np.abs(A).max()
        assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0.0
    # a scaled rotation and a matrix with repeated singular values
    R0 = _rot((1.0, 2.0, -0.5), 0.7)
    for A in (3.5 * R0, R0 @ np.diag([2.0, 2.0, 0.5])):
        assert np.abs(rg.polar(torch.tensor(A, dtype=DT)).numpy() - R0).max() < 1e-13


def test_polar_derivative_matches_finite_differences():
    rng = np.random.default_rng(1)
    # repeated singular values (an isotropic body) included: the polar factor
    # stays smooth there although the SVD's factors do not
    for A in (rng.normal(size=(3, 3)) + 2.0 * np.eye(3), 2.0 * _rot((0.3, 1.0, 0.2), 1.1)):
        At = torch.tensor(A, dtype=DT, requires_grad=True)
        G = torch.tensor(rng.normal(size=(3, 3)), dtype=DT)
        (rg.polar(At) * G).sum().backward()
        an = At.grad.numpy()
        h = 1e-6
        fd = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                E = np.zeros((3, 3))
                E[i, j] = h
                fd[i, j] = ((_polar_svd(A + E) - _polar_svd(A - E)) * G.numpy()).sum() / (2 * h)
        assert np.abs(an - fd).max() < 1e-8 * max(1.0, np.abs(fd).max())


def _pdist(x):
    """Pairwise distances by explicit differences (cdist's matrix-product
    form loses half the digits near zero)."""
    return (x[:, None, :] - x[None, :, :]).norm(dim=-1)


def _object(n=60, seed=2):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-0.05, 0.05, size=(n, 3)) * np.array([1.0, 0.6, 1.4])
    m = torch.tensor(rng.uniform(0.5, 1.5, size=n), dtype=DT)
    idx = torch.arange(n)
    rbar = rg.rest_offsets(X + 0.4, m, idx)
    return m, idx, rbar


def test_projection_reproduces_a_rigid_configuration():
    m, idx, rbar = _object()
    n = idx.shape[0]
    R0 = _rot((0.2, 1.0, -0.4), 0.9)
    c0 = np.array([0.45, 0.3, 0.52])
    x = torch.tensor(c0 + rbar.numpy() @ R0.T, dtype=DT)
    rng = np.random.default_rng(3)
    v = torch.tensor(rng.normal(size=(n, 3)), dtype=DT)
    C = torch.tensor(rng.normal(size=(n, 3, 3)), dtype=DT)
    F = torch.eye(3, dtype=DT).expand(n, 3, 3).clone()
    xn, vn, Cn, Fn, c, R = rg.project(x, v, C, F, m, 1e-4, idx, rbar)
    assert np.abs(R.numpy() - R0).max() < 1e-13
    assert np.abs(c.numpy() - c0).max() < 1e-15
    assert (xn - x).abs().max().item() < 1e-15
    assert (vn - v).abs().max().item() < 1e-9      # (x' - x) / dt with x' = x to round-off
    assert np.abs(Fn.numpy() - R0).max() < 1e-13
    # only the skew part of C survives
    assert (Cn + Cn.transpose(1, 2)).abs().max().item() < 1e-15
    assert (Cn - 0.5 * (C - C.transpose(1, 2))).abs().max().item() == 0.0


def test_projection_conserves_centroid_and_momentum_and_is_rigid():
    m, idx, rbar = _object(seed=4)
    n = idx.shape[0]
    rng = np.random.default_rng(5)
    R0 = _rot((1.0, 0.1, 0.3), 0.4)
    x = torch.tensor(0.5 + rbar.numpy() @ R0.T + 0.01 * rng.normal(size=(n, 3)), dtype=DT)
    v = torch.tensor(rng.normal(size=(n, 3)), dtype=DT)
    C = torch.zeros(n, 3, 3, dtype=DT)
    F = torch.eye(3, dtype=DT).expand(n, 3, 3).clone()
    dt = 1e-3
    xn, vn, _, _, c, R = rg.project(x, v, C, F, m, dt, idx, rbar)
    M = m.sum()
    assert ((m[:, None] * xn).sum(0) - (m[:, None] * x).sum(0)).abs().max().item() < 1e-15 * M.item() * 4
    mom0 = (m[:, None] * v).sum(0)
    assert ((m[:, None] * vn).sum(0) - mom0).abs().max().item() < 1e-9 * mom0.abs().max().item()
    # pairwise distances are those of the rest shape
    assert (_pdist(xn) - _pdist(rbar)).abs().max().item() < 1e-15 * 8


def test_fitted_rotation_minimises_the_weighted_squared_distance():
    """Shape matching: no nearby rotation fits the particles better."""
    m, idx, rbar = _object(seed=6)
    n = idx.shape[0]
    rng = np.random.default_rng(7)
    R0 = _rot((0.5, -1.0, 0.2), 1.3)
    x = torch.tensor(0.5 + rbar.numpy() @ R0.T + 0.02 * rng.normal(size=(n, 3)), dtype=DT)
    F = torch.eye(3, dtype=DT).expand(n, 3, 3).clone()
    _, _, _, _, c, R = rg.project(x, x, torch.zeros(n, 3, 3, dtype=DT), F, m, 1.0, idx, rbar)

    def obj(Rm):
        r = x.numpy() - c.numpy() - rbar.numpy() @ Rm.T
        return float((m.numpy()[:, None] * r ** 2).sum())

    best = obj(R.numpy())
    for k in range(30):
        ax = rng.normal(size=3)
        for eps in (1e-2, 1e-4):
            assert obj(R.numpy() @ _rot(ax, eps)) >= best
            assert obj(_rot(ax, eps) @ R.numpy()) >= best


def test_rigid_block_free_fall_is_exact():
    sc = scenes.small_block(31, 16, [scenes.RIGID], ppc=2, size_cells=4, lo_cell=(6, 6, 6), n_steps=10,
                            dt=2e-4, bound=0)
    x0 = torch.tensor(sc.x, dtype=DT)
    x, v, C, F = mpm.rollout(sc)
    n, dt = sc.n_steps, sc.dt
    g = np.array(sc.gravity)
    # the velocity update (x' - x) / dt turns the rounding of x (~1e-16 * |x|)
    # into ~1e-13 of velocity per step
    v_tol = n * 20.0 * np.finfo(np.float64).eps * float(np.abs(sc.x).max()) / dt
    assert np.abs(v.numpy() - n * dt * g).max() < v_tol
    assert np.abs(x.numpy() - (x0.numpy() + g * dt * dt * n * (n + 1) / 2)).max() < 1e-13
    assert np.abs(C.numpy()).max() < 1e-10
    assert np.abs(F.numpy() - np.eye(3)).max() < 1e-13


def test_spinning_rigid_block_stays_rigid_and_turns_at_its_carried_rate():
    """A spinning block (v = omega (r_z, 0, -r_x), C = 0 at the start) stays
    rigid; every particle carries the object's rotation about +y, which turns
    at the angular rate the particles' affine velocity C carries (the first
    transfers from C = 0 settle that rate below omega, an APIC property)."""
    omega, n_steps, dt = 20.0, 40, 2e-4
    sc = scenes.small_block(32, 16, [scenes.RIGID], ppc=4, size_cells=4, lo_cell=(6, 6, 6), n_steps=n_steps,
                            dt=dt, spin=omega, gravity=(0.0, 0.0, 0.0), bound=0)
    x0 = torch.tensor(sc.x, dtype=DT)
    states = mpm.rollout(sc, keep_states=True)
    x, v, C, F = states[-1]
    assert (_pdist(x) - _pdist(x0)).abs().max().item() < 1e-13

    def angle(Fs):
        R = Fs[0].numpy()
        assert np.abs(Fs.numpy() - R).max() < 1e-14
        # about y up to the slight wobble of the jittered (not exactly symmetric) body
        assert np.abs(R - _rot((0.0, 1.0, 0.0), np.arctan2(R[0, 2], R[0, 0]))).max() < 2e-3
        return np.arctan2(R[0, 2], R[0, 0])

    rate = np.mean([float(s[2][0, 0, 2]) for s in states[11:]])
    assert 0.7 * omega < rate < omega
    turned = angle(F) - angle(states[10][3])
    assert abs(turned - rate * 30 * dt) < 2e-3 * rate * 30 * dt
    # C keeps each particle's skew part of the G2P velocity gradient: skew
    # exactly, and close to the common rotation rate on every particle
    assert float((C + C.transpose(1, 2)).abs().max()) == 0.0
    assert float((C - C[0]).abs().max()) < 1e-3 * rate


@pytest.mark.parametrize("kinds", [[5], [0, 5]])
def test_rollout_gradient_with_rigid_body(kinds):
    sc = scenes.small_block(33, 12, kinds, ppc=2, size_cells=4, lo_cell=(4, 3, 4), n_steps=12,
                            v0=(0.2, -0.3, 0.1), spin=8.0, dt=2e-4)
    x0 = torch.tensor(sc.x, dtype=DT)
    v0 = torch.tensor(sc.v, dtype=DT)

    def f(x, v):
        xs, vs, C, F = mpm.rollout(sc, x0=x, v0=v)
        return mpm.scene_loss(sc, xs) + 0.1 * (vs ** 2).sum() + (F ** 2).sum()

    rng = np.random.default_rng(8)
    ps = [x0.clone().requires_grad_(True), v0.clone().requires_grad_(True)]
    L = f(*ps)
    grads = torch.autograd.grad(L, ps)
    h = 1e-7
    for _ in range(3):
        us = [torch.tensor(rng.normal(size=p.shape), dtype=DT) for p in (x0, v0)]
        an = sum((g * u).sum() for g, u in zip(grads, us)).item()
        with torch.no_grad():
            fd = (f(x0 + h * us[0], v0 + h * us[1]) - f(x0 - h * us[0], v0 - h * us[1])).item() / (2 * h)
        assert abs(an - fd) <= 2e-5 * max(abs(fd), 1e-8 * abs(L.item())), (an, fd)
