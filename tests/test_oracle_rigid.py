"""Pins of the oracle's particle-represented rigid bodies (Sec. 3.2 "Rigid
body": elastic MLS-MPM, then an object-level rigid transformation fitted and
enforced): the polar factor against numpy's SVD and finite differences of it,
exact reproduction of a motion that is already rigid, conservation of the
object's centroid, linear momentum and angular momentum, least-squares
optimality of the fitted rotation and rigid velocity field, exact free fall,
a spinning block staying rigid and turning at its carried spin, and the
gradient of a rollout with a rigid body in liquid against finite
differences."""
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


def _state(n):
    C = torch.zeros(n, 3, 3, dtype=DT)
    F = torch.eye(3, dtype=DT).expand(n, 3, 3).clone()
    return C, F


def test_projection_reproduces_a_rigid_motion():
    """Particles already on a rigid placement with a rigid velocity field are
    left unchanged; the fit recovers the rotation, centroid and spin."""
    m, idx, rbar = _object()
    n = idx.shape[0]
    R0 = _rot((0.2, 1.0, -0.4), 0.9)
    c0 = np.array([0.45, 0.3, 0.52])
    u0, w0 = np.array([0.3, -1.2, 0.5]), np.array([4.0, -2.0, 7.0])
    r0 = rbar.numpy() @ R0.T
    x = torch.tensor(c0 + r0, dtype=DT)
    v = torch.tensor(u0 + np.cross(w0, r0), dtype=DT)
    rng = np.random.default_rng(3)
    C = torch.tensor(rng.normal(size=(n, 3, 3)), dtype=DT)
    _, F = _state(n)
    xn, vn, Cn, Fn, c, R, w = rg.project(x, v, C, F, m, idx, rbar)
    assert np.abs(R.numpy() - R0).max() < 1e-13
    assert np.abs(c.numpy() - c0).max() < 1e-15
    assert np.abs(w.numpy() - w0).max() < 1e-11
    assert (xn - x).abs().max().item() < 1e-15
    assert (vn - v).abs().max().item() < 1e-12
    assert np.abs(Fn.numpy() - R0).max() < 1e-13
    K = np.array([[0, -w0[2], w0[1]], [w0[2], 0, -w0[0]], [-w0[1], w0[0], 0]])
    assert np.abs(Cn.numpy() - K).max() < 1e-11


def test_projection_conserves_centroid_momenta_and_is_rigid():
    m, idx, rbar = _object(seed=4)
    n = idx.shape[0]
    rng = np.random.default_rng(5)
    R0 = _rot((1.0, 0.1, 0.3), 0.4)
    x = torch.tensor(0.5 + rbar.numpy() @ R0.T + 0.01 * rng.normal(size=(n, 3)), dtype=DT)
    v = torch.tensor(rng.normal(size=(n, 3)), dtype=DT)
    C, F = _state(n)
    xn, vn, _, _, c, R, w = rg.project(x, v, C, F, m, idx, rbar)
    M = m.sum().item()
    mx = lambda a: (m[:, None] * a).sum(0)
    assert (mx(xn) - mx(x)).abs().max().item() < 4e-16 * M
    assert (mx(vn) - mx(v)).abs().max().item() < 1e-14 * M
    # angular momentum about c with the projected lever arms
    r = xn - c
    L0 = (m[:, None] * torch.linalg.cross(r, v)).sum(0)
    L1 = (m[:, None] * torch.linalg.cross(r, vn)).sum(0)
    assert (L1 - L0).abs().max().item() < 1e-12 * L0.abs().max().item()
    # pairwise distances are those of the rest shape
    assert (_pdist(xn) - _pdist(rbar)).abs().max().item() < 1e-15 * 8


def test_fitted_motion_is_the_weighted_least_squares_one():
    """Shape matching: no nearby rotation fits the positions better, and no
    nearby rigid velocity field fits the velocities better."""
    m, idx, rbar = _object(seed=6)
    n = idx.shape[0]
    rng = np.random.default_rng(7)
    R0 = _rot((0.5, -1.0, 0.2), 1.3)
    x = torch.tensor(0.5 + rbar.numpy() @ R0.T + 0.02 * rng.normal(size=(n, 3)), dtype=DT)
    v = torch.tensor(rng.normal(size=(n, 3)), dtype=DT)
    C, F = _state(n)
    _, vn, _, _, c, R, w = rg.project(x, v, C, F, m, idx, rbar)
    mm = m.numpy()[:, None]

    def obj_x(Rm):
        return float((mm * (x.numpy() - c.numpy() - rbar.numpy() @ Rm.T) ** 2).sum())

    r = rbar.numpy() @ R.numpy().T
    vbar = (vn.numpy() - np.cross(w.numpy(), r))[0]

    def obj_v(a, om):
        return float((mm * (v.numpy() - a - np.cross(om, r)) ** 2).sum())

    best_x, best_v = obj_x(R.numpy()), obj_v(vbar, w.numpy())
    for k in range(30):
        ax = rng.normal(size=3)
        for eps in (1e-2, 1e-4):
            assert obj_x(R.numpy() @ _rot(ax, eps)) >= best_x
            assert obj_x(_rot(ax, eps) @ R.numpy()) >= best_x
            assert obj_v(vbar + eps * ax, w.numpy()) >= best_v
            assert obj_v(vbar, w.numpy() + eps * ax) >= best_v


def test_rigid_block_free_fall_is_exact():
    sc = scenes.small_block(31, 16, [scenes.RIGID], ppc=2, size_cells=4, lo_cell=(6, 6, 6), n_steps=10,
                            dt=2e-4, bound=0)
    x0 = torch.tensor(sc.x, dtype=DT)
    x, v, C, F = mpm.rollout(sc)
    n, dt = sc.n_steps, sc.dt
    g = np.array(sc.gravity)
    assert np.abs(v.numpy() - n * dt * g).max() < 1e-13
    assert np.abs(x.numpy() - (x0.numpy() + g * dt * dt * n * (n + 1) / 2)).max() < 1e-13
    assert np.abs(C.numpy()).max() < 1e-10
    assert np.abs(F.numpy() - np.eye(3)).max() < 1e-13


def test_spinning_rigid_block_stays_rigid_and_turns_at_its_spin_rate():
    """A spinning block (v = omega (r_z, 0, -r_x) about the block centre, C = 0
    at the start) stays rigid; every particle carries the object's rotation
    about +y, which turns at the spin the velocities carry."""
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

    # C = [w]_x on every particle; w_y = C[0, 2]
    rates = [float(s[2][0, 0, 2]) for s in states[1:]]
    assert all(float((s[2] - s[2][0]).abs().max()) == 0.0 for s in states[1:])
    assert 0.5 * omega < rates[0] < omega  # the first transfer from C = 0 loses some spin
    assert np.std(rates[1:]) < 1e-2 * np.mean(rates[1:])
    turned = angle(F) - angle(states[10][3])
    assert abs(turned - sum(rates[10:]) * dt) < 1e-3 * turned


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
