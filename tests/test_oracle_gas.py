"""Pins of the gas-solver oracle (Sec. 3.2 "Gas", Stam 1999): interpolation
and advection exactness cases, the symmetry of the fixed-sweep Poisson solver
and the projection's limit against a direct sparse least-squares solve of the
same Poisson system (scipy), solid cells, buoyancy, and autograd against
finite differences."""
import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.linalg
import torch

from oracle import gas as G

DT = torch.float64


def _box_solid(n, obstacle=False):
    s = np.zeros((n, n, n), dtype=bool)
    s[0, :, :] = s[-1, :, :] = s[:, 0, :] = s[:, -1, :] = s[:, :, 0] = s[:, :, -1] = True
    if obstacle:
        c = n // 2
        s[c - 1:c + 1, c - 1:c + 1, c:c + 2] = True
    return s


def test_trilinear_reproduces_linear_fields():
    n = 7
    idx = torch.arange(n, dtype=DT)
    I = torch.stack(torch.meshgrid(idx, idx, idx, indexing="ij"))
    q = 0.3 + 1.1 * I[0] - 0.7 * I[1] + 0.25 * I[2]
    rng = np.random.default_rng(0)
    X = torch.tensor(rng.uniform(0.0, n - 1.0, size=(3, n, n, n)), dtype=DT)
    ref = 0.3 + 1.1 * X[0] - 0.7 * X[1] + 0.25 * X[2]
    assert torch.allclose(G.trilinear(q, X), ref, atol=1e-12)


def test_advection_identity_shift_and_constant():
    n, dx, dt = 8, 1.0 / 8, 0.01
    rng = np.random.default_rng(1)
    q = torch.tensor(rng.normal(size=(n, n, n)), dtype=DT)
    zero = torch.zeros(3, n, n, n, dtype=DT)
    assert torch.allclose(G.advect(q, zero, dt, dx), q, atol=1e-14)
    # a uniform velocity of exactly one cell per step along x moves the field by one cell
    u = torch.zeros(3, n, n, n, dtype=DT)
    u[0] = dx / dt
    out = G.advect(q, u, dt, dx)
    assert torch.allclose(out[1:], q[:-1], atol=1e-12)
    # a constant field stays constant under any velocity (clamped sampling)
    c = torch.full((n, n, n), 2.5, dtype=DT)
    uu = torch.tensor(rng.normal(size=(3, n, n, n)), dtype=DT) * 3.0
    assert torch.allclose(G.advect(c, uu, dt, dx), c, atol=1e-13)


def _laplacian_matrix(fluid):
    n = fluid.shape[0]
    ids = -np.ones(fluid.shape, dtype=int)
    cells = np.argwhere(fluid)
    ids[tuple(cells.T)] = np.arange(len(cells))
    rows, cols, vals = [], [], []
    for r, (i, j, k) in enumerate(cells):
        deg = 0
        for d in range(3):
            for s in (-1, 1):
                q = [i, j, k]
                q[d] += s
                if 0 <= q[d] < n and fluid[tuple(q)]:
                    rows.append(r)
                    cols.append(ids[tuple(q)])
                    vals.append(1.0)
                    deg += 1
        rows.append(r)
        cols.append(r)
        vals.append(-float(deg))
    return scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(len(cells), len(cells))), cells


@pytest.mark.parametrize("obstacle", [False, True])
def test_projection_limit_matches_direct_solve(obstacle):
    """Many Jacobi sweeps converge (in u, which only sees grad p) to the
    projection with the least-squares solution of the same Poisson system."""
    n = 8
    dx = 1.0 / n
    solid = _box_solid(n, obstacle)
    fluid = G.fluid_of(solid)
    rng = np.random.default_rng(2)
    u = torch.tensor(rng.normal(size=(3, n, n, n)), dtype=DT) * fluid.to(DT)
    b = G.remove_mean(G.divergence(u, fluid, dx), fluid)
    A, cells = _laplacian_matrix(fluid.numpy())
    rhs = (dx * dx * b.numpy())[tuple(cells.T)]
    x = scipy.sparse.linalg.lsqr(A, rhs, atol=1e-14, btol=1e-14, iter_lim=20000)[0]
    p = np.zeros((n, n, n))
    p[tuple(cells.T)] = x
    u_direct = u - G.gradient(torch.tensor(p, dtype=DT), fluid, dx)
    assert np.linalg.norm(A @ x - rhs) < 1e-10 * np.linalg.norm(rhs)  # consistent system
    u_jac = G.project(u, fluid, dx, 4000)
    assert float((u_jac - u_direct).norm() / u_direct.norm()) < 1e-9


def test_fixed_sweep_solver_is_symmetric_and_projection_linear():
    """J_K (K damped Jacobi sweeps from 0) is a symmetric linear map, so the
    adjoint of the projection can run the same sweeps on its own right-hand
    side; the projection is linear in u."""
    n, K = 8, 30
    dx = 1.0 / n
    fluid = G.fluid_of(_box_solid(n, True))
    f = fluid.to(DT)
    rng = np.random.default_rng(3)
    b = torch.tensor(rng.normal(size=(n, n, n)), dtype=DT) * f
    c = torch.tensor(rng.normal(size=(n, n, n)), dtype=DT) * f
    Jb, Jc = G.jacobi(b, fluid, dx, K), G.jacobi(c, fluid, dx, K)
    assert abs(float((Jb * c).sum() - (b * Jc).sum())) < 1e-12 * float(Jb.norm() * c.norm())
    u = torch.tensor(rng.normal(size=(3, n, n, n)), dtype=DT) * f
    v = torch.tensor(rng.normal(size=(3, n, n, n)), dtype=DT) * f
    Pu, Pv = G.project(u, fluid, dx, K), G.project(v, fluid, dx, K)
    assert torch.allclose(G.project(2.0 * u - v, fluid, dx, K), 2.0 * Pu - Pv, atol=1e-11)


def test_step_zeroes_solids_and_buoyancy_lifts():
    n, dt, beta = 10, 0.02, 5.0
    solid = _box_solid(n, True)
    fluid = G.fluid_of(solid)
    u = torch.zeros(3, n, n, n, dtype=DT)
    d = torch.zeros(n, n, n, dtype=DT)
    d[3:6, 2:4, 3:6] = 1.0
    un, dn = G.step(u, d, fluid, dt, 1.0 / n, beta, 40)
    assert float(un[:, torch.as_tensor(solid)].abs().max()) == 0.0
    assert float(dn[torch.as_tensor(solid)].abs().max()) == 0.0
    # the smoke region is pushed up (+y)
    assert float(un[1][3:6, 2:4, 3:6].mean()) > 0.0


def test_rollout_gradient_matches_finite_differences():
    n, T, dt, beta, K = 6, 3, 0.03, 2.0, 12
    solid = _box_solid(n)
    rng = np.random.default_rng(4)
    u0 = torch.tensor(rng.normal(size=(3, n, n, n)) * 0.5, dtype=DT) * G.fluid_of(solid).to(DT)
    d0 = torch.tensor(rng.random((n, n, n)), dtype=DT) * G.fluid_of(solid).to(DT)
    wu = torch.tensor(rng.normal(size=(3, n, n, n)), dtype=DT)
    wd = torch.tensor(rng.normal(size=(n, n, n)), dtype=DT)

    def L(u, d):
        uT, dT = G.rollout(u, d, solid, T, dt, beta, K)
        return (wu * uT).sum() + (wd * dT).sum()

    ur = u0.clone().requires_grad_(True)
    dr = d0.clone().requires_grad_(True)
    gu, gd = torch.autograd.grad(L(ur, dr), (ur, dr))
    eps = 1e-6
    for (c, i, j, k) in [(0, 2, 2, 2), (1, 3, 2, 1), (2, 1, 4, 3)]:
        up, um = u0.clone(), u0.clone()
        up[c, i, j, k] += eps
        um[c, i, j, k] -= eps
        fd = float(L(up, d0) - L(um, d0)) / (2 * eps)
        assert abs(fd - float(gu[c, i, j, k])) < 1e-6 * max(1.0, abs(fd))
    for (i, j, k) in [(2, 2, 2), (3, 1, 4)]:
        dp, dm = d0.clone(), d0.clone()
        dp[i, j, k] += eps
        dm[i, j, k] -= eps
        fd = float(L(u0, dp) - L(u0, dm)) / (2 * eps)
        assert abs(fd - float(gd[i, j, k])) < 1e-6 * max(1.0, abs(fd))


def _central(a, d, dx):
    """(a[i + e_d] - a[i - e_d]) / (2 dx), zero outside the grid."""
    return (G._shift(a, d, +1, 0.0) - G._shift(a, d, -1, 0.0)) / (2.0 * dx)


def test_projection_keeps_a_discretely_divergence_free_field():
    """u = the central-difference curl of a smooth vector potential supported
    well inside the fluid has zero discrete divergence (central differences
    commute), so the projection returns it unchanged. A one-sided or
    sign-slipped divergence stencil would not."""
    n = 16
    dx = 1.0 / n
    fluid = G.fluid_of(_box_solid(n, obstacle=False))
    idx = torch.arange(n, dtype=DT)
    I, J, K = torch.meshgrid(idx, idx, idx, indexing="ij")
    r2 = ((I - 7.3) ** 2 + (J - 8.1) ** 2 + (K - 7.6) ** 2) / 9.0
    bump = torch.where(r2 < 1.0, (1.0 - r2) ** 4, torch.zeros_like(r2))
    A = torch.stack([bump * torch.sin(0.7 * J), bump * torch.cos(0.5 * K), bump * (I - 7.0)])
    u = torch.stack([_central(A[2], 1, dx) - _central(A[1], 2, dx),
                     _central(A[0], 2, dx) - _central(A[2], 0, dx),
                     _central(A[1], 0, dx) - _central(A[0], 1, dx)])
    assert u.abs().max() > 1.0
    # support clear of the walls, so no solid neighbour enters the stencils
    for ax in (1, 2, 3):
        assert u.narrow(ax, 0, 3).abs().max() == 0 and u.narrow(ax, n - 3, 3).abs().max() == 0
    b = G.divergence(u, fluid, dx)
    assert b.abs().max() <= 1e-12 * u.abs().max() / dx
    out = G.project(u, fluid, dx, 40)
    assert torch.allclose(out, u, atol=1e-12 * u.abs().max())
