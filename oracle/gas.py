"""Oracle of the grid-based gas solver (Sec. 3.2 "Gas": incompressible flow
after Stam 1999, "Stable Fluids"; App. A: the gradient of the projection step
is written by hand).

TEST INFRASTRUCTURE ONLY: the product never imports it; tests, smoke() and
bench.py's CPU legs do. Plain torch FP64 on the CPU; gradients by autograd of
the forward definition.

Discretisation (readings where the paper is silent):
* n^3 cells of size dx = 1/n, velocity u (3 components) and smoke density d
  at cell centres (Stam's collocated layout). A solid mask marks cells that
  belong to obstacles (the paper treats cells occupied by meshes as the gas
  field's boundaries); cells outside the grid count as solid.
* One step: buoyancy u_y += dt beta d; semi-Lagrangian advection of u and d
  (back-trace X = i - dt u(i) / dx in cell-index space, clamped to
  [0, n - 1], trilinear interpolation of the old fields); zero u and d in
  solid cells; pressure projection. No diffusion (inviscid gas).
* Projection: b = central-difference divergence of u (a solid neighbour
  contributes zero velocity), minus its mean over the fluid cells (the
  zero-flux Poisson problem is solvable only for right-hand sides of zero
  sum); K damped Jacobi sweeps (weight 2/3) from p = 0 on the Laplacian of
  the fluid cells with zero-flux walls,
    p_i <- p_i / 3 + (2/3) (sum over fluid neighbours of p_j - dx^2 b_i) / n_i
  (n_i fluid neighbours); u -= central-difference gradient of p with p
  mirrored across solid faces (p_solid = p_i). Stam used Gauss-Seidel; the
  damped Jacobi sweep is parallel and, unlike the plain one, converges on the
  grid's bipartite graph. A fixed K makes the projection a fixed linear map
  of u, and its sweep operator is symmetric, so the adjoint reuses it.
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64


def _t(a, dtype=DT):
    if isinstance(a, torch.Tensor):
        return a.to(dtype)
    return torch.tensor(np.asarray(a), dtype=dtype)


def _shift(a, d, s, fill):
    """a[i + s e_d] with `fill` outside the grid (s = +1 or -1)."""
    out = torch.full_like(a, fill)
    n = a.shape[d]
    src = [slice(None)] * a.ndim
    dst = [slice(None)] * a.ndim
    if s > 0:
        src[d], dst[d] = slice(1, n), slice(0, n - 1)
    else:
        src[d], dst[d] = slice(0, n - 1), slice(1, n)
    out[tuple(dst)] = a[tuple(src)]
    return out


def fluid_of(solid):
    """Boolean fluid mask from a solid mask (n, n, n)."""
    return ~torch.as_tensor(np.asarray(solid)).bool()


def trilinear(q, X):
    """Trilinear sample of the cell field q (n, n, n) at index-space points X
    (3, n, n, n), each coordinate clamped to [0, n - 1]."""
    n = q.shape[0]
    Xc = torch.stack([X[a].clamp(0.0, n - 1.0) for a in range(3)])
    i0 = torch.floor(Xc).clamp(max=n - 2).long()
    t = Xc - i0.to(DT)
    out = torch.zeros_like(q)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                w = ((t[0] if a else 1.0 - t[0]) * (t[1] if b else 1.0 - t[1]) * (t[2] if c else 1.0 - t[2]))
                out = out + w * q[i0[0] + a, i0[1] + b, i0[2] + c]
    return out


def advect(q, u, dt, dx):
    """Semi-Lagrangian advection of the cell field q by the cell velocity u."""
    n = q.shape[0]
    idx = torch.arange(n, dtype=DT)
    I = torch.stack(torch.meshgrid(idx, idx, idx, indexing="ij"))
    X = I - (dt / dx) * u
    return trilinear(q, X)


def divergence(u, fluid, dx):
    """b_i = sum_d (u_d[i + e_d] - u_d[i - e_d]) / (2 dx) on fluid cells; a
    solid or outside neighbour contributes zero velocity."""
    f = fluid.to(DT)
    b = torch.zeros_like(u[0])
    for d in range(3):
        up = _shift(u[d] * f, d, +1, 0.0)
        um = _shift(u[d] * f, d, -1, 0.0)
        b = b + (up - um) / (2.0 * dx)
    return b * f


OMEGA = 2.0 / 3.0


def remove_mean(b, fluid):
    f = fluid.to(DT)
    return (b - (b * f).sum() / f.sum()) * f


def jacobi(b, fluid, dx, iters):
    """K damped Jacobi sweeps from p = 0 on the zero-flux Laplacian of the fluid cells."""
    f = fluid.to(DT)
    nf = torch.zeros_like(b)
    for d in range(3):
        nf = nf + _shift(f, d, +1, 0.0) + _shift(f, d, -1, 0.0)
    inv = torch.where(nf > 0, 1.0 / torch.where(nf > 0, nf, torch.ones_like(nf)), torch.zeros_like(nf)) * f
    p = torch.zeros_like(b)
    for _ in range(iters):
        s = torch.zeros_like(b)
        for d in range(3):
            s = s + _shift(p * f, d, +1, 0.0) + _shift(p * f, d, -1, 0.0)
        p = (1.0 - OMEGA) * p + OMEGA * (s - dx * dx * b) * inv
    return p


def gradient(p, fluid, dx):
    """Central-difference gradient on fluid cells, p mirrored across solid or
    outside faces (zero flux)."""
    f = fluid.to(DT)
    g = []
    for d in range(3):
        fp = _shift(f, d, +1, 0.0)
        fm = _shift(f, d, -1, 0.0)
        pp = torch.where(fp > 0, _shift(p, d, +1, 0.0), p)
        pm = torch.where(fm > 0, _shift(p, d, -1, 0.0), p)
        g.append((pp - pm) / (2.0 * dx) * f)
    return torch.stack(g)


def project(u, fluid, dx, iters):
    p = jacobi(remove_mean(divergence(u, fluid, dx), fluid), fluid, dx, iters)
    return u - gradient(p, fluid, dx)


def step(u, d, fluid, dt, dx, beta, iters):
    """One gas step (buoyancy, advection, solids, projection)."""
    f = fluid.to(DT)
    uy = u[1] + dt * beta * d
    ub = torch.stack([u[0], uy, u[2]])
    un = torch.stack([advect(ub[c], ub, dt, dx) for c in range(3)]) * f
    dn = advect(d, ub, dt, dx) * f
    return project(un, fluid, dx, iters), dn


def rollout(u0, d0, solid, T, dt, beta, iters):
    n = u0.shape[-1]
    fluid = fluid_of(solid)
    u, d = _t(u0), _t(d0)
    for _ in range(T):
        u, d = step(u, d, fluid, dt, 1.0 / n, beta, iters)
    return u, d
