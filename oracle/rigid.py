"""Oracle of rigid bodies represented by particles (Sec. 3.2 "Rigid body":
the object's particles are simulated as an elastic material by MLS-MPM, then
an object-level transformation is fitted to them and the rigidity constraint
enforced).

TEST INFRASTRUCTURE ONLY: the product never imports it; tests, smoke() and
bench.py's CPU legs do. Plain torch FP64; gradients by autograd.

Readings where the paper gives no formulas:
* An object is the set of particles of one rigid material in one scene. Its
  rest shape is the particles' positions when they are handed to the
  simulator; rbar_p = X_p - X_c are the rest offsets from the mass-weighted
  rest centroid X_c (so sum_p m_p rbar_p = 0). The particles must not all lie
  in one plane.
* Positions: after the G2P of every step the object-level transformation is
  the rigid motion closest to the particles in the mass-weighted least-squares
  sense (shape matching, Mueller et al. 2005, "Meshless deformations based on
  shape matching"): c = sum m x / M, A = sum m (x - c) rbar^T, R = the
  orthogonal polar factor of A, and x' = c + R rbar.
* Velocities: the mass-weighted least-squares rigid motion closest to the G2P
  velocities, with the new lever arms r = R rbar: v' = vbar + w x r with
  vbar = sum m v / M and w = I^{-1} L, L = sum m r x v, I = sum m (|r|^2 1 -
  r r^T). It keeps the object's linear momentum and its angular momentum
  about c (sum m r x v' = I w = L).
* The affine velocity of every particle becomes that of the rigid motion,
  C' = [w]_x (so the APIC transfers of the next step carry the rotation
  exactly), and the deformation gradient becomes the rotation, F' = R.
* With F a rotation the corotated elastic stress vanishes identically, so the
  constitutive prologue of a rigid particle is tau = 0, F_p = F (the elastic
  model evaluated at F = R, with its exact derivative).
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64
POLAR_ITERS = 40


def polar(A, iters=POLAR_ITERS):
    """Orthogonal polar factor R of a nonsingular 3x3 A (A = R S, S symmetric
    positive definite) by Newton's iteration X <- (X + X^{-T}) / 2 (Higham
    1986, "Computing the polar decomposition - with applications"), started
    from A scaled to unit mean squared singular value. Differentiable by
    autograd; converges quadratically, so `iters` steps reach FP64 round-off."""
    X = A / (A.norm() / 3.0 ** 0.5)
    for _ in range(iters):
        X = 0.5 * (X + torch.linalg.inv(X).transpose(-1, -2))
    return X


def skew(w):
    """[w]_x: skew(w) @ a = w x a."""
    z = torch.zeros((), dtype=w.dtype)
    return torch.stack([torch.stack([z, -w[2], w[1]]), torch.stack([w[2], z, -w[0]]),
                        torch.stack([-w[1], w[0], z])])


def rest_offsets(x_rest, mass, idx):
    """rbar_p = X_p - X_c of the particles idx (X_c the mass-weighted
    centroid); the rest shape is a constant of the object (no gradient)."""
    X = torch.as_tensor(np.asarray(x_rest), dtype=DT)[idx].detach()
    m = mass[idx].detach()
    Xc = (m[:, None] * X).sum(0) / m.sum()
    return X - Xc


def project(x, v, C, F, mass, idx, rbar):
    """Rigidity projection of the particles idx (one object) of the state
    (x, v, C, F) after G2P. Returns the new state and (c, R, w)."""
    m = mass[idx]
    M = m.sum()
    xo, vo = x[idx], v[idx]
    c = (m[:, None] * xo).sum(0) / M
    A = torch.einsum("p,pi,pj->ij", m, xo - c, rbar)
    R = polar(A)
    r = rbar @ R.T
    vbar = (m[:, None] * vo).sum(0) / M
    L = (m[:, None] * torch.linalg.cross(r, vo)).sum(0)
    eye = torch.eye(3, dtype=DT)
    I = torch.einsum("p,pij->ij", m, (r * r).sum(1)[:, None, None] * eye - r[:, :, None] * r[:, None, :])
    w = torch.linalg.solve(I, L)
    n = idx.shape[0]
    xn = c + r
    vn = vbar + torch.linalg.cross(w.expand(n, 3), r)
    Cn = skew(w).expand(n, 3, 3)
    Fn = R.expand(n, 3, 3)
    x = x.index_copy(0, idx, xn)
    v = v.index_copy(0, idx, vn)
    C = C.index_copy(0, idx, Cn)
    F = F.index_copy(0, idx, Fn)
    return x, v, C, F, c, R, w
