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
  rest centroid X_c (so sum_p m_p rbar_p = 0).
* After the G2P of every step the object-level transformation is the rigid
  motion closest to the particles in the mass-weighted least-squares sense
  (shape matching, Mueller et al. 2005, "Meshless deformations based on shape
  matching"): c = sum m x / M, A = sum m (x - c) rbar^T, R = the orthogonal
  polar factor of A.
* Rigidity is enforced on the whole state: x' = c + R rbar; the velocity takes
  the position correction, v' = v + (x' - x) / dt (position-based velocity
  update of the same paper), so the object's linear momentum is unchanged; the
  affine velocity keeps only its rotational (skew) part, C' = (C - C^T) / 2;
  the deformation gradient becomes the rotation, F' = R.
* With F a rotation the corotated elastic stress of the next step vanishes
  identically, so the constitutive prologue of a rigid particle is tau = 0,
  F_p = F (this is the elastic model evaluated at F = R, with its exact
  derivative).
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


def rest_offsets(x_rest, mass, idx):
    """rbar_p = X_p - X_c of the particles idx (X_c the mass-weighted
    centroid); the rest shape is a constant of the object (no gradient)."""
    X = torch.as_tensor(np.asarray(x_rest), dtype=DT)[idx].detach()
    m = mass[idx].detach()
    Xc = (m[:, None] * X).sum(0) / m.sum()
    return X - Xc


def project(x, v, C, F, mass, dt, idx, rbar):
    """Rigidity projection of the particles idx (one object) of the state
    (x, v, C, F) after G2P. Returns the new state and (c, R)."""
    m = mass[idx]
    M = m.sum()
    xo = x[idx]
    c = (m[:, None] * xo).sum(0) / M
    A = torch.einsum("p,pi,pj->ij", m, xo - c, rbar)
    R = polar(A)
    xn = c + rbar @ R.T
    vn = v[idx] + (xn - xo) / dt
    Co = C[idx]
    Cn = 0.5 * (Co - Co.transpose(-1, -2))
    Fn = R.expand(idx.shape[0], 3, 3)
    x = x.index_copy(0, idx, xn)
    v = v.index_copy(0, idx, vn)
    C = C.index_copy(0, idx, Cn)
    F = F.index_copy(0, idx, Fn)
    return x, v, C, F, c, R
