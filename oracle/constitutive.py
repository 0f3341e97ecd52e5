"""FP64 oracle: constitutive models and return mappings (test infrastructure).

Follows Sec. 3.2 "Elastic, plastic, and liquid": corotated stress for solids and
liquids, the deformation gradient of liquids reset every step, von Mises
plasticity for the non-Newtonian elastoplastic material (as in PlasticineLab),
and, for granular material, the Drucker-Prager projection of Klar et al. 2016
(sand is named only as future work in Sec. 6). The SVD-based gradient these
models need (Sec. 3.3 and App. A: the SVD gradient is written by hand) is given
here as a custom autograd VJP built from the spectral (divided-difference) form
of the derivative of an isotropic matrix function.

Conventions
-----------
* F = U diag(sigma) V^T with det U = det V = +1 (sigma_3 < 0 only if det F < 0).
* Hencky strain eps = log(max(sigma, SIGMA_FLOOR)).
* A solid's output is the projected deformation gradient F_p and the Kirchhoff
  stress tau. On the elastic branch F_p = F exactly (no re-synthesis).
* von Mises (fixed-corotated): yield when ||dev eps|| > tau_Y / (2 mu); then
  eps_p = mean(eps) + (tau_Y / 2 mu) dev eps / ||dev eps||, F_p = U exp(eps_p) V^T.
  tau = 2 mu (F_p - R) F_p^T + lambda J (J - 1) I, R = U V^T, J = det F_p,
  i.e. tau = U diag(2 mu (s - 1) s + lambda J (J - 1)) U^T with s = sigma(F_p).
* Drucker-Prager (Klar et al. 2016, Hencky StVK, no hardening):
  dgamma = ||dev eps|| + (3 lambda + 2 mu) / (2 mu) tr(eps) alpha,
  alpha = sqrt(2/3) 2 sin(phi) / (3 - sin(phi)).
  Case I dgamma <= 0: elastic. Case II tr(eps) > 0 or ||dev eps|| = 0: apex,
  eps_p = 0. Case III: eps_p = eps - dgamma dev eps / ||dev eps||.
  tau = U diag(2 mu eps_p + lambda tr(eps_p)) U^T.
* Box yield (plastic material of Sec. 3.2: the box criterion of Stomakhin et
  al. 2013, no hardening): s = clamp(sigma, 1 - theta_c, 1 + theta_s),
  F_p = U diag(s) V^T when a value was clamped, and the fixed-corotated stress
  of F_p as for von Mises: tau = U diag(2 mu (s - 1) s + lambda J (J - 1)) U^T.
* Liquid: J = det F, tau = K J (J - 1) I and F_p = J^(1/3) I (the diagonal
  reset of Sec. 3.2; with mu = 0 every diagonal matrix of determinant J gives
  this stress).
* Viscous liquid (Sec. 3.2: corotated liquid with mu > 0 and the same reset):
  tau is the fixed-corotated stress of the trial F = (I + dt C) J^(1/3) I,
  tau = U diag(2 mu (sigma - 1) sigma + lambda J (J - 1)) U^T, and
  F_p = J^(1/3) I: the shear stress comes from one step's deformation only.
"""
from __future__ import annotations

import math

import torch

SIGMA_FLOOR = 1e-4
ELASTIC, PROJECT, APEX = 0, 1, 2
_DD_REL = 1e-8     # relative gap below which a divided difference takes its limit
_DEN_MIN = 1e-12   # floor on |sigma_i + sigma_j| (reached only by inverted particles)


def lame(E, nu):
    """Lame parameters (mu, lambda) of isotropic linear elasticity from (E, nu)."""
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def dp_alpha(friction_deg):
    """Drucker-Prager cone coefficient of Klar et al. 2016 (Sec. 7.3 there)."""
    sp = math.sin(math.radians(friction_deg))
    return math.sqrt(2.0 / 3.0) * 2.0 * sp / (3.0 - sp)


def svd3(F):
    """Batched 3x3 SVD (LAPACK) with rotations U, V (det = +1)."""
    U, S, Vh = torch.linalg.svd(F)
    U = U.clone()
    V = Vh.transpose(-1, -2).clone()
    S = S.clone()
    du = torch.linalg.det(U) < 0
    U[du, :, 2] = -U[du, :, 2]
    S[du, 2] = -S[du, 2]
    dv = torch.linalg.det(V) < 0
    V[dv, :, 2] = -V[dv, :, 2]
    S[dv, 2] = -S[dv, 2]
    return U, S, V


def _hencky(sig):
    return torch.log(torch.clamp(sig, min=SIGMA_FLOOR))


def von_mises_sigma_map(sig, mu, lam, tau_y):
    """Singular values -> (projected singular values s, stress eigenvalues t, branch)."""
    eps = _hencky(sig)
    mean = eps.mean(-1, keepdim=True)
    ehat = eps - mean
    nrm = ehat.norm(dim=-1, keepdim=True)
    k = tau_y / (2.0 * mu)
    yld = (nrm - k) > 0.0
    nrm_safe = torch.where(yld, nrm, torch.ones_like(nrm))
    eps_p = torch.where(yld, mean + k * ehat / nrm_safe, eps)
    s = torch.where(yld, torch.exp(eps_p), sig)
    J = s.prod(-1, keepdim=True)
    t = 2.0 * mu * (s - 1.0) * s + lam * J * (J - 1.0)
    branch = torch.where(yld[:, 0], PROJECT, ELASTIC)
    return s, t, branch


def drucker_prager_sigma_map(sig, mu, lam, alpha):
    eps = _hencky(sig)
    tr = eps.sum(-1, keepdim=True)
    ehat = eps - tr / 3.0
    nrm = ehat.norm(dim=-1, keepdim=True)
    dgamma = nrm + (3.0 * lam + 2.0 * mu) / (2.0 * mu) * tr * alpha
    elastic = dgamma <= 0.0
    apex = (~elastic) & ((tr > 0.0) | (nrm == 0.0))
    proj = (~elastic) & (~apex)
    nrm_safe = torch.where(proj, nrm, torch.ones_like(nrm))
    eps_p = torch.where(elastic, eps,
                        torch.where(apex, torch.zeros_like(eps), eps - dgamma * ehat / nrm_safe))
    s = torch.where(elastic, sig, torch.exp(eps_p))
    t = 2.0 * mu * eps_p + lam * eps_p.sum(-1, keepdim=True)
    branch = torch.where(elastic[:, 0], ELASTIC, torch.where(apex[:, 0], APEX, PROJECT))
    return s, t, branch


def box_yield_sigma_map(sig, mu, lam, theta_c, theta_s):
    """Box criterion: singular values clamped to [1 - theta_c, 1 + theta_s];
    fixed-corotated stress eigenvalues of the clamped values."""
    s = torch.clamp(sig, min=1.0 - theta_c, max=1.0 + theta_s)
    J = s.prod(-1, keepdim=True)
    t = 2.0 * mu * (s - 1.0) * s + lam * J * (J - 1.0)
    clamped = (s != sig).any(-1)
    branch = torch.where(clamped, PROJECT, ELASTIC)
    return s, t, branch


def corotated_sigma_map(sig, mu, lam):
    """No projection: fixed-corotated stress eigenvalues of sigma."""
    J = sig.prod(-1, keepdim=True)
    t = 2.0 * mu * (sig - 1.0) * sig + lam * J * (J - 1.0)
    return sig, t, torch.full(sig.shape[:1], ELASTIC, dtype=torch.long)


def _sigma_map(kind, sig, p):
    if kind == 4:
        return corotated_sigma_map(sig, p["mu"], p["lam"])
    if kind == 1:
        return von_mises_sigma_map(sig, p["mu"], p["lam"], p["tau_y"])
    if kind == 3:
        return box_yield_sigma_map(sig, p["mu"], p["lam"], p["theta_c"], p["theta_s"])
    return drucker_prager_sigma_map(sig, p["mu"], p["lam"], p["alpha"])


def _jacobian(fn, sig):
    """Per-row Jacobians d fn(sig)_i / d sig_k of a batched R^3 -> R^3 map."""
    with torch.enable_grad():
        x = sig.detach().clone().requires_grad_(True)
        y = fn(x)
        rows = [torch.autograd.grad(y[:, i].sum(), x, retain_graph=(i < 2))[0] for i in range(3)]
    return torch.stack(rows, dim=1)


def _divided_difference(g, sig, Jg):
    """D_ij = (g_i - g_j) / (sigma_i - sigma_j), and its limit
    d g_i/d sigma_i - d g_i/d sigma_j (averaged over i, j) when sigma_i ~ sigma_j."""
    num = g[:, :, None] - g[:, None, :]
    den = sig[:, :, None] - sig[:, None, :]
    scale = 1.0 + sig.abs()[:, :, None] + sig.abs()[:, None, :]
    close = den.abs() <= _DD_REL * scale
    diag = torch.diagonal(Jg, dim1=1, dim2=2)
    lim = 0.5 * (diag[:, :, None] - Jg + diag[:, None, :] - Jg.transpose(1, 2))
    return torch.where(close, lim, num / torch.where(close, torch.ones_like(den), den))


def _safe_sum_den(sig):
    den = sig[:, :, None] + sig[:, None, :]
    sgn = torch.where(den >= 0, 1.0, -1.0).to(den.dtype)
    return sgn * torch.clamp(den.abs(), min=_DEN_MIN)


class _SolidFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, F, kind, p):
        U, S, V = svd3(F)
        s, t, branch = _sigma_map(kind, S, p)
        proj = branch != ELASTIC
        Fp_proj = U @ torch.diag_embed(s) @ V.transpose(1, 2)
        Fp = torch.where(proj[:, None, None], Fp_proj, F)
        tau = U @ torch.diag_embed(t) @ U.transpose(1, 2)
        ctx.save_for_backward(U, S, V, s, t, proj)
        ctx.kind = kind
        ctx.p = p
        return Fp, tau

    @staticmethod
    def backward(ctx, gFp, gtau):
        U, S, V, s, t, proj = ctx.saved_tensors
        kind, p = ctx.kind, ctx.p
        Ut, Vt = U.transpose(1, 2), V.transpose(1, 2)
        Js = _jacobian(lambda x: _sigma_map(kind, x, p)[0], S)
        Jt = _jacobian(lambda x: _sigma_map(kind, x, p)[1], S)
        eye = torch.eye(3, dtype=S.dtype)
        off = 1.0 - eye
        sum_den = _safe_sum_den(S)
        Fbar = torch.zeros_like(U)
        if gFp is not None:
            # F_p = U diag(s) V^T:  Z_ii = sum_k M_kk ds_k/dsig_i,
            # Z_ij = a_ij M_ij + b_ij M_ji, a/b = (D^- +/- D^+)/2.
            M = Ut @ gFp @ V
            Dm = _divided_difference(s, S, Js)
            Dp = (s[:, :, None] + s[:, None, :]) / sum_den
            a = 0.5 * (Dm + Dp)
            b = 0.5 * (Dm - Dp)
            Z = off * (a * M + b * M.transpose(1, 2))
            Md = torch.diagonal(M, dim1=1, dim2=2)
            Z = Z + torch.diag_embed(torch.einsum("nk,nki->ni", Md, Js))
            Fbar = torch.where(proj[:, None, None], U @ Z @ Vt, gFp)
        if gtau is not None:
            # tau = U diag(t) U^T:  Z_ij = D^t_ij sigma_j (N_ij + N_ji) / (sigma_i + sigma_j),
            # Z_ii = sum_k N_kk dt_k/dsig_i.
            N = Ut @ gtau @ U
            Dt = _divided_difference(t, S, Jt)
            Nsym = N + N.transpose(1, 2)
            Z = off * (Dt * S[:, None, :] * Nsym / sum_den)
            Nd = torch.diagonal(N, dim1=1, dim2=2)
            Z = Z + torch.diag_embed(torch.einsum("nk,nki->ni", Nd, Jt))
            Fbar = Fbar + U @ Z @ Vt
        return Fbar, None, None


def solid_stress(F, kind, p):
    """(F_p, tau) of a batch of solid particles of one material kind
    (1 = von Mises, 2 = Drucker-Prager, 3 = box yield); p holds mu, lam,
    tau_y, alpha, theta_c, theta_s."""
    return _SolidFunction.apply(F, kind, p)


def _cbrt(J):
    return torch.sign(J) * torch.abs(J) ** (1.0 / 3.0)


def liquid_stress(F, bulk, mu=0.0):
    """Liquid with the diagonal reset F_p = J^(1/3) I, J = det F. mu = 0:
    tau = K J (J - 1) I; mu > 0 (viscous liquid): the fixed-corotated stress
    of F with lambda = K."""
    J = torch.linalg.det(F)
    eye = torch.eye(3, dtype=F.dtype).expand(F.shape[0], 3, 3)
    Fp = _cbrt(J)[:, None, None] * eye
    if mu > 0.0:
        _, tau = _SolidFunction.apply(F, 4, dict(mu=mu, lam=bulk))
    else:
        tau = (bulk * J * (J - 1.0))[:, None, None] * eye
    return Fp, tau
