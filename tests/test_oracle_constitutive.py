"""Pins of the oracle's constitutive models (Sec. 3.2) and of their hand-written
SVD-based gradient (Sec. 3.3, App. A).

Pins used: the paper's Table 5 Lame constants (golden file), LAPACK via numpy,
scipy's polar decomposition, the yield-surface and idempotence properties of
each return map, and central finite differences of the oracle's own forward map
(the VJP is written independently of it)."""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats
import torch

from oracle import constitutive as cm

DT = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _params(kind, E=5e3, nu=0.2, tau_y=50.0, phi=30.0, theta_c=2.5e-2, theta_s=7.5e-3):
    mu, lam = cm.lame(E, nu)
    return dict(kind=kind, mu=mu, lam=lam, tau_y=tau_y, alpha=cm.dp_alpha(phi), theta_c=theta_c,
                theta_s=theta_s)


def test_lame_matches_table5():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table5_materials.txt"))
            if l.strip() and not l.startswith("#")]
    elastic = [r for r in rows if r[1] == "elastic"][0]
    mu, lam = cm.lame(1000.0, 0.2)
    assert mu == pytest.approx(float(elastic[2]), abs=5e-3)
    assert lam == pytest.approx(float(elastic[3]), abs=5e-3)


def test_dp_alpha_30deg():
    # sqrt(2/3) * 2 * 0.5 / 2.5
    assert cm.dp_alpha(30.0) == pytest.approx(math.sqrt(2.0 / 3.0) * 0.4, rel=1e-14)
    assert cm.dp_alpha(30.0) == pytest.approx(0.326599, abs=1e-6)


def _rand_F(rng, N, scale=0.3):
    return torch.tensor(np.eye(3) + scale * rng.normal(size=(N, 3, 3)), dtype=DT)


def test_svd_against_lapack():
    rng = np.random.default_rng(0)
    F = _rand_F(rng, 400, 0.7)
    U, S, V = cm.svd3(F)
    rec = U @ torch.diag_embed(S) @ V.transpose(1, 2)
    assert (rec - F).abs().max().item() <= 1e-13 * F.abs().max().item()
    I = torch.eye(3, dtype=DT)
    assert torch.allclose(U.transpose(1, 2) @ U, I.expand_as(U), atol=1e-13)
    assert torch.allclose(V.transpose(1, 2) @ V, I.expand_as(V), atol=1e-13)
    assert torch.allclose(torch.linalg.det(U), torch.ones(400, dtype=DT), atol=1e-13)
    assert torch.allclose(torch.linalg.det(V), torch.ones(400, dtype=DT), atol=1e-13)
    ref = np.linalg.svd(F.numpy(), compute_uv=False)
    assert np.allclose(np.abs(S.numpy()), ref, atol=1e-13)
    # sign of sigma_3 carries the sign of det F
    assert torch.equal(torch.sign(S.prod(-1)), torch.sign(torch.linalg.det(F)))


def test_corotated_elastic_branch_matches_polar():
    """Below yield, F_p = F and tau = 2 mu (F - R) F^T + lambda J (J - 1) I with R
    from scipy's polar decomposition."""
    rng = np.random.default_rng(1)
    p = _params(1, tau_y=1e9)
    F = _rand_F(rng, 50, 0.2)
    Fp, tau = cm.solid_stress(F, 1, p)
    assert torch.equal(Fp, F)
    for a in range(50):
        Fa = F[a].numpy()
        R, _ = scipy.linalg.polar(Fa)
        J = np.linalg.det(Fa)
        ref = 2 * p["mu"] * (Fa - R) @ Fa.T + p["lam"] * J * (J - 1) * np.eye(3)
        assert np.allclose(tau[a].numpy(), ref, atol=1e-9 * np.abs(ref).max())


def test_von_mises_yield_surface_and_idempotence():
    rng = np.random.default_rng(2)
    p = _params(1, tau_y=50.0)
    k = p["tau_y"] / (2 * p["mu"])
    F = _rand_F(rng, 300, 0.25)
    Fp, _ = cm.solid_stress(F, 1, p)
    _, S, _ = cm.svd3(Fp)
    eps = torch.log(S.clamp(min=cm.SIGMA_FLOOR))
    dev = eps - eps.mean(-1, keepdim=True)
    assert (dev.norm(dim=-1) <= k + 1e-12).all()
    # some must have yielded, and volume is preserved by the projection
    _, S0, _ = cm.svd3(F)
    yielded = (S0 - S).abs().max(-1).values > 1e-9
    assert yielded.sum() > 50
    J0 = torch.linalg.det(F)[yielded]
    J1 = torch.linalg.det(Fp)[yielded]
    pos = J0 > cm.SIGMA_FLOOR ** 3
    assert torch.allclose(J0[pos], J1[pos], rtol=1e-12)
    Fpp, _ = cm.solid_stress(Fp, 1, p)
    assert torch.allclose(Fpp, Fp, atol=1e-12)


def test_box_yield_bounds_stress_and_idempotence():
    """Box criterion: projected singular values in [1 - theta_c, 1 + theta_s],
    unclamped particles keep F, the projection is idempotent and preserves the
    singular vectors, and tau is the fixed-corotated stress of F_p (scipy polar)."""
    rng = np.random.default_rng(12)
    p = _params(3)
    F = torch.cat([_rand_F(rng, 150, 0.05), _rand_F(rng, 150, 0.002)])
    Fp, tau = cm.solid_stress(F, 3, p)
    U0, S0, V0 = cm.svd3(F)
    _, S, _ = cm.svd3(Fp)
    lo, hi = 1.0 - p["theta_c"], 1.0 + p["theta_s"]
    assert (S >= lo - 1e-12).all() and (S <= hi + 1e-12).all()
    inside = ((S0 >= lo) & (S0 <= hi)).all(-1)
    assert inside.sum() > 0 and (~inside).sum() > 100
    assert torch.equal(Fp[inside], F[inside])
    # F_p = U clamp(sigma) V^T with F's own singular vectors
    ref = U0 @ torch.diag_embed(S0.clamp(lo, hi)) @ V0.transpose(1, 2)
    assert torch.allclose(Fp[~inside], ref[~inside], atol=1e-12)
    Fpp, _ = cm.solid_stress(Fp, 3, p)
    assert torch.allclose(Fpp, Fp, atol=1e-12)
    for a in range(0, 300, 7):
        Fa = Fp[a].numpy()
        R, _ = scipy.linalg.polar(Fa)
        J = np.linalg.det(Fa)
        want = 2 * p["mu"] * (Fa - R) @ Fa.T + p["lam"] * J * (J - 1) * np.eye(3)
        assert np.allclose(tau[a].numpy(), want, atol=1e-9 * np.abs(want).max())


def test_drucker_prager_cone_and_idempotence():
    rng = np.random.default_rng(3)
    p = _params(2)
    c = (3 * p["lam"] + 2 * p["mu"]) / (2 * p["mu"]) * p["alpha"]
    F = _rand_F(rng, 400, 0.25)
    Fp, tau = cm.solid_stress(F, 2, p)
    _, S, _ = cm.svd3(Fp)
    eps = torch.log(S.clamp(min=cm.SIGMA_FLOOR))
    tr = eps.sum(-1)
    dev = (eps - tr[:, None] / 3).norm(dim=-1)
    assert (tr <= 1e-12).all()
    assert (dev + c * tr <= 1e-10).all()
    Fpp, _ = cm.solid_stress(Fp, 2, p)
    assert torch.allclose(Fpp, Fp, atol=1e-10)
    # expansion goes to the apex: F_p is a rotation and tau = 0
    Fe = 1.05 * torch.eye(3, dtype=DT)[None]
    Fpe, taue = cm.solid_stress(Fe, 2, p)
    assert torch.allclose(Fpe, torch.eye(3, dtype=DT)[None], atol=1e-14)
    assert taue.abs().max().item() == 0.0


def test_drucker_prager_elastic_stress_is_hencky():
    """Inside the cone (pure compression), tau = U (2 mu eps + lambda tr eps) U^T;
    for F = diag(a) it is diagonal with 2 mu log a_i + lambda sum log a."""
    p = _params(2)
    a = torch.tensor([0.97, 0.98, 0.99], dtype=DT)
    F = torch.diag(a)[None]
    Fp, tau = cm.solid_stress(F, 2, p)
    assert torch.equal(Fp, F)
    la = torch.log(a)
    ref = torch.diag(2 * p["mu"] * la + p["lam"] * la.sum())
    assert torch.allclose(tau[0], ref, atol=1e-10)


def test_liquid_stress():
    F = torch.diag(torch.tensor([0.9, 1.0, 1.05], dtype=DT))[None]
    Fp, tau = cm.liquid_stress(F, 1e4)
    J = 0.9 * 1.05
    assert torch.allclose(tau[0], 1e4 * J * (J - 1) * torch.eye(3, dtype=DT))
    assert torch.linalg.det(Fp).item() == pytest.approx(J, rel=1e-14)
    # the diagonal reset is J^(1/3) I
    assert torch.allclose(Fp[0], J ** (1.0 / 3.0) * torch.eye(3, dtype=DT), rtol=1e-14)


def test_viscous_liquid_stress_is_corotated_of_the_trial_F():
    """mu > 0: tau = 2 mu (F - R) F^T + K J (J - 1) I with R from scipy's polar
    decomposition, F_p = J^(1/3) I; mu -> 0 gives the plain liquid."""
    rng = np.random.default_rng(13)
    F = _rand_F(rng, 40, 0.1)
    mu, K = 1e3, 1e4
    Fp, tau = cm.liquid_stress(F, K, mu)
    for a in range(40):
        Fa = F[a].numpy()
        R, _ = scipy.linalg.polar(Fa)
        J = np.linalg.det(Fa)
        ref = 2 * mu * (Fa - R) @ Fa.T + K * J * (J - 1) * np.eye(3)
        assert np.allclose(tau[a].numpy(), ref, atol=1e-9 * np.abs(ref).max())
        assert np.allclose(Fp[a].numpy(), np.cbrt(J) * np.eye(3), rtol=1e-13)
    _, tau0 = cm.liquid_stress(F, K, 1e-12)
    _, tau_plain = cm.liquid_stress(F, K)
    assert torch.allclose(tau0, tau_plain, atol=1e-6)


def test_viscous_liquid_vjp_against_finite_differences():
    rng = np.random.default_rng(14)
    F = _rand_F(rng, 20, 0.1)
    mu, K = 1e3, 1e4
    gFp = torch.tensor(rng.normal(size=(20, 3, 3)), dtype=DT)
    gtau = torch.tensor(rng.normal(size=(20, 3, 3)), dtype=DT) * 1e-3
    Fr = F.clone().requires_grad_(True)
    Fp, tau = cm.liquid_stress(Fr, K, mu)
    g, = torch.autograd.grad((Fp * gFp).sum() + (tau * gtau).sum(), Fr)
    h = 1e-6
    fd = torch.zeros_like(F)
    for i in range(3):
        for j in range(3):
            Fa, Fb = F.clone(), F.clone()
            Fa[:, i, j] += h
            Fb[:, i, j] -= h
            a1, b1 = cm.liquid_stress(Fa, K, mu)
            a0, b0 = cm.liquid_stress(Fb, K, mu)
            fd[:, i, j] = (((a1 - a0) * gFp).sum((1, 2)) + ((b1 - b0) * gtau).sum((1, 2))) / (2 * h)
    assert ((g - fd).norm() / fd.norm()).item() < 1e-6


def _fd_vjp(kind, p, F, gFp, gtau, h=1e-6):
    out = torch.zeros_like(F)
    for i in range(3):
        for j in range(3):
            Fpl = F.clone()
            Fmi = F.clone()
            Fpl[:, i, j] += h
            Fmi[:, i, j] -= h
            a1, b1 = cm.solid_stress(Fpl, kind, p)
            a0, b0 = cm.solid_stress(Fmi, kind, p)
            out[:, i, j] = (((a1 - a0) * gFp).sum((1, 2)) + ((b1 - b0) * gtau).sum((1, 2))) / (2 * h)
    return out


@pytest.mark.parametrize("case", ["vm_elastic", "vm_yield", "vm_near_identity", "vm_degenerate",
                                  "dp_elastic", "dp_project", "dp_apex", "box_elastic", "box_project",
                                  "box_degenerate"])
def test_solid_vjp_against_finite_differences(case):
    rng = np.random.default_rng(hash(case) % 2 ** 32)
    N = 40
    if case.startswith("vm"):
        kind = 1
        p = _params(1, tau_y=50.0 if case != "vm_elastic" else 1e9)
    elif case.startswith("box"):
        kind = 3
        p = _params(3)
    else:
        kind = 2
        p = _params(2)
    if case in ("vm_elastic", "vm_yield"):
        F = _rand_F(rng, N, 0.25)
    elif case == "vm_near_identity":
        F = _rand_F(rng, N, 1e-4)
    elif case == "vm_degenerate":
        # two equal singular values, random rotations
        Q1 = torch.tensor(scipy.stats.special_ortho_group.rvs(3, N, random_state=1), dtype=DT)
        Q2 = torch.tensor(scipy.stats.special_ortho_group.rvs(3, N, random_state=2), dtype=DT)
        S = torch.tensor([[1.3, 0.8, 0.8]] * N, dtype=DT)
        S[: N // 2] = torch.tensor([1.1, 1.1, 0.7], dtype=DT)
        F = Q1 @ torch.diag_embed(S) @ Q2.transpose(1, 2)
    elif case == "dp_elastic":
        # compression with a small deviatoric part stays inside the cone
        Q1 = torch.tensor(scipy.stats.special_ortho_group.rvs(3, N, random_state=3), dtype=DT)
        Q2 = torch.tensor(scipy.stats.special_ortho_group.rvs(3, N, random_state=4), dtype=DT)
        S = torch.tensor(0.95 + 0.01 * rng.random((N, 3)), dtype=DT)
        F = Q1 @ torch.diag_embed(S) @ Q2.transpose(1, 2)
    elif case == "dp_project":
        Q1 = torch.tensor(scipy.stats.special_ortho_group.rvs(3, N, random_state=5), dtype=DT)
        Q2 = torch.tensor(scipy.stats.special_ortho_group.rvs(3, N, random_state=6), dtype=DT)
        S = torch.tensor(np.exp(np.array([-0.08, 0.0, 0.05]) + 0.01 * rng.random((N, 3))), dtype=DT)
        F = Q1 @ torch.diag_embed(S) @ Q2.transpose(1, 2)
    elif case == "box_elastic":
        F = _rand_F(rng, N, 1e-3)
    elif case == "box_project":
        F = _rand_F(rng, N, 0.08)
    elif case == "box_degenerate":
        # two singular values clamped to the same bound, one inside
        Q1 = torch.tensor(scipy.stats.special_ortho_group.rvs(3, N, random_state=7), dtype=DT)
        Q2 = torch.tensor(scipy.stats.special_ortho_group.rvs(3, N, random_state=8), dtype=DT)
        S = torch.tensor([[1.05, 1.02, 0.999]] * N, dtype=DT)
        S[: N // 2] = torch.tensor([1.001, 0.9, 0.95], dtype=DT)
        F = Q1 @ torch.diag_embed(S) @ Q2.transpose(1, 2)
    else:  # dp_apex
        F = _rand_F(rng, N, 0.02) * 1.1
    gFp = torch.tensor(rng.normal(size=(N, 3, 3)), dtype=DT)
    gtau = torch.tensor(rng.normal(size=(N, 3, 3)), dtype=DT) * 1e-3
    # check that the intended branch is exercised
    _, S, _ = cm.svd3(F)
    if kind == 3:
        branch = cm.box_yield_sigma_map(S, p["mu"], p["lam"], p["theta_c"], p["theta_s"])[2]
    else:
        sm = cm.von_mises_sigma_map if kind == 1 else cm.drucker_prager_sigma_map
        args = (p["mu"], p["lam"], p["tau_y"] if kind == 1 else p["alpha"])
        branch = sm(S, *args)[2]
    want = {"vm_elastic": 0, "vm_yield": None, "vm_near_identity": 0, "vm_degenerate": None,
            "dp_elastic": 0, "dp_project": 1, "dp_apex": 2, "box_elastic": 0, "box_project": None,
            "box_degenerate": 1}[case]
    if want is not None:
        assert (branch == want).all(), branch
    if case in ("vm_yield", "box_project"):
        assert (branch == 1).sum() > 10
    Fr = F.clone().requires_grad_(True)
    Fp, tau = cm.solid_stress(Fr, kind, p)
    g, = torch.autograd.grad((Fp * gFp).sum() + (tau * gtau).sum(), Fr)
    fd = _fd_vjp(kind, p, F, gFp, gtau)
    err = (g - fd).norm() / fd.norm()
    assert err.item() < 1e-6, err.item()


def test_solid_vjp_exactly_degenerate_identity():
    """At F = I (all singular values equal) the VJP of the smooth elastic map
    exists; the limit branch of the divided differences must reproduce FD."""
    p = _params(1, tau_y=1e9)
    F = torch.eye(3, dtype=DT)[None].repeat(3, 1, 1)
    rng = np.random.default_rng(9)
    gFp = torch.tensor(rng.normal(size=(3, 3, 3)), dtype=DT)
    gtau = torch.tensor(rng.normal(size=(3, 3, 3)), dtype=DT) * 1e-3
    Fr = F.clone().requires_grad_(True)
    Fp, tau = cm.solid_stress(Fr, 1, p)
    g, = torch.autograd.grad((Fp * gFp).sum() + (tau * gtau).sum(), Fr)
    fd = _fd_vjp(1, p, F, gFp, gtau)
    assert ((g - fd).norm() / fd.norm()).item() < 1e-6


def _rand_rot(rng, n):
    """n random rotations (det +1) from the QR factors of Gaussian matrices."""
    out = []
    for _ in range(n):
        q, r = np.linalg.qr(rng.standard_normal((3, 3)))
        q = q @ np.diag(np.sign(np.diag(r)))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        out.append(q)
    return torch.tensor(np.array(out), dtype=DT)


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_return_maps_are_objective_and_isotropic(kind):
    """Frame indifference and material isotropy of every solid model, elastic
    and plastic branches alike: for rotations R (spatial) and Q (material),
    Phi(R F Q) = R Phi(F) Q and tau(R F Q) = R tau(F) R^T. A transposed
    singular-vector factor, or a stress built from V instead of U, breaks one
    of the two."""
    rng = np.random.default_rng(40 + kind)
    p = _params(kind)
    # large random deformations (mostly plastic), then slight compression with
    # small shear (elastic for all three criteria: inside the box, inside the
    # sand's cone, below the von Mises stress)
    F = torch.cat([_rand_F(rng, 100, 0.2), 0.985 * _rand_F(rng, 100, 0.002)])
    R, Q = _rand_rot(rng, 200), _rand_rot(rng, 200)
    Fp, tau = cm.solid_stress(F, kind, p)
    Fp2, tau2 = cm.solid_stress(R @ F @ Q, kind, p)
    # both branches occur
    _, S0, _ = cm.svd3(F)
    _, S1, _ = cm.svd3(Fp)
    yielded = (S0 - S1).abs().max(-1).values > 1e-9
    assert 10 < int(yielded.sum()) < 190
    scale = tau.abs().max()
    assert torch.allclose(Fp2, R @ Fp @ Q, atol=1e-10)
    assert torch.allclose(tau2, R @ tau @ R.transpose(1, 2), atol=1e-10 * scale)


def test_viscous_liquid_stress_is_objective_and_its_reset_is_isotropic():
    """Viscous liquid: tau(R F Q) = R tau(F) R^T, and the reset J^(1/3) I depends
    on J alone (unchanged by both rotations)."""
    rng = np.random.default_rng(45)
    F = _rand_F(rng, 100, 0.2)
    R, Q = _rand_rot(rng, 100), _rand_rot(rng, 100)
    Fp, tau = cm.liquid_stress(F, 1e4, mu=300.0)
    Fp2, tau2 = cm.liquid_stress(R @ F @ Q, 1e4, mu=300.0)
    assert torch.allclose(Fp2, Fp, atol=1e-12)
    assert torch.allclose(tau2, R @ tau @ R.transpose(1, 2), atol=1e-10 * tau.abs().max())
