"""Pins of the oracle's tool model: box SDF (closed forms and finite
differences), the soft Coulomb contact of Sec. 3.2 / Sec. 5.1, and the tool
kinematics of Sec. 4.2 (6-vector velocity action)."""
import math

import numpy as np
import pytest
import torch

from oracle import tool as tl

DT = torch.float64


def test_box_sdf_closed_forms():
    half = torch.tensor([0.1, 0.2, 0.3], dtype=DT)
    y = torch.tensor([[0.0, 0.0, 0.0],     # centre: -min(half)
                      [0.3, 0.0, 0.0],     # face: 0.2 outside in x
                      [0.2, 0.4, 0.0],     # edge region
                      [0.05, 0.0, 0.25],   # inside, nearest face z
                      [-0.3, 0.0, 0.0]], dtype=DT)
    phi, g = tl.box_sdf(y, half)
    assert phi[0].item() == pytest.approx(-0.1)
    assert phi[1].item() == pytest.approx(0.2)
    assert phi[2].item() == pytest.approx(math.hypot(0.1, 0.2))
    assert phi[3].item() == pytest.approx(-0.05)
    assert torch.allclose(g[1], torch.tensor([1.0, 0.0, 0.0], dtype=DT))
    assert torch.allclose(g[4], torch.tensor([-1.0, 0.0, 0.0], dtype=DT))
    assert torch.allclose(g[3], torch.tensor([0.0, 0.0, 1.0], dtype=DT))
    assert torch.allclose(g[2], torch.tensor([0.1, 0.2, 0.0], dtype=DT) / math.hypot(0.1, 0.2))


def test_box_sdf_gradient_is_fd_gradient_and_distance_is_brute_force():
    rng = np.random.default_rng(0)
    half = torch.tensor([0.1, 0.05, 0.2], dtype=DT)
    y = torch.tensor(rng.uniform(-0.4, 0.4, (300, 3)), dtype=DT)
    phi, g = tl.box_sdf(y, half)
    h = 1e-7
    for k in range(3):
        e = torch.zeros(3, dtype=DT)
        e[k] = h
        fd = (tl.box_sdf(y + e, half)[0] - tl.box_sdf(y - e, half)[0]) / (2 * h)
        assert torch.allclose(fd, g[:, k], atol=1e-6)
    # outside points: distance to the nearest point of the box by clamping
    out = phi > 0
    nearest = torch.maximum(torch.minimum(y, half), -half)
    assert torch.allclose(phi[out], (y - nearest).norm(dim=-1)[out], atol=1e-14)


def _contact_args(n=200, seed=1):
    rng = np.random.default_rng(seed)
    half = torch.tensor([0.1, 0.05, 0.1], dtype=DT)
    xi = torch.tensor(rng.uniform(-0.2, 0.2, (n, 3)), dtype=DT) + 0.5
    u = torch.tensor(rng.normal(size=(n, 3)), dtype=DT)
    p = torch.tensor([0.5, 0.5, 0.5], dtype=DT)
    q = torch.tensor([math.cos(0.3), 0.0, math.sin(0.3), 0.0], dtype=DT)
    R = tl.quat_to_rot(q)
    pdot = torch.tensor([0.2, -0.5, 0.1], dtype=DT)
    omega = torch.tensor([0.0, 2.0, 1.0], dtype=DT)
    return u, xi, p, R, pdot, omega, half


def test_contact_frictionless_keeps_tangential_and_inside_nodes_separate():
    u, xi, p, R, pdot, omega, half = _contact_args()
    eps_c, ell = 0.05, 0.02
    v = tl.contact(u, xi, p, R, pdot, omega, half, eps_c, ell, 0.0)
    y = (xi - p) @ R
    phi, g = tl.box_sdf(y, half)
    n = g @ R.T
    vT = pdot + torch.cross(omega.expand_as(xi), xi - p, dim=-1)
    vr0 = u - vT
    vn0 = (vr0 * n).sum(-1)
    # far nodes and separating nodes are unchanged
    keep = (phi >= eps_c) | (vn0 >= 0)
    assert torch.allclose(v[keep], u[keep], rtol=0, atol=1e-14)
    # frictionless: tangential relative velocity unchanged on contact nodes
    act = ~keep
    vr1 = v - vT
    t0 = vr0 - vn0[:, None] * n
    t1 = vr1 - (vr1 * n).sum(-1)[:, None] * n
    assert act.sum() > 5
    assert torch.allclose(t0[act], t1[act], atol=1e-13)
    # inside nodes (alpha = 1) end with non-negative relative normal velocity
    inside = act & (phi < 0)
    assert inside.sum() > 0
    assert ((vr1 * n).sum(-1)[inside] >= -1e-13).all()


def test_contact_sticky_friction_blend():
    """With large friction an approaching node inside the tool takes the tool's
    velocity; outside it blends by alpha = exp(-phi / ell)."""
    u, xi, p, R, pdot, omega, half = _contact_args(seed=2)
    eps_c, ell = 0.05, 0.02
    v = tl.contact(u, xi, p, R, pdot, omega, half, eps_c, ell, 1e6)
    y = (xi - p) @ R
    phi, g = tl.box_sdf(y, half)
    n = g @ R.T
    vT = pdot + torch.cross(omega.expand_as(xi), xi - p, dim=-1)
    vn0 = ((u - vT) * n).sum(-1)
    act = (phi < eps_c) & (vn0 < 0)
    alpha = torch.exp(-phi.clamp(min=0) / ell)
    ref = alpha[:, None] * vT + (1 - alpha[:, None]) * u
    assert torch.allclose(v[act], ref[act], atol=1e-13)


def test_kinematics_constant_rates():
    """Constant pdot and omega: p moves linearly and q turns by |omega| T dt
    about omega."""
    pose0 = torch.tensor([0.5, 0.5, 0.5, 1.0, 0.0, 0.0, 0.0], dtype=DT)
    acts = torch.tensor([[0.1, -0.2, 0.3, 0.0, 3.0, 4.0]] * 5, dtype=DT)
    P, Q, PD, OM = tl.tool_trajectory(pose0, acts, 50, 1e-3, 10)
    T = 49
    assert torch.allclose(P[T], pose0[:3] + T * 1e-3 * acts[0, :3], atol=1e-15)
    ang = 5.0 * T * 1e-3
    ref = torch.tensor([math.cos(ang / 2), 0.0, 0.6 * math.sin(ang / 2), 0.8 * math.sin(ang / 2)],
                       dtype=DT)
    assert torch.allclose(Q[T], ref, atol=1e-13)
    R = tl.quat_to_rot(Q[T])
    assert torch.allclose(R @ R.T, torch.eye(3, dtype=DT), atol=1e-14)
    # actions are held for 10 steps
    acts2 = torch.arange(30, dtype=DT).reshape(5, 6)
    _, _, PD2, _ = tl.tool_trajectory(pose0, acts2, 50, 1e-3, 10)
    assert torch.equal(PD2[19], acts2[1, :3]) and torch.equal(PD2[20], acts2[2, :3])


def test_quat_to_rot_matches_rodrigues():
    axis = torch.tensor([1.0, 2.0, -2.0], dtype=DT) / 3.0
    ang = 0.7
    q = torch.cat([torch.tensor([math.cos(ang / 2)], dtype=DT), math.sin(ang / 2) * axis])
    K = torch.tensor([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]],
                     dtype=DT)
    Rr = torch.eye(3, dtype=DT) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K
    assert torch.allclose(tl.quat_to_rot(q), Rr, atol=1e-15)


def test_contact_coulomb_sliding_and_sticking_inside_the_tool():
    """Coulomb friction at finite mu on approaching nodes inside the tool
    (alpha = 1): the relative velocity loses its normal part, and its
    tangential part keeps its direction and shrinks in length by mu times the
    removed normal speed, to zero (sticking) when that exceeds its length."""
    u, xi, p, R, pdot, omega, half = _contact_args(n=4000, seed=3)
    mu = 1.0
    v = tl.contact(u, xi, p, R, pdot, omega, half, 0.05, 0.02, mu)
    y = (xi - p) @ R
    phi, g = tl.box_sdf(y, half)
    n = g @ R.T
    vT = pdot + torch.cross(omega.expand_as(xi), xi - p, dim=-1)
    vr0, vr1 = u - vT, v - vT
    vn0 = (vr0 * n).sum(-1)
    t0 = vr0 - vn0[:, None] * n
    sel = (phi < 0) & (vn0 < 0)
    slide = sel & (t0.norm(dim=-1) > mu * (-vn0))
    stick = sel & ~slide
    assert slide.sum() > 10 and stick.sum() > 10
    # no normal part left
    assert torch.allclose((vr1 * n).sum(-1)[sel], torch.zeros(int(sel.sum()), dtype=DT), atol=1e-13)
    # sliding: same direction, length reduced by mu |vn|
    l0, l1 = t0.norm(dim=-1)[slide], vr1.norm(dim=-1)[slide]
    assert torch.allclose(l1, l0 - mu * (-vn0[slide]), atol=1e-13)
    cos = (vr1[slide] * t0[slide]).sum(-1) / (l0 * l1)
    assert torch.allclose(cos, torch.ones_like(cos), atol=1e-12)
    # sticking: the node moves with the tool
    assert torch.allclose(v[stick], vT[stick], atol=1e-13)
