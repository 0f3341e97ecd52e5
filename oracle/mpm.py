"""FP64 oracle of one MLS-MPM time step and of a rollout (test infrastructure).

Sec. 3.2: solids and liquids are particles simulated with the Moving Least
Squares Material Point Method (Hu et al. 2018); deformation gradient, internal
force and stress enter in the particle-to-grid (P2G) step and boundary
conditions in the grid operations; contact with SDF objects is part of the grid
operations. The order of one step n -> n+1 used here (each function below is one
stage, written in plain vectorised torch with no blocking or fusion):

1. constitutive prologue: (F_p, tau) from the trial F carried by the particle;
2. P2G with quadratic B-splines, MLS affine momentum
   A = -dt V_p (4 / dx^2) tau + m_p C_p,
   m_i = sum_p W_ip m_p, mv_i = sum_p W_ip (m_p v_p + A_p (x_i - x_p));
3. grid update on nodes with m_i > 0: u = mv / m + dt g, soft tool contact,
   sticky walls (every node with an index < bound or >= n - bound gets v = 0);
4. G2P: v_p = sum W v_i, C_p = (4 / dx^2) sum W v_i (x_i - x_p)^T,
   x_p += dt v_p, F <- (I + dt C_p) F_p;
5. rigidity projection of every particle-represented rigid object (`rigid`).

Node i sits at i dx on an n^3 grid over the unit cube; base = floor(x/dx - 0.5).
A particle whose stencil [base, base + 2] leaves the grid raises DomainError.
Gradients come from torch autograd (the SVD-dependent part from the VJP in
`constitutive`). This module is test infrastructure: only the tests, the smoke
check and the CPU-baseline leg of the benchmark use it.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.utils.checkpoint

from . import constitutive as cm
from . import rigid as rg
from . import tool as tl

DT = torch.float64
_OFFS = torch.tensor([[i, j, k] for i in range(3) for j in range(3) for k in range(3)])


class DomainError(RuntimeError):
    pass


class Model:
    """Constants of a scene, as the oracle derives them from the raw inputs."""

    def __init__(self, scene):
        self.n = int(scene.grid_n)
        self.dx = 1.0 / self.n
        self.inv_dx = float(self.n)
        self.dt = float(scene.dt)
        self.gravity = torch.tensor(scene.gravity, dtype=DT)
        self.bound = int(scene.bound)
        self.spa = int(scene.substeps_per_action)
        self.mats = []
        for m in scene.materials:
            if m.kind == 0:
                mu, lam = 0.0, float(m.bulk)
            elif m.kind == 4:
                mu, lam = float(getattr(m, "shear", 0.0)), float(m.bulk)
            else:
                mu, lam = cm.lame(float(m.E), float(m.nu))
            self.mats.append(dict(kind=int(m.kind), mu=mu, lam=lam, tau_y=float(m.yield_stress),
                                  alpha=cm.dp_alpha(float(m.friction_deg)), rho=float(m.rho),
                                  vol=float(m.volume), theta_c=float(getattr(m, "crit_compress", 2.5e-2)),
                                  theta_s=float(getattr(m, "crit_stretch", 7.5e-3))))
        self.tool = bool(scene.tool_enabled)
        self.tool_half = torch.tensor(scene.tool_half, dtype=DT)
        self.eps_c = float(scene.contact_eps)
        self.ell = float(scene.contact_soft) if scene.contact_soft > 0 else self.dx
        self.mu_f = float(scene.friction)

    def particle_mass_volume(self, mat):
        rho = torch.tensor([m["rho"] for m in self.mats], dtype=DT)
        vol = torch.tensor([m["vol"] for m in self.mats], dtype=DT)
        mat = torch.as_tensor(np.asarray(mat), dtype=torch.long)
        return rho[mat] * vol[mat], vol[mat]


# ----------------------------------------------------------------------------
# quadratic B-spline stencil
# ----------------------------------------------------------------------------
def stencil(x, model):
    """base (N,3) long, weights W (N,27), offsets dpos = x_i - x_p (N,27,3),
    node linear indices (N,27) for the 27 nodes base + o, o in {0,1,2}^3."""
    xs = x * model.inv_dx
    base = torch.floor(xs - 0.5).detach()
    f = xs - base
    w = torch.stack([0.5 * (1.5 - f) ** 2, 0.75 - (f - 1.0) ** 2, 0.5 * (f - 0.5) ** 2], dim=1)
    o = _OFFS
    W = w[:, o[:, 0], 0] * w[:, o[:, 1], 1] * w[:, o[:, 2], 2]
    dpos = (o[None].to(DT) - f[:, None, :]) * model.dx
    b = base.long()
    n = model.n
    if bool(((b < 0) | (b > n - 3)).any()):
        raise DomainError("particle stencil leaves the grid")
    node = b[:, None, :] + o[None]
    lin = (node[..., 0] * n + node[..., 1]) * n + node[..., 2]
    return W, dpos, lin


# ----------------------------------------------------------------------------
# stages of one step
# ----------------------------------------------------------------------------
def constitutive(F, mat, model):
    """(F_p, tau) for every particle, grouped by material."""
    mat = torch.as_tensor(np.asarray(mat), dtype=torch.long)
    Fp = torch.zeros_like(F)
    tau = torch.zeros_like(F)
    for mi, m in enumerate(model.mats):
        idx = torch.nonzero(mat == mi)[:, 0]
        if idx.numel() == 0:
            continue
        Fm = F.index_select(0, idx)
        if m["kind"] == 5:
            # rigid: F is a rotation, where the corotated stress vanishes
            a, b = Fm, torch.zeros_like(Fm)
        elif m["kind"] in (0, 4):
            a, b = cm.liquid_stress(Fm, m["lam"], m["mu"])
        else:
            a, b = cm.solid_stress(Fm, m["kind"], m)
        Fp = Fp.index_copy(0, idx, a)
        tau = tau.index_copy(0, idx, b)
    return Fp, tau


def p2g(x, v, C, tau, mass, vol, model):
    """Grid mass m (n^3) and momentum mv (n^3, 3)."""
    W, dpos, lin = stencil(x, model)
    n3 = model.n ** 3
    A = (-model.dt * 4.0 * model.inv_dx ** 2) * vol[:, None, None] * tau + mass[:, None, None] * C
    mom = mass[:, None, None] * v[:, None, :] + torch.einsum("pij,poj->poi", A, dpos)
    m = torch.zeros(n3, dtype=DT).index_add(0, lin.reshape(-1), (W * mass[:, None]).reshape(-1))
    mv = torch.zeros(n3, 3, dtype=DT).index_add(0, lin.reshape(-1), (W[..., None] * mom).reshape(-1, 3))
    return m, mv


def node_positions(idx, model):
    n = model.n
    i = idx // (n * n)
    j = (idx // n) % n
    k = idx % n
    return torch.stack([i, j, k], dim=-1), torch.stack([i, j, k], dim=-1).to(DT) * model.dx


def grid_update(m, mv, model, tool_state=None):
    """Node velocities (n^3, 3) after gravity, tool contact and sticky walls."""
    act = torch.nonzero(m > 0)[:, 0]
    ma = m.index_select(0, act)
    u = mv.index_select(0, act) / ma[:, None] + model.dt * model.gravity
    ijk, xi = node_positions(act, model)
    if model.tool and tool_state is not None:
        p, q, pdot, omega = tool_state
        R = tl.quat_to_rot(q)
        u = tl.contact(u, xi, p, R, pdot, omega, model.tool_half, model.eps_c, model.ell, model.mu_f)
    wall = ((ijk < model.bound) | (ijk >= model.n - model.bound)).any(dim=-1)
    u = torch.where(wall[:, None], torch.zeros_like(u), u)
    return torch.zeros(model.n ** 3, 3, dtype=DT).index_copy(0, act, u)


def g2p(x, Fp, vg, model):
    W, dpos, lin = stencil(x, model)
    vi = vg.index_select(0, lin.reshape(-1)).reshape(lin.shape[0], 27, 3)
    v_new = (W[..., None] * vi).sum(1)
    C_new = (4.0 * model.inv_dx ** 2) * torch.einsum("po,poi,poj->pij", W, vi, dpos)
    x_new = x + model.dt * v_new
    eye = torch.eye(3, dtype=DT)
    F_new = (eye + model.dt * C_new) @ Fp
    return x_new, v_new, C_new, F_new


def rigid_objects(model, mat, mass, x_rest):
    """(particle indices, rest offsets) of every rigid object of one scene."""
    mat = torch.as_tensor(np.asarray(mat), dtype=torch.long)
    out = []
    for mi, m in enumerate(model.mats):
        idx = torch.nonzero(mat == mi)[:, 0]
        if m["kind"] == 5 and idx.numel() > 0:
            out.append((idx, rg.rest_offsets(x_rest, mass, idx)))
    return out


def step(x, v, C, F, mat, mass, vol, model, tool_state=None, rigid=()):
    Fp, tau = constitutive(F, mat, model)
    m, mv = p2g(x, v, C, tau, mass, vol, model)
    vg = grid_update(m, mv, model, tool_state)
    x, v, C, F = g2p(x, Fp, vg, model)
    for idx, rbar in rigid:
        x, v, C, F, _, _, _ = rg.project(x, v, C, F, mass, idx, rbar)
    return x, v, C, F


# ----------------------------------------------------------------------------
# rollout
# ----------------------------------------------------------------------------
def initial_state(x0, v0):
    N = x0.shape[0]
    C = torch.zeros(N, 3, 3, dtype=DT)
    F = torch.eye(3, dtype=DT).expand(N, 3, 3).clone()
    return x0, v0, C, F


def rollout(scene, n_steps=None, x0=None, v0=None, actions=None, scene_index=0,
            keep_states=False, checkpoint_steps=False):
    """Simulate one scene of `scene` for n_steps and return the final state
    (x, v, C, F), or the list of all states if keep_states. x0/v0/actions may be
    tensors that require grad."""
    model = Model(scene)
    lo = int(sum(scene.scene_counts[:scene_index]))
    hi = lo + int(scene.scene_counts[scene_index])
    if x0 is None:
        x0 = torch.tensor(scene.x[lo:hi], dtype=DT)
    if v0 is None:
        v0 = torch.tensor(scene.v[lo:hi], dtype=DT)
    mat = scene.mat[lo:hi]
    mass, vol = model.particle_mass_volume(mat)
    # rest shape of rigid objects: the positions handed to the simulator
    rigid = rigid_objects(model, mat, mass, scene.x[lo:hi])
    T = scene.n_steps if n_steps is None else n_steps
    tool_states = None
    if model.tool:
        if actions is None:
            actions = torch.tensor(scene.tool_actions[scene_index], dtype=DT)
        pose0 = torch.tensor(scene.tool_pose0[scene_index], dtype=DT)
        P, Q, PD, OM = tl.tool_trajectory(pose0, actions, T, model.dt, model.spa)
        tool_states = [(P[n], Q[n], PD[n], OM[n]) for n in range(T)]
    state = initial_state(x0, v0)
    states = [state]
    for n in range(T):
        ts = tool_states[n] if tool_states is not None else None
        if checkpoint_steps:
            def fn(x, v, C, F, *tsa, _mat=mat):
                return step(x, v, C, F, _mat, mass, vol, model, tsa if tsa else None, rigid)
            args = tuple(state) + (tuple(ts) if ts is not None else ())
            state = torch.utils.checkpoint.checkpoint(fn, *args, use_reentrant=False)
        else:
            state = step(*state, mat, mass, vol, model, ts, rigid)
        if keep_states:
            states.append(state)
    return states if keep_states else state


# ----------------------------------------------------------------------------
# losses (App. C)
# ----------------------------------------------------------------------------
def position_loss(x, target, weight=1.0):
    """Point-goal loss, squared reading: w sum_p |x_p - x*|^2."""
    t = torch.as_tensor(target, dtype=DT)
    return weight * ((x - t) ** 2).sum()


def grid_mass_loss(x, mass, model, target_mass, target_dist, total_mass):
    """Chamfer-style grid analogue: with m the P2G mass field of x,
    L = sum_i (m_i - m*_i)^2 / M^2 + sum_i m_i d*_i / M."""
    W, _, lin = stencil(x, model)
    m = torch.zeros(model.n ** 3, dtype=DT).index_add(0, lin.reshape(-1), (W * mass[:, None]).reshape(-1))
    tm = torch.as_tensor(target_mass, dtype=DT)
    td = torch.as_tensor(target_dist, dtype=DT)
    M = float(total_mass)
    return ((m - tm) ** 2).sum() / M ** 2 + (m * td).sum() / M


def scene_loss(scene, x, scene_index=0):
    model = Model(scene)
    lo = int(sum(scene.scene_counts[:scene_index]))
    hi = lo + int(scene.scene_counts[scene_index])
    L = scene.loss
    if L["kind"] == "position":
        return position_loss(x, L["target"], L.get("weight", 1.0))
    mass, _ = model.particle_mass_volume(scene.mat[lo:hi])
    return grid_mass_loss(x, mass, model, L["target_mass"], L["target_dist"], L["total_mass"])
