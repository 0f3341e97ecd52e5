"""GPU parity of restarting from a saved state (sim_set_state) and of
adjoints seeded on the whole state (sim_add_state_grad, including dL/dC),
against the FP64 oracle stepping from the same state."""
import numpy as np
import pytest
import torch

import scenes
from gpu_util import rel
from oracle import mpm as omp

pytestmark = pytest.mark.gpu
DT = torch.float64


def _scene():
    return scenes.small_block(seed=21, grid_n=16, kinds=[0, 1, 2], ppc=2, size_cells=6, v0=(0.2, 0.0, -0.1),
                              spin=3.0, n_steps=12)


def _oracle_states(sc, T):
    model = omp.Model(sc)
    mass, vol = model.particle_mass_volume(sc.mat)
    st = omp.initial_state(torch.tensor(sc.x, dtype=DT), torch.tensor(sc.v, dtype=DT))
    out = [st]
    with torch.no_grad():
        for _ in range(T):
            st = omp.step(*st, sc.mat, mass, vol, model)
            out.append(st)
    return out, model, mass, vol


def _gpu_F(F, mat, sc):
    """Oracle F -> the library's convention: a liquid carries J = det F as diag(J, 1, 1)."""
    F = F.clone()
    liquid = torch.tensor([sc.materials[m].kind == 0 for m in sc.mat])
    J = torch.linalg.det(F[liquid])
    F[liquid] = torch.diag_embed(torch.stack([J, torch.ones_like(J), torch.ones_like(J)], dim=-1))
    return F


def test_set_state_round_trip_and_steps_match_oracle():
    from paper_2303_02346_gb300 import binding as B
    from paper_2303_02346_gb300.simulator import Simulator
    sc = _scene()
    states, _, _, _ = _oracle_states(sc, 12)
    x6, v6, C6, F6 = states[6]
    sim = Simulator(sc, checkpoint_every=0, max_steps=6)
    f32 = lambda t: t.to(torch.float32).contiguous().cuda()
    B.sim_set_state(sim.h, -1, f32(x6), f32(v6), f32(C6.reshape(-1, 9)), f32(_gpu_F(F6, sc.mat, sc).reshape(-1, 9)),
                    torch.tensor(sc.mat, dtype=torch.uint8).cuda())
    x, v, C, F = sim.state(with_CF=True)
    assert torch.equal(x.cpu(), x6.float()) and torch.equal(v.cpu(), v6.float())
    assert torch.equal(C.cpu(), C6.float())
    assert torch.allclose(F.cpu().double(), _gpu_F(F6, sc.mat, sc), rtol=1e-6, atol=1e-7)
    sim.step(6)
    x, v = sim.state()
    x12, v12 = states[12][0], states[12][1]
    assert rel(x.cpu(), x12) < 1e-4
    assert rel(v.cpu(), v12) < 1e-4


def test_state_seeded_adjoint_with_C_matches_oracle():
    """L = sum wx.x_T + wv.v_T + wC:C_T from a state with nonzero C and F;
    gradients w.r.t. x0 and v0."""
    from paper_2303_02346_gb300 import binding as B
    from paper_2303_02346_gb300.simulator import Simulator
    sc = _scene()
    rng = np.random.default_rng(3)
    N = sc.n_particles
    C0 = torch.tensor(0.5 * rng.normal(size=(N, 3, 3)), dtype=DT)
    F0 = torch.eye(3, dtype=DT) + torch.tensor(0.01 * rng.normal(size=(N, 3, 3)), dtype=DT)
    liquid = torch.tensor([sc.materials[m].kind == 0 for m in sc.mat])
    # a liquid particle is described by J only: start it from J^(1/3) I
    J0 = torch.linalg.det(F0[liquid])
    F0[liquid] = J0.pow(1.0 / 3.0)[:, None, None] * torch.eye(3, dtype=DT)
    wx = torch.tensor(rng.normal(size=(N, 3)), dtype=DT)
    wv = torch.tensor(rng.normal(size=(N, 3)), dtype=DT)
    wC = torch.tensor(0.01 * rng.normal(size=(N, 3, 3)), dtype=DT)
    T = 8
    # oracle
    model = omp.Model(sc)
    mass, vol = model.particle_mass_volume(sc.mat)
    x0 = torch.tensor(sc.x, dtype=DT, requires_grad=True)
    v0 = torch.tensor(sc.v, dtype=DT, requires_grad=True)
    st = (x0, v0, C0, F0)
    for _ in range(T):
        st = omp.step(*st, sc.mat, mass, vol, model)
    L = (wx * st[0]).sum() + (wv * st[1]).sum() + (wC * st[2]).sum()
    gx0, gv0 = torch.autograd.grad(L, (x0, v0))
    # library
    sim = Simulator(sc, checkpoint_every=4, max_steps=T)
    f32 = lambda t: t.to(torch.float32).contiguous().cuda()
    B.sim_set_state(sim.h, -1, f32(x0.detach()), f32(v0.detach()), f32(C0.reshape(-1, 9)),
                    f32(_gpu_F(F0, sc.mat, sc).reshape(-1, 9)), torch.tensor(sc.mat, dtype=torch.uint8).cuda())
    sim.step(T)
    B.sim_add_state_grad(sim.h, -1, f32(wx), f32(wv), f32(wC.reshape(-1, 9)))
    gx, gv, _ = sim.backward(want_actions=False)
    assert rel(gv.cpu(), gv0) < 1e-3
    assert rel(gx.cpu(), gx0) < 1e-3
