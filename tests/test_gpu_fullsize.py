"""GPU-vs-oracle parity at the full workload sizes, in the launch
configuration bench.py times (checkpoint every 20 steps, 200-step horizon).

Where the oracle cannot afford the whole run, the check is on outputs it can
compute one by one: the oracle's own single step applied to the GPU's state at
step 199 must give the GPU's state at step 200; the full horizon with
gradients is checked on a 5% copy of the scene. Tolerances as in
test_gpu_parity: 1e-4 relative L2 on x and v, 1e-3 on gradients.
"""
import numpy as np
import pytest
import torch

import scenes
from gpu_util import oracle_forward, oracle_grad, rel
from oracle import mpm as omp
from oracle import tool as otl

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL_X = 1e-4
TOL_G = 1e-3
DT = torch.float64


def _bench_sim(sc):
    from paper_2303_02346_gb300.simulator import Simulator
    sim = Simulator(sc)  # the scene's own checkpoint interval and horizon, as bench.py
    sim.reset()
    return sim


def test_full_size_three_steps_forward_and_gradient():
    sc = scenes.multi_material()
    sim = _bench_sim(sc)
    T = 3
    sim.step(T)
    x, v = sim.state()
    xo, vo, _, _ = oracle_forward(sc, n_steps=T)
    assert rel(x.cpu(), xo) < TOL_X
    assert rel(v.cpu(), vo) < TOL_X
    L = sc.loss
    Lg = sim.grid_mass_loss(L["target_mass"], L["target_dist"], L["total_mass"])
    gx, gv, ga = sim.backward()
    ref = oracle_grad(sc, n_steps=T, want_actions=True)
    assert abs(Lg - ref["loss"]) / abs(ref["loss"]) < TOL_X
    assert rel(gx.cpu(), ref["x0"]) < TOL_G
    assert rel(gv.cpu(), ref["v0"]) < TOL_G
    # only the first action acts in 3 steps
    assert np.abs(ref["actions"][0]).max() > 0
    assert rel(ga.cpu()[0], ref["actions"]) < TOL_G


def test_full_size_full_horizon_last_step_matches_oracle_step():
    sc = scenes.multi_material()
    sim = _bench_sim(sc)
    T = sc.n_steps
    sim.step(T - 1)
    x, v, C, F = sim.state(with_CF=True)
    sim.step(1)
    x1, v1 = sim.state()
    assert torch.isfinite(x1).all() and torch.isfinite(v1).all()
    model = omp.Model(sc)
    mass, vol = model.particle_mass_volume(sc.mat)
    act = torch.tensor(sc.tool_actions[0], dtype=DT)
    pose0 = torch.tensor(sc.tool_pose0[0], dtype=DT)
    P_, Q_, PD, OM = otl.tool_trajectory(pose0, act, T, sc.dt, sc.substeps_per_action)
    ts = (P_[T - 1], Q_[T - 1], PD[T - 1], OM[T - 1])
    with torch.no_grad():
        xo, vo, Co, Fo = omp.step(x.cpu().double(), v.cpu().double(), C.cpu().double(), F.cpu().double(),
                                  sc.mat, mass, vol, model, ts)
    assert rel(x1.cpu(), xo) < TOL_X
    assert rel(v1.cpu(), vo) < TOL_X
    # the scene really evolved: the liquid compressed, solids deformed
    Jl = torch.linalg.det(F.cpu().double())[torch.tensor(sc.mat == 0)]
    assert 0.9 < float(Jl.mean()) < 1.05
    assert float((F.cpu()[torch.tensor(sc.mat != 0)] - torch.eye(3)).abs().max()) > 1e-3


def test_scaled_copy_full_horizon_gradient():
    """5% of the particles, same grid, same 200-step horizon and checkpoints."""
    sc = scenes.multi_material(scale=0.05)
    sim = _bench_sim(sc)
    sim.step(sc.n_steps)
    x, v = sim.state()
    L = sc.loss
    Lg = sim.grid_mass_loss(L["target_mass"], L["target_dist"], L["total_mass"])
    gx, gv, ga = sim.backward()
    ref = oracle_grad(sc, want_actions=True, checkpoint=True)
    xo, vo, _, _ = oracle_forward(sc)
    assert rel(x.cpu(), xo) < TOL_X and rel(v.cpu(), vo) < TOL_X
    assert abs(Lg - ref["loss"]) / abs(ref["loss"]) < TOL_X
    assert rel(ga.cpu()[0], ref["actions"]) < TOL_G
    assert rel(gx.cpu(), ref["x0"]) < TOL_G


def test_batched_64_scenes_sampled_against_oracle():
    """All 64 scenes (about 3.3M particles) in one handle; four of them checked
    scene by scene against the oracle after 10 steps, one with gradients."""
    sc = scenes.batched_scenes()
    from paper_2303_02346_gb300.simulator import Simulator
    T = 10
    sim = Simulator(sc, checkpoint_every=5, max_steps=T)
    sim.reset()
    sim.step(T)
    sim.position_loss(sc.loss["target"], 1.0, scene=-1)
    gx, gv, ga = sim.backward()
    offs = np.concatenate([[0], np.cumsum(sc.scene_counts)])
    for s_i in (0, 17, 40, 63):
        xo, vo, _, _ = oracle_forward(sc, n_steps=T, scene_index=s_i)
        # the GPU state after the backward is still the state at step T
        sim_x, sim_v = sim.state(scene=s_i)
        assert rel(sim_x.cpu(), xo) < TOL_X, s_i
        assert rel(sim_v.cpu(), vo) < TOL_X, s_i
    ref = oracle_grad(sc, n_steps=T, scene_index=17, want_actions=True)
    assert rel(gx.cpu()[offs[17]:offs[18]], ref["x0"]) < TOL_G
    # 10 steps use only the first action
    assert rel(ga.cpu()[17], ref["actions"][:1]) < TOL_G
    assert np.abs(ref["actions"][1:]).max() == 0.0


def test_dam_break_two_million_particles_first_steps():
    """2M particles on 256^3 (70% water, 30% von Mises): 4 steps against the
    oracle at full size."""
    sc = scenes.dam_break()
    from paper_2303_02346_gb300.simulator import Simulator
    T = 4
    sim = Simulator(sc, checkpoint_every=0, max_steps=T)
    sim.reset()
    sim.step(T)
    x, v = sim.state()
    xo, vo, _, _ = oracle_forward(sc, n_steps=T)
    assert rel(x.cpu(), xo) < TOL_X
    assert rel(v.cpu(), vo) < TOL_X


def test_dam_break_first_checkpoint_interval_full_size():
    """2M particles on 256^3: the whole first checkpoint interval (50 steps)
    against the oracle at full size, in the launch path the bench's forward
    takes (checkpoints every 50 steps; the lean fused steps between re-sorts)."""
    sc = scenes.dam_break()
    from paper_2303_02346_gb300.simulator import Simulator
    T = 50
    sim = Simulator(sc, checkpoint_every=sc.checkpoint_every, max_steps=sc.n_steps)
    sim.reset()
    sim.step(T)
    x, v = sim.state()
    sim.close()
    xo, vo, _, _ = oracle_forward(sc, n_steps=T)
    assert rel(x.cpu(), xo) < TOL_X
    assert rel(v.cpu(), vo) < TOL_X
    # the column has started to collapse: the water moved
    assert float(np.abs(vo).max()) > 0.05


def test_dam_break_scaled_copy_full_horizon_gradient_k50():
    """The 2M-particle scene's recompute path at 1/500 of its particles on a
    32^3 grid (same column height in cells): the full 1000-step horizon with a
    checkpoint every 50 steps (20 chunks, re-sorts at every checkpoint, the
    two-buffer recompute overlapped with the reverse sweep), gradients of the
    final-position loss w.r.t. the initial state against the oracle's."""
    sc = scenes.dam_break(scale=0.002, grid_n=32)
    assert sc.n_steps == 1000 and sc.checkpoint_every == 50
    from paper_2303_02346_gb300.simulator import Simulator
    sim = Simulator(sc)
    sim.reset()
    sim.step(sc.n_steps)
    x, v = sim.state()
    L = sc.loss
    Lg = float(sim.position_loss(L["target"], L["weight"], scene=0)[0])
    gx, gv, _ = sim.backward()
    sim.close()
    ref = oracle_grad(sc, checkpoint=True)
    xo, vo, _, _ = oracle_forward(sc)
    assert rel(x.cpu(), xo) < TOL_X and rel(v.cpu(), vo) < TOL_X
    assert abs(Lg - ref["loss"]) / abs(ref["loss"]) < TOL_X
    assert rel(gx.cpu(), ref["x0"]) < TOL_G
    assert rel(gv.cpu(), ref["v0"]) < TOL_G
