"""Per-step losses and past states through the C-ABI, against the FP64 oracle.

App. C writes the task losses as sums over the trajectory, L = sum_t
CD(s_t, s*_t); the library takes each term's gradient as a seed of the state
at step t (evaluated while the trajectory passes step t, or later on a state
it keeps) and propagates all of them in one sim_backward. These tests pin the
step bookkeeping: seeds inside a checkpoint chunk, at a chunk boundary and at
the final step, a loss evaluated afterwards on a retained checkpoint state, a
caller gradient handed in for a past step, the retained states sim_get_state
returns, and the tool pose of any step.
"""
import numpy as np
import pytest
import torch

import scenes
from gpu_util import rel
from oracle import mpm as omp
from oracle import tool as otl

pytestmark = pytest.mark.gpu
DT = torch.float64
TOL_X, TOL_G = 1e-4, 1e-3


def _scene():
    # 10k particles of the three-material tool scene on 64^3, 24 steps,
    # checkpoints every 6 (chunks [0,6) [6,12) [12,18) [18,24))
    return scenes.multi_material(scale=0.05, grid_n=64, n_steps=24, checkpoint_every=6)


def _targets(sc, steps):
    """A distinct box target per loss term, so that a seed applied at the
    wrong step changes the gradient."""
    M = sc.loss["total_mass"]
    out = {}
    for i, t in enumerate(steps):
        c = (0.46 + 0.02 * i, 0.08 + 0.01 * i, 0.5 - 0.015 * i)
        out[t] = scenes.box_target(sc.grid_n, c, (0.08, 0.04, 0.07), M)
    return out, M


def _oracle_states(sc, x0, v0, act):
    return omp.rollout(sc, x0=x0, v0=v0, actions=act, keep_states=True)


def _leaf(sc):
    x0 = torch.tensor(sc.x, dtype=DT, requires_grad=True)
    v0 = torch.tensor(sc.v, dtype=DT, requires_grad=True)
    act = torch.tensor(sc.tool_actions[0], dtype=DT, requires_grad=True)
    return x0, v0, act


def test_time_summed_grid_mass_loss_in_one_backward():
    from paper_2303_02346_gb300.simulator import Simulator
    sc = _scene()
    # 3: inside chunk 0; 6: chunk 0's last state (= checkpoint 1, evaluated
    # while passing); 11: inside chunk 1; 12: checkpoint 2, evaluated at the
    # end from the retained checkpoint; 24: the final state
    steps = [3, 6, 11, 12, 24]
    tg, M = _targets(sc, steps)
    sim = Simulator(sc)
    sim.reset()
    losses = {}
    cur = 0
    for t in [3, 6, 11, 24]:
        sim.step(t - cur)
        cur = t
        losses[t] = sim.grid_mass_loss(tg[t][0], tg[t][1], M)
    losses[12] = sim.grid_mass_loss(tg[12][0], tg[12][1], M, step=12)
    gx, gv, ga = sim.backward()

    x0, v0, act = _leaf(sc)
    states = _oracle_states(sc, x0, v0, act)
    model = omp.Model(sc)
    mass, _ = model.particle_mass_volume(sc.mat)
    terms = {t: omp.grid_mass_loss(states[t][0], mass, model, tg[t][0], tg[t][1], M) for t in steps}
    for t in steps:
        assert abs(losses[t] - terms[t].item()) / abs(terms[t].item()) < TOL_X, t
    sum(terms.values()).backward()
    assert np.abs(act.grad.numpy()).max() > 0
    assert rel(ga.cpu()[0], act.grad.numpy()) < TOL_G
    assert rel(gx.cpu(), x0.grad.numpy()) < TOL_G
    assert rel(gv.cpu(), v0.grad.numpy()) < TOL_G
    sim.close()


def test_caller_gradients_for_past_steps_and_position_loss_on_a_checkpoint():
    """dL/dx of a point-goal term at step 7 (inside chunk 1) handed in after the
    trajectory reached step 24, plus the library's own point-goal loss on the
    retained checkpoint of step 18: one backward gives the gradient of the sum."""
    from paper_2303_02346_gb300.simulator import Simulator
    sc = _scene()
    target7, target18 = (0.5, 0.2, 0.45), (0.52, 0.1, 0.5)
    x0, v0, act = _leaf(sc)
    states = _oracle_states(sc, x0, v0, act)
    with torch.no_grad():
        g7 = 2.0 * 0.5 * (states[7][0] - torch.tensor(target7, dtype=DT))  # weight 0.5
    sim = Simulator(sc)
    sim.reset()
    sim.step(24)
    sim.add_loss_grad(g7.float().cuda().contiguous(), None, step=7)
    L18 = float(sim.position_loss(target18, 2.0, scene=0, step=18)[0])
    gx, gv, ga = sim.backward()
    L = 0.5 * omp.position_loss(states[7][0], target7) + 2.0 * omp.position_loss(states[18][0], target18)
    assert abs(L18 - 2.0 * omp.position_loss(states[18][0], target18).item()) / L18 < TOL_X
    L.backward()
    assert rel(gx.cpu(), x0.grad.numpy()) < TOL_G
    assert rel(gv.cpu(), v0.grad.numpy()) < TOL_G
    assert rel(ga.cpu()[0], act.grad.numpy()) < TOL_G
    sim.close()


def test_retained_states_and_refusals():
    from paper_2303_02346_gb300 import binding as B
    from paper_2303_02346_gb300.simulator import Simulator
    sc = _scene()
    with torch.no_grad():
        states = omp.rollout(sc, keep_states=True)
    sim = Simulator(sc)
    sim.reset()
    sim.step(20)
    for t in (0, 6, 12, 18, 20, -1):
        x, v, C, F = sim.state(with_CF=True, step=t)
        ref = states[20 if t == -1 else t]
        assert rel(x.cpu(), ref[0]) < TOL_X, t
        if t != 0:
            assert rel(v.cpu(), ref[1]) < TOL_X, t
            assert rel(C.cpu(), ref[2]) < 1e-3, t
        else:
            assert torch.equal(x.cpu(), torch.tensor(sc.x, dtype=torch.float32))
    for t in (5, 13, 19, 21):
        with pytest.raises(B.SimError) as e:
            sim.state(step=t)
        assert e.value.status == 6, t
    tg, M = _targets(sc, [5])
    with pytest.raises(B.SimError) as e:  # not a retained state
        sim.grid_mass_loss(tg[5][0], tg[5][1], M, step=5)
    assert e.value.status == 6
    with pytest.raises(B.SimError) as e:  # in the future
        sim.add_loss_grad(torch.zeros(sc.n_particles, 3, device="cuda"), None, step=21)
    assert e.value.status == 6
    with pytest.raises(B.SimError) as e:  # step 0 takes no seed
        sim.add_loss_grad(torch.zeros(sc.n_particles, 3, device="cuda"), None, step=0)
    assert e.value.status == 6
    sim.close()


def test_tool_pose_of_every_step_matches_oracle_kinematics():
    from paper_2303_02346_gb300.simulator import Simulator
    sc = _scene()
    sim = Simulator(sc)
    sim.reset()
    P, Q, PD, OM = otl.tool_trajectory(torch.tensor(sc.tool_pose0[0], dtype=DT),
                                       torch.tensor(sc.tool_actions[0], dtype=DT), sc.n_steps, sc.dt,
                                       sc.substeps_per_action)
    for t in (0, 1, 9, 10, 17, 23):
        pose = sim.tool_pose(t).cpu().double()[0]
        q = Q[t] * torch.sign(Q[t][0]) * torch.sign(pose[3])
        assert torch.allclose(pose[:3], P[t], atol=1e-6), t
        assert torch.allclose(pose[3:7], q, atol=1e-6), t
        assert torch.allclose(pose[7:10], PD[t].float().double(), atol=1e-6), t
        assert torch.allclose(pose[10:13], OM[t].float().double(), atol=1e-6), t
    sim.close()
