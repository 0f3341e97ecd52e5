"""The persistent forward (the forward's steps between re-sorts as one
cooperative launch: fused G2P -> constitutive -> P2G phase, grid-wide barrier,
grid update, barrier, per step) against the FP64 oracle, on one scene and on
many scenes in one handle, with and without checkpoints; and the bound on its
barrier waits, exercised by the barrier self-test (a wait that cannot complete
gives up after its timeout, reports SIM_E_TIMEOUT and leaves the context
usable). Tolerances as in the other parity tests."""
import numpy as np
import pytest
import torch

import scenes
from gpu_util import oracle_forward, oracle_grad, rel

pytestmark = pytest.mark.gpu
TOL_X, TOL_G = 1e-4, 1e-3


def _sim(sc, **kw):
    from paper_2303_02346_gb300 import binding as B
    from paper_2303_02346_gb300.simulator import Simulator
    sim = Simulator(sc, **kw)
    B.sim_set_launch(sim.h, 256, 128, 4, 8, 0, 1)
    sim.reset()
    return sim


def test_persistent_forward_single_scene_with_gradients():
    from paper_2303_02346_gb300 import binding as B
    sc = scenes.multi_material(scale=0.05, grid_n=64, n_steps=40, checkpoint_every=20)
    sim = _sim(sc)
    B.sim_profile_enable(sim.h, 1)
    # two calls: a call that runs to the horizon from the first chunk the
    # forward keeps would run its chunks the way the recompute does; these run
    # as persistent runs (counted per step), and the backward recomputes every
    # chunk
    sim.step(sc.checkpoint_every)
    sim.step(sc.n_steps - sc.checkpoint_every)
    prof = B.sim_profile_read(sim.h)
    B.sim_profile_enable(sim.h, 0)
    assert prof["fwd_run"][1] == sc.n_steps, prof
    x, v = sim.state()
    xo, vo, _, _ = oracle_forward(sc)
    assert rel(x.cpu(), xo) < TOL_X and rel(v.cpu(), vo) < TOL_X
    L = sc.loss
    sim.grid_mass_loss(L["target_mass"], L["target_dist"], L["total_mass"])
    gx, gv, ga = sim.backward()
    ref = oracle_grad(sc, want_actions=True)
    assert rel(ga.cpu()[0], ref["actions"]) < TOL_G
    assert rel(gx.cpu(), ref["x0"]) < TOL_G
    sim.close()


@pytest.mark.parametrize("T", [1, 2, 9])
def test_persistent_forward_without_checkpoints_and_short_runs(T):
    """Re-sorts every 4 steps: runs of 1 to 4 steps, the state completed by
    the G2P after each run (runs of one step are a lone P2G)."""
    from paper_2303_02346_gb300 import binding as B
    from paper_2303_02346_gb300.simulator import Simulator
    sc = scenes.small_block(seed=61, grid_n=16, kinds=[0, 1, 2], ppc=2, size_cells=6, v0=(0.3, 0.0, -0.2),
                            spin=2.0, n_steps=T)
    sim = Simulator(sc, checkpoint_every=0, max_steps=T)
    B.sim_set_launch(sim.h, 128, 128, 1, 4, 0, 1)
    sim.reset()
    sim.step(T)
    x, v = sim.state()
    xo, vo, _, _ = oracle_forward(sc, n_steps=T)
    assert rel(x.cpu(), xo) < TOL_X and rel(v.cpu(), vo) < TOL_X
    sim.close()


def test_persistent_forward_batched_scenes():
    """Many scenes of uneven sizes in one handle stepped by the persistent
    launch (tiles of particles balanced by a counter across all scenes)."""
    sc = scenes.batched_scenes(n_scenes=8, grid_n=32, n_steps=12, lo=2000, hi=12000)
    sim = _sim(sc, checkpoint_every=6, max_steps=12)
    sim.step(5)
    sim.step(7)
    sim.position_loss(sc.loss["target"], 1.0, scene=-1)
    gx, gv, ga = sim.backward()
    offs = np.concatenate([[0], np.cumsum(sc.scene_counts)])
    for s_i in (0, 3, 7):
        xo, vo, _, _ = oracle_forward(sc, n_steps=12, scene_index=s_i)
        x, v = sim.state(scene=s_i)
        assert rel(x.cpu(), xo) < TOL_X, s_i
        assert rel(v.cpu(), vo) < TOL_X, s_i
    ref = oracle_grad(sc, n_steps=12, scene_index=3, want_actions=True)
    assert rel(gx.cpu()[offs[3]:offs[4]], ref["x0"]) < TOL_G
    sim.close()


def test_grid_barrier_completes_and_its_wait_is_bounded():
    from paper_2303_02346_gb300 import binding as B
    # every CTA arrives: all barriers complete
    st, passed = B.sim_selftest_grid_barrier(152, 0, 50, 2000.0)
    assert st == 0 and passed == 152 * 50
    # one arrival never comes: every CTA gives up after 20 ms
    st, passed = B.sim_selftest_grid_barrier(64, 1, 3, 20.0)
    assert st == 7 and passed == 0  # SIM_E_TIMEOUT
    # the context is still usable
    st, passed = B.sim_selftest_grid_barrier(8, 0, 4, 2000.0)
    assert st == 0 and passed == 32
    sc = scenes.small_block(seed=62, grid_n=16, kinds=[0], ppc=2, size_cells=4, n_steps=3)
    sim = _sim(sc, checkpoint_every=0, max_steps=3)
    sim.step(3)
    x, _ = sim.state()
    xo, _, _, _ = oracle_forward(sc, n_steps=3)
    assert rel(x.cpu(), xo) < TOL_X
    sim.close()
