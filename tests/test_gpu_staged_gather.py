"""The fused G2P -> P2G kernel with its gather staged in shared memory by a
tensor-copy (TMA) load of the CTA's grid box, against the FP64 oracle: the
200k-particle tool scene at 5% size with gradients (the recompute's fused
steps stage from the per-step grids), many scenes of uneven sizes in one
handle (the box carries the scene coordinate), and a thin cloud whose CTAs'
boxes do not fit (those CTAs gather from global memory). Tolerances as in the
other parity tests."""
import pytest

import scenes
from gpu_util import oracle_forward, oracle_grad, rel

pytestmark = pytest.mark.gpu
TOL_X, TOL_G = 1e-4, 1e-3


def _sim(sc, **kw):
    from paper_2303_02346_gb300 import binding as B
    from paper_2303_02346_gb300.simulator import Simulator
    sim = Simulator(sc, **kw)
    B.sim_set_launch(sim.h, 256, 128, 4, 8, 0, 0, 1)
    sim.reset()
    return sim


def test_staged_gather_tool_scene_forward_and_gradients():
    sc = scenes.multi_material(scale=0.05, grid_n=64, n_steps=40, checkpoint_every=20)
    sim = _sim(sc)
    sim.step(sc.n_steps)
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


def test_staged_gather_batched_scenes():
    sc = scenes.batched_scenes(n_scenes=8, grid_n=32, n_steps=12, lo=2000, hi=12000)
    sim = _sim(sc, checkpoint_every=0, max_steps=12)
    sim.step(12)
    for s_i in (0, 4, 7):
        xo, vo, _, _ = oracle_forward(sc, n_steps=12, scene_index=s_i)
        x, v = sim.state(scene=s_i)
        assert rel(x.cpu(), xo) < TOL_X, s_i
        assert rel(v.cpu(), vo) < TOL_X, s_i
    sim.close()


def test_staged_gather_sparse_cloud_falls_back():
    """Particles spread thinly over the grid: every CTA's stencil box exceeds
    the staged box, so the kernel gathers from global memory."""
    sc = scenes.small_block(seed=71, grid_n=32, kinds=[0, 1], ppc=1, size_cells=20, n_steps=6)
    sim = _sim(sc, checkpoint_every=0, max_steps=6)
    sim.step(6)
    x, v = sim.state()
    xo, vo, _, _ = oracle_forward(sc, n_steps=6)
    assert rel(x.cpu(), xo) < TOL_X and rel(v.cpu(), vo) < TOL_X
    sim.close()
