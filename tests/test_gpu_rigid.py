"""GPU-vs-oracle parity of particle-represented rigid bodies (Sec. 3.2 "Rigid
body") through the C-ABI: the rigidity projection after every G2P, its
adjoint in the reverse sweep (with the chunk recompute), forward-only runs
with periodic re-sorts, several scenes with one object each, and a tool
pushing a rigid block in liquid (gradient w.r.t. the actions).

Tolerances as in test_gpu_parity: relative L2 <= 1e-4 on the state, <= 1e-3
on gradients."""
import numpy as np
import pytest
import torch

import scenes
from gpu_util import oracle_forward, oracle_grad, rel

pytestmark = pytest.mark.gpu

TOL_X = 1e-4
TOL_G = 1e-3
RIGID = scenes.RIGID


def _sim(sc, **kw):
    from paper_2303_02346_gb300.simulator import Simulator
    s = Simulator(sc, **kw)
    s.reset()
    return s


def _check_state(sim, sc, scene=0):
    x, v, C, F = sim.state(scene=scene, with_CF=True)
    xo, vo, Co, Fo = oracle_forward(sc, scene_index=scene)
    assert rel(x.cpu(), xo) < TOL_X
    assert rel(v.cpu(), vo) < TOL_X
    lo = int(sum(sc.scene_counts[:scene]))
    mat = sc.mat[lo:lo + sc.scene_counts[scene]]
    rig = np.isin(mat, [i for i, m in enumerate(sc.materials) if m.kind == RIGID])
    assert rig.any()
    # the rigid particles carry the object's rotation in F and its spin in C
    assert rel(F.cpu()[rig], Fo[rig]) < TOL_X
    assert rel(C.cpu()[rig], Co[rig]) < TOL_X
    return x, v


@pytest.mark.parametrize("kinds", [[RIGID], [0, RIGID], [0, 1, RIGID]])
def test_rigid_forward_and_gradient(kinds):
    sc = scenes.small_block(61, 16, kinds, ppc=4, size_cells=6, lo_cell=(5, 3, 5), n_steps=24,
                            v0=(0.2, -0.4, 0.1), spin=10.0, dt=2e-4, yield_stress=5.0, E=2e4)
    sim = _sim(sc, checkpoint_every=8)
    sim.step(sc.n_steps)
    _check_state(sim, sc)
    sim.position_loss(sc.loss["target"], 1.0, scene=0)
    gx, gv, _ = sim.backward()
    ref = oracle_grad(sc)
    assert rel(gx.cpu(), ref["x0"]) < TOL_G
    assert rel(gv.cpu(), ref["v0"]) < TOL_G


def test_rigid_forward_only_with_resorts():
    """Forward-only runs re-sort the particles every few steps; the rest
    offsets are looked up through the sort's permutation."""
    sc = scenes.small_block(62, 16, [0, RIGID], ppc=3, size_cells=6, lo_cell=(5, 3, 5), n_steps=20,
                            v0=(0.1, -0.2, 0.3), spin=-12.0, dt=2e-4)
    for r in (1, 3):
        sim = _sim(sc, checkpoint_every=0, resort_every=r)
        sim.step(sc.n_steps)
        _check_state(sim, sc)
        sim.close()


def test_rigid_objects_in_several_scenes():
    """Each scene's rigid particles form their own object."""
    parts = [scenes.small_block(63 + i, 16, [0, RIGID], ppc=p, size_cells=s, lo_cell=(5, 3, 5), n_steps=16,
                                spin=8.0 * (i + 1), dt=2e-4)
             for i, (p, s) in enumerate([(2, 4), (3, 6)])]
    sc = scenes.merge_scenes(parts)
    sim = _sim(sc, checkpoint_every=5)
    sim.step(sc.n_steps)
    for s_i in range(2):
        _check_state(sim, sc, scene=s_i)
    sim.position_loss(sc.loss["target"], 1.0, scene=-1)
    gx, gv, _ = sim.backward()
    off = 0
    for s_i in range(2):
        ref = oracle_grad(sc, scene_index=s_i)
        cnt = sc.scene_counts[s_i]
        assert rel(gx.cpu()[off:off + cnt], ref["x0"]) < TOL_G, s_i
        assert rel(gv.cpu()[off:off + cnt], ref["v0"]) < TOL_G, s_i
        off += cnt


def test_tool_pushing_rigid_block_gradient_wrt_actions():
    sc = scenes.small_block(64, 16, [0, RIGID], ppc=2, size_cells=6, lo_cell=(5, 3, 5), n_steps=30,
                            dt=2e-4, tool=True)
    sim = _sim(sc, checkpoint_every=7)
    sim.step(sc.n_steps)
    _check_state(sim, sc)
    sim.position_loss(sc.loss["target"], 1.0, scene=0)
    gx, gv, ga = sim.backward()
    ref = oracle_grad(sc, want_actions=True)
    assert np.abs(ref["actions"]).max() > 0
    assert rel(gx.cpu(), ref["x0"]) < TOL_G
    assert rel(ga.cpu()[0], ref["actions"]) < TOL_G
