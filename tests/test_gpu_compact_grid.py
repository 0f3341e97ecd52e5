"""Chunk buffers that keep each step's grid as a compact copy (the active-block
list entries' nodes, up to an eighth of the grid's blocks) instead of a
full-size grid: the forward that reaches the horizon keeps chunks in them,
the reverse sweep expands each step back into a full-size grid before the
kernels that read it by node index, and a chunk whose steps outgrow the copy
is recomputed instead. Gradients against the FP64 oracle in both cases."""
import numpy as np
import pytest

import scenes
from gpu_util import oracle_grad, rel

pytestmark = pytest.mark.gpu

TOL_X = 1e-4
TOL_G = 1e-3


def _run(sc, k, profile):
    from paper_2303_02346_gb300.simulator import Simulator
    sim = Simulator(sc, checkpoint_every=k)
    sim.reset()
    if profile:
        sim.profile(True)
    sim.step(sc.n_steps)
    L = sim.position_loss(sc.loss["target"], 1.0, scene=0)[0]
    gx, gv, _ = sim.backward()
    prof = sim.profile_read() if profile else {}
    sim.close()
    return L, gx.cpu(), gv.cpu(), prof


@pytest.mark.parametrize("profile", [False, True])
def test_compact_chunks_swept_without_recompute(profile):
    """Water cube on the floor, 50 steps, a checkpoint every 10: five chunk
    buffers, of which buffers 2-4 (chunks 2, 1, 0) are compact; the cube's
    27 grid blocks fit the 64-block copy of the 32^3 grid, so the backward
    sweeps every chunk as the forward left it (the profiled run counts the
    expansions: one per step of the three compact chunks)."""
    sc = scenes.water_cube(on_floor=True, v_down=1.0)
    L, gx, gv, prof = _run(sc, 10, profile)
    ref = oracle_grad(sc)
    assert abs(L - ref["loss"]) / ref["loss"] < TOL_X
    assert rel(gx, ref["x0"]) < TOL_G
    assert rel(gv, ref["v0"]) < TOL_G
    if profile:
        assert prof.get("expand", (0.0, 0))[1] == 3 * 10
        # nothing recomputed: the forward ran every step once
        assert prof.get("g2p2g", (0.0, 0))[1] == 50 - 5


def test_overflowing_compact_chunks_are_recomputed():
    """A thin cloud over 20^3 cells of the 32^3 grid touches about 200 grid
    blocks, more than the 64 a compact step holds: the compact chunks (0 and 1
    of four) overflow, are not swept from their copies (no expansion) but
    recomputed, and the gradient still matches the oracle."""
    sc = scenes.small_block(31, 32, [0, 1, 2], ppc=1, size_cells=20, lo_cell=(6, 6, 6), n_steps=16,
                            v0=(0.1, -0.2, 0.05), dt=2e-4, yield_stress=5.0, E=2e4)
    keep = np.random.Generator(np.random.PCG64(31)).random(sc.n_particles) < 0.2
    sc.x, sc.v, sc.mat = sc.x[keep], sc.v[keep], sc.mat[keep]
    sc.scene_counts = [int(keep.sum())]
    base = np.floor(sc.x * sc.grid_n - 0.5).astype(int)
    assert len({tuple(b) for b in base // 4}) > 64
    for profile in (False, True):
        L, gx, gv, prof = _run(sc, 4, profile)
        ref = oracle_grad(sc)
        assert abs(L - ref["loss"]) / ref["loss"] < TOL_X
        assert rel(gx, ref["x0"]) < TOL_G
        assert rel(gv, ref["v0"]) < TOL_G
        if profile:
            assert prof.get("expand", (0.0, 0))[1] == 0
            # chunks 0 and 1 recomputed: 2 x (4 - 1) fused steps more than the forward's 12
            assert prof.get("g2p2g", (0.0, 0))[1] == 12 + 6
