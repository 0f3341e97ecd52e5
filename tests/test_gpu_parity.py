"""GPU-vs-oracle parity of the CUDA library through the C-ABI.

Tolerances: relative L2 error <= 1e-4 on
particle positions and velocities after the stated steps, <= 1e-3 on
gradients. The GPU computes in FP32, the oracle in FP64; FP32 atomics make the
GPU result vary run to run at ~1e-7, any result within tolerance is accepted.
"""
import numpy as np
import pytest
import torch

import scenes
from gpu_util import oracle_forward, oracle_grad, rel

pytestmark = pytest.mark.gpu

TOL_X = 1e-4
TOL_G = 1e-3


def _sim(sc, **kw):
    from paper_2303_02346_gb300.simulator import Simulator
    s = Simulator(sc, **kw)
    s.reset()
    return s


def test_water_cube_forward_parity():
    """8,192 water particles, 32^3 grid, 50 steps."""
    sc = scenes.water_cube()
    sim = _sim(sc, checkpoint_every=0)
    sim.step(sc.n_steps)
    x, v, C, F = sim.state(with_CF=True)
    xo, vo, Co, Fo = oracle_forward(sc)
    assert rel(x.cpu(), xo) < TOL_X
    assert rel(v.cpu(), vo) < TOL_X
    # liquid carries J only: F = diag(J, 1, 1); compare J = det F
    assert rel(F.cpu()[:, 0, 0], np.linalg.det(Fo)) < TOL_X
    # the cube is in free fall for these 50 steps, so C is zero up to rounding:
    # compare it on the scale of the velocity gradient |v| / dx
    scale = float(np.abs(vo).max()) * sc.grid_n
    assert float(np.abs(C.cpu().numpy() - Co).max()) < 1e-4 * scale


def test_water_cube_gradient_parity():
    """Adjoint of the final-position loss w.r.t. x0 and v0, checkpoints every 10
    steps (5 chunks recomputed)."""
    sc = scenes.water_cube()
    sim = _sim(sc, checkpoint_every=10)
    sim.step(sc.n_steps)
    L = sim.position_loss(sc.loss["target"], 1.0, scene=0)[0]
    gx, gv, _ = sim.backward()
    ref = oracle_grad(sc)
    assert abs(L - ref["loss"]) / ref["loss"] < TOL_X
    assert rel(gx.cpu(), ref["x0"]) < TOL_G
    assert rel(gv.cpu(), ref["v0"]) < TOL_G


def test_water_cube_on_floor_forward_and_gradient_parity():
    """The water cube resting on the sticky floor and pushed down at 1 m/s:
    the liquid is compressed against the wall from the first step (J falls to
    about 0.84 in the oracle), so the pressure term of the P2G stress and the
    affine C are exercised, not only free fall. Forward after 50 steps, then the
    final-position gradient with checkpoints every 10 steps."""
    sc = scenes.water_cube(on_floor=True, v_down=1.0)
    sim = _sim(sc, checkpoint_every=0)
    sim.step(sc.n_steps)
    x, v, C, F = sim.state(with_CF=True)
    xo, vo, Co, Fo = oracle_forward(sc)
    Jo = np.linalg.det(Fo)
    assert Jo.min() < 0.9 and float(np.abs(Co).max()) > 1.0   # the case is not vacuous
    print("water cube on floor: rel x %.2e v %.2e J %.2e C %.2e" % (
        rel(x.cpu(), xo), rel(v.cpu(), vo), rel(F.cpu()[:, 0, 0], Jo), rel(C.cpu(), Co)))
    assert rel(x.cpu(), xo) < TOL_X
    assert rel(v.cpu(), vo) < TOL_X
    assert rel(F.cpu()[:, 0, 0], Jo) < TOL_X
    assert rel(C.cpu(), Co) < TOL_X
    sim.close()

    sim = _sim(sc, checkpoint_every=10)
    sim.step(sc.n_steps)
    L = sim.position_loss(sc.loss["target"], 1.0, scene=0)[0]
    gx, gv, _ = sim.backward()
    ref = oracle_grad(sc)
    print("water cube on floor: gradient rel x0 %.2e v0 %.2e" % (rel(gx.cpu(), ref["x0"]),
                                                                 rel(gv.cpu(), ref["v0"])))
    assert abs(L - ref["loss"]) / ref["loss"] < TOL_X
    assert rel(gx.cpu(), ref["x0"]) < TOL_G
    assert rel(gv.cpu(), ref["v0"]) < TOL_G
    sim.close()


@pytest.mark.parametrize("kinds", [[1], [2], [3], [4], [0, 1, 2], [0, 1, 2, 3, 4]])
def test_small_block_materials_forward_and_gradient(kinds):
    sc = scenes.small_block(21, 16, kinds, ppc=4, size_cells=6, lo_cell=(5, 3, 5), n_steps=24,
                            v0=(0.2, -0.4, 0.1), spin=10.0, dt=2e-4, yield_stress=5.0, E=2e4)
    sim = _sim(sc, checkpoint_every=8)
    sim.step(sc.n_steps)
    x, v, C, F = sim.state(with_CF=True)
    xo, vo, Co, Fo = oracle_forward(sc)
    assert rel(x.cpu(), xo) < TOL_X
    assert rel(v.cpu(), vo) < TOL_X
    liquid_idx = [i for i, k in enumerate(kinds) if k in (0, 4)]
    liquid = np.isin(sc.mat, liquid_idx)
    solid = ~liquid
    if solid.any():
        assert rel(F.cpu()[solid], Fo[solid]) < TOL_X
    if liquid.any():  # a liquid carries J only: F = diag(J, 1, 1)
        assert rel(F.cpu()[liquid][:, 0, 0], np.linalg.det(Fo[liquid])) < TOL_X
    if 3 in kinds:
        # the box criterion is active: the final trial F has singular values
        # outside the box, which every step's projection clamps
        m = sc.materials[kinds.index(3)]
        sv = np.linalg.svd(Fo[sc.mat == kinds.index(3)], compute_uv=False)
        assert (sv > 1 + m.crit_stretch).any() and (sv < 1 - m.crit_compress).any()
    sim.position_loss(sc.loss["target"], 1.0, scene=0)
    gx, gv, _ = sim.backward()
    ref = oracle_grad(sc)
    assert rel(gx.cpu(), ref["x0"]) < TOL_G
    assert rel(gv.cpu(), ref["v0"]) < TOL_G


def test_tool_contact_gradient_wrt_actions():
    sc = scenes.small_block(12, 16, [0, 1, 2], ppc=2, size_cells=6, lo_cell=(5, 3, 5), n_steps=30,
                            dt=2e-4, tool=True, yield_stress=20.0)
    sim = _sim(sc, checkpoint_every=7)
    sim.step(sc.n_steps)
    x, v = sim.state()
    xo, vo, _, _ = oracle_forward(sc)
    assert rel(x.cpu(), xo) < TOL_X and rel(v.cpu(), vo) < TOL_X
    sim.position_loss(sc.loss["target"], 1.0, scene=0)
    gx, gv, ga = sim.backward()
    ref = oracle_grad(sc, want_actions=True)
    assert np.abs(ref["actions"]).max() > 0
    assert rel(ga.cpu()[0], ref["actions"]) < TOL_G
    assert rel(gx.cpu(), ref["x0"]) < TOL_G


def test_multi_material_scaled_forward_and_grid_mass_gradient():
    """The three-material tool scene at 5% size (10k particles, 64^3), 60 steps,
    checkpoints every 20, grid-mass loss gradient w.r.t. the tool actions."""
    sc = scenes.multi_material(scale=0.05, grid_n=64, n_steps=60, checkpoint_every=20)
    sim = _sim(sc)
    sim.step(sc.n_steps)
    x, v = sim.state()
    xo, vo, _, _ = oracle_forward(sc)
    assert rel(x.cpu(), xo) < TOL_X and rel(v.cpu(), vo) < TOL_X
    Lg = sim.grid_mass_loss(sc.loss["target_mass"], sc.loss["target_dist"], sc.loss["total_mass"])
    gx, gv, ga = sim.backward()
    ref = oracle_grad(sc, want_actions=True)
    assert abs(Lg - ref["loss"]) / abs(ref["loss"]) < TOL_X
    assert np.abs(ref["actions"]).max() > 0
    assert rel(ga.cpu()[0], ref["actions"]) < TOL_G
    assert rel(gx.cpu(), ref["x0"]) < TOL_G


def test_batched_scenes_match_oracle_per_scene():
    """Three independent scenes of uneven sizes (one with a ragged count) in one
    handle; each matches the oracle run on that scene alone."""
    parts = [scenes.small_block(31 + i, 16, [0, 1, 2], ppc=p, size_cells=s, lo_cell=(5, 3, 5),
                                n_steps=16, dt=2e-4, tool=True)
             for i, (p, s) in enumerate([(2, 4), (3, 5), (1, 7)])]
    sc = scenes.merge_scenes(parts)
    sim = _sim(sc, checkpoint_every=16)
    sim.step(sc.n_steps)
    for s_i in range(3):
        x, v = sim.state(scene=s_i)
        xo, vo, _, _ = oracle_forward(sc, scene_index=s_i)
        assert rel(x.cpu(), xo) < TOL_X, s_i
        assert rel(v.cpu(), vo) < TOL_X, s_i
    sim.position_loss(sc.loss["target"], 1.0, scene=-1)
    gx, gv, ga = sim.backward()
    off = 0
    for s_i in range(3):
        ref = oracle_grad(sc, scene_index=s_i, want_actions=True)
        cnt = sc.scene_counts[s_i]
        assert rel(gx.cpu()[off:off + cnt], ref["x0"]) < TOL_G, s_i
        assert rel(ga.cpu()[s_i], ref["actions"]) < TOL_G, s_i
        off += cnt


def test_empty_scene_and_forward_only_resort():
    a = scenes.small_block(41, 16, [0, 1], ppc=3, size_cells=5, lo_cell=(5, 3, 5), n_steps=12, dt=2e-4)
    empty = scenes.small_block(42, 16, [0, 1], ppc=3, size_cells=5, lo_cell=(5, 3, 5), n_steps=12, dt=2e-4)
    empty.x = empty.x[:0]
    empty.v = empty.v[:0]
    empty.mat = empty.mat[:0]
    empty.scene_counts = [0]
    sc = scenes.merge_scenes([empty, a])
    xo, vo, _, _ = oracle_forward(a)
    for k, r in [(0, 1), (0, 5), (4, 0)]:
        sim = _sim(sc, checkpoint_every=k, resort_every=r)
        sim.step(sc.n_steps)
        x, v = sim.state(scene=1)
        assert rel(x.cpu(), xo) < TOL_X and rel(v.cpu(), vo) < TOL_X, (k, r)
        assert sim.state(scene=0)[0].shape[0] == 0
        sim.close()


def test_domain_error_reported_not_faulted():
    from paper_2303_02346_gb300.binding import SimError
    sc = scenes.small_block(51, 16, [0], ppc=2, size_cells=3, lo_cell=(11, 8, 8), n_steps=40,
                            v0=(60.0, 0.0, 0.0), dt=2e-4, bound=0, gravity=(0.0, 0.0, 0.0))
    sim = _sim(sc, checkpoint_every=0)
    with pytest.raises(SimError) as e:
        sim.step(sc.n_steps)
    assert e.value.status == 4
    # the context is still usable
    sim2 = _sim(scenes.water_cube(n_steps=2), checkpoint_every=0)
    sim2.step(2)
    torch.cuda.synchronize()


@pytest.mark.parametrize("graphs", [True, False])
def test_graph_replay_and_direct_launch_match_oracle(graphs):
    """The same trajectory run twice (the second run replays the captured
    graphs of sim_step and sim_backward) and with graphs off."""
    from paper_2303_02346_gb300.simulator import Simulator
    sc = scenes.small_block(71, 16, [0, 1, 2], ppc=2, size_cells=6, lo_cell=(5, 3, 5), n_steps=24,
                            dt=2e-4, tool=True, yield_stress=20.0)
    sim = Simulator(sc, checkpoint_every=6, graphs=graphs)
    ref = oracle_grad(sc, want_actions=True)
    xo, vo, _, _ = oracle_forward(sc)
    for rep in range(2):
        sim.reset()
        sim.step(sc.n_steps)
        x, v = sim.state()
        assert rel(x.cpu(), xo) < TOL_X and rel(v.cpu(), vo) < TOL_X, rep
        sim.position_loss(sc.loss["target"], 1.0, scene=0)
        gx, gv, ga = sim.backward()
        assert rel(gx.cpu(), ref["x0"]) < TOL_G, rep
        assert rel(ga.cpu()[0], ref["actions"]) < TOL_G, rep


def test_autotune_choices_keep_parity():
    from paper_2303_02346_gb300 import binding as B
    from paper_2303_02346_gb300.simulator import Simulator
    sc = scenes.multi_material(scale=0.05, grid_n=64, n_steps=40, checkpoint_every=20)
    sim = Simulator(sc)
    sim.reset()
    choices = B.sim_autotune(sim.h, 8)
    assert choices[0] in (128, 256) and choices[1] in (128, 256, 512) and choices[2] in (1, 2, 4)
    assert choices[4] in (0, 1) and choices[5] in (0, 1) and choices[6] in (0, 1) and choices[7] in (3, 4)
    assert sim.current_step == 0
    sim.step(sc.n_steps)
    x, v = sim.state()
    xo, vo, _, _ = oracle_forward(sc)
    assert rel(x.cpu(), xo) < TOL_X and rel(v.cpu(), vo) < TOL_X
    L = sc.loss
    sim.grid_mass_loss(L["target_mass"], L["target_dist"], L["total_mass"])
    gx, gv, ga = sim.backward()
    ref = oracle_grad(sc, want_actions=True)
    assert rel(ga.cpu()[0], ref["actions"]) < TOL_G
    # every launch shape gives the same trajectory and gradient
    for st, gt, gb, rs, fu, pe, sg, oc in [(128, 128, 1, 4, 1, 0, 1, 3), (256, 512, 2, 32, 0, 1, 0, 4),
                                           (128, 256, 4, 8, 0, 0, 0, 3), (256, 128, 4, 8, 1, 1, 1, 3),
                                           (128, 128, 2, 4, 1, 1, 0, 3), (256, 256, 4, 16, 0, 0, 1, 4),
                                           (256, 128, 4, 8, 0, 0, 0, 4)]:
        sim2 = Simulator(sc)
        B.sim_set_launch(sim2.h, st, gt, gb, rs, fu, pe, sg, oc)
        sim2.reset()
        sim2.step(sc.n_steps)
        x2, _ = sim2.state()
        assert rel(x2.cpu(), xo) < TOL_X, (st, gt, gb)
        sim2.grid_mass_loss(L["target_mass"], L["target_dist"], L["total_mass"])
        _, _, ga2 = sim2.backward()
        assert rel(ga2.cpu()[0], ref["actions"]) < TOL_G, (st, gt, gb)
        sim2.close()
        sim3 = Simulator(sc, checkpoint_every=0)
        B.sim_set_launch(sim3.h, st, gt, gb, rs, fu, pe, sg, oc)
        sim3.reset()
        sim3.step(sc.n_steps)
        x3, _ = sim3.state()
        assert rel(x3.cpu(), xo) < TOL_X, (st, gt, gb, rs)
        sim3.close()


def test_bad_material_index_rejected():
    from paper_2303_02346_gb300.binding import SimError
    sc = scenes.small_block(52, 16, [0, 1], ppc=2, size_cells=3, n_steps=2)
    sc.mat = sc.mat.copy()
    sc.mat[3] = 7
    from paper_2303_02346_gb300.simulator import Simulator
    sim = Simulator(sc, checkpoint_every=0)
    with pytest.raises(SimError) as e:
        sim.set_particles()
    assert e.value.status == 1


def test_autograd_function_matches_backward():
    from paper_2303_02346_gb300.simulator import Simulator, rollout
    sc = scenes.small_block(61, 16, [0, 1, 2], ppc=2, size_cells=5, lo_cell=(5, 3, 5), n_steps=12,
                            dt=2e-4, tool=True)
    sim = Simulator(sc, checkpoint_every=5)
    x0 = torch.tensor(sc.x, dtype=torch.float32, device="cuda", requires_grad=True)
    v0 = torch.tensor(sc.v, dtype=torch.float32, device="cuda", requires_grad=True)
    act = torch.tensor(sc.tool_actions, dtype=torch.float32, device="cuda", requires_grad=True)
    x, v = rollout(sim, sc.n_steps, x0, v0, act)
    t = torch.tensor(sc.loss["target"], dtype=torch.float32, device="cuda")
    L = ((x - t) ** 2).sum()
    L.backward()
    ref = oracle_grad(sc, want_actions=True)
    assert rel(x0.grad.cpu(), ref["x0"]) < TOL_G
    assert rel(act.grad.cpu()[0], ref["actions"]) < TOL_G


def _tile_nodes_per_range(x, grid_n, per):
    """Nodes of the bounding box (stencil origins + 2) of each run of `per`
    particles in cell Morton order: what a CTA's scatter tile must hold."""
    base = np.floor(x * grid_n - 0.5).astype(np.int64)

    def spread(v):
        v = v & 0x3ff
        v = (v | (v << 16)) & 0x030000ff
        v = (v | (v << 8)) & 0x0300f00f
        v = (v | (v << 4)) & 0x030c30c3
        return (v | (v << 2)) & 0x09249249

    code = (spread(base[:, 0]) << 2) | (spread(base[:, 1]) << 1) | spread(base[:, 2])
    order = np.argsort(code, kind="stable")
    out = []
    for s in range(0, len(order), per):
        b = base[order[s:s + per]]
        out.append(int(np.prod(b.max(0) - b.min(0) + 3)))
    return out


def test_sparse_cloud_scatters_without_the_tile():
    """A thin cloud of three materials over a 20^3-cell region of a 32^3 grid
    (about 0.2 particles per cell): every CTA's particle range spans more
    nodes than the 1280-node scatter tile, so P2G and the G2P adjoint take the
    untiled path (one global float4 reduction per particle and node)."""
    sc = scenes.small_block(31, 32, [0, 1, 2], ppc=1, size_cells=20, lo_cell=(6, 6, 6), n_steps=16,
                            v0=(0.1, -0.2, 0.05), dt=2e-4, yield_stress=5.0, E=2e4)
    keep = np.random.Generator(np.random.PCG64(31)).random(sc.n_particles) < 0.2
    sc.x, sc.v, sc.mat = sc.x[keep], sc.v[keep], sc.mat[keep]
    sc.scene_counts = [int(keep.sum())]
    assert min(_tile_nodes_per_range(sc.x, sc.grid_n, 128)) > 1280
    sim = _sim(sc, checkpoint_every=8)
    sim.step(sc.n_steps)
    x, v = sim.state()
    xo, vo, _, _ = oracle_forward(sc)
    assert rel(x.cpu(), xo) < TOL_X
    assert rel(v.cpu(), vo) < TOL_X
    sim.position_loss(sc.loss["target"], 1.0, scene=0)
    gx, gv, _ = sim.backward()
    ref = oracle_grad(sc)
    assert rel(gx.cpu(), ref["x0"]) < TOL_G
    assert rel(gv.cpu(), ref["v0"]) < TOL_G
