"""The seeded synthetic workloads match their stated recipe: particle counts
and material splits, placement inside the grid's interior, step sizes and
horizons, log-uniform batched counts with Dirichlet(5, 3, 2) material
fractions, and determinism under a fixed seed."""
import numpy as np

import scenes


def _inside(sc):
    """Every particle's stencil origin floor(x / dx - 0.5) lies in [0, n - 3]
    (the domain the simulator accepts)."""
    base = np.floor(sc.x * sc.grid_n - 0.5)
    return bool(((base >= 0) & (base <= sc.grid_n - 3)).all())


def _clear_of_walls(sc):
    lo = sc.bound / sc.grid_n
    return bool(((sc.x >= lo) & (sc.x < 1.0 - lo)).all())


def test_water_cube_recipe():
    sc = scenes.water_cube()
    assert sc.n_particles == 8192 and sc.grid_n == 32 and sc.dt == 2e-4 and sc.n_steps == 50
    assert (sc.x >= 0.375).all() and (sc.x < 0.625).all()
    cells = np.floor(sc.x * 32).astype(int)
    _, per_cell = np.unique(cells, axis=0, return_counts=True)
    assert len(per_cell) == 512 and (per_cell == 16).all()
    assert (sc.mat == 0).all() and not sc.v.any()
    fl = scenes.water_cube(on_floor=True, v_down=1.0)
    assert fl.n_particles == 8192 and _inside(fl)
    assert fl.x[:, 1].min() >= 3 / 32 and fl.x[:, 1].max() < 11 / 32
    assert (fl.v[:, 1] == -1.0).all() and not fl.v[:, [0, 2]].any()


def test_three_material_tool_scene_recipe():
    sc = scenes.multi_material()
    assert sc.n_particles == 200_000 and sc.grid_n == 128
    assert np.bincount(sc.mat).tolist() == [100_000, 60_000, 40_000]
    assert sc.dt == 1e-4 and sc.n_steps == 200 and sc.checkpoint_every == 20
    assert sc.tool_enabled and sc.tool_actions.shape == (1, 20, 6)
    assert _inside(sc) and _clear_of_walls(sc)
    liq = sc.x[sc.mat == 0]
    assert np.allclose(liq.min(0), [0.35, 0.03, 0.35], atol=2e-3)
    assert np.allclose(liq.max(0)[[0, 2]], [0.65, 0.65], atol=2e-3)
    # 8 particles per dx^3 of material volume
    dx = 1.0 / 128
    assert np.isclose(sc.materials[0].volume, dx ** 3 / 8)
    # the tool starts above the elastoplastic cube, a quarter cell clear of it
    top = sc.x[sc.mat == 1][:, 1].max()
    bottom_of_tool = sc.tool_pose0[0, 1] - sc.tool_half[1]
    assert 0.0 < bottom_of_tool - top < 0.5 * dx
    again = scenes.multi_material()
    assert np.array_equal(sc.x, again.x) and np.array_equal(sc.tool_actions, again.tool_actions)


def test_batched_scenes_recipe():
    sc = scenes.batched_scenes()
    counts = np.array(sc.scene_counts)
    assert len(counts) == 64 and sc.grid_n == 64 and sc.n_steps == 100
    assert (counts >= 10_000).all() and (counts <= 150_000).all()
    # log-uniform on [1e4, 1.5e5]: mean of the logs near the midpoint
    mid = 0.5 * (np.log(1e4) + np.log(1.5e5))
    assert abs(np.log(counts).mean() - mid) < 0.3
    assert 2.5e6 < counts.sum() < 4.0e6
    lo = np.concatenate([[0], np.cumsum(counts)[:-1]])
    fr = np.array([np.bincount(sc.mat[a:a + c], minlength=3) / c for a, c in zip(lo, counts)])
    assert np.allclose(fr.mean(0), [0.5, 0.3, 0.2], atol=0.06)
    assert sc.tool_pose0.shape == (64, 7) and sc.tool_actions.shape[0] == 64
    assert _inside(sc)
    # the layout's floor (y = 0.03) lies inside the 3-node wall layer of a 64^3
    # grid: each scene's lowest particles start on sticky wall nodes
    assert not _clear_of_walls(sc) and sc.x[:, 1].min() >= 0.03


def test_dam_break_recipe():
    sc = scenes.dam_break(scale=0.01)
    assert sc.n_particles == 20_000 and sc.grid_n == 256
    assert np.bincount(sc.mat).tolist() == [14_000, 6_000]
    assert sc.n_steps == 1000 and sc.checkpoint_every == 50
    assert _inside(sc) and _clear_of_walls(sc)
    # water in a column against the -x wall, blocks downstream
    assert sc.x[sc.mat == 0][:, 0].max() < 0.3 and sc.x[sc.mat == 1][:, 0].min() > 0.6
