"""Seeded synthetic scene generators.

This module builds the inputs that every other part of the repository consumes:
particle positions, velocities and material ids, material constants, the tool's
initial pose and action sequence, and loss targets. It holds none of the
simulation method's arithmetic (no B-spline weights, transfers, stresses or
contact): only random placement of particles in boxes, material constants as
given (Young's modulus, Poisson ratio, bulk modulus, density), seeded action
sequences, and simple geometric loss targets. Both the FP64 oracle and
the CUDA library read the same generated arrays; they share no other code.

The workloads stand in for the paper's task scale (a 64^3 MPM grid with about
100,000 particles, Sec. 4.2; a frame of 2e-3 s made of 10 substeps of 1e-4 s,
App. B.1) since the paper's task assets are not available. Every generator is
deterministic in its seed (numpy PCG64).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

LIQUID, VON_MISES, DRUCKER_PRAGER, BOX_YIELD, VISCOUS_LIQUID, RIGID = 0, 1, 2, 3, 4, 5
KIND_NAMES = {LIQUID: "liquid", VON_MISES: "von_mises", DRUCKER_PRAGER: "drucker_prager", BOX_YIELD: "box_yield",
              VISCOUS_LIQUID: "viscous_liquid", RIGID: "rigid"}


@dataclasses.dataclass
class Material:
    """Constants of one material. `volume` is the per-particle volume V_p."""
    kind: int
    rho: float
    volume: float
    E: float = 0.0
    nu: float = 0.0
    bulk: float = 0.0          # liquid bulk modulus K (lambda of a mu=0 corotated solid)
    yield_stress: float = 50.0  # von Mises yield stress tau_Y
    friction_deg: float = 30.0  # Drucker-Prager friction angle
    crit_compress: float = 2.5e-2  # box yield: singular values kept >= 1 - crit_compress
    crit_stretch: float = 7.5e-3   # box yield: singular values kept <= 1 + crit_stretch
    shear: float = 0.0             # viscous liquid: mu of the corotated model


@dataclasses.dataclass
class Scene:
    name: str
    grid_n: int
    dt: float
    n_steps: int
    materials: list
    x: np.ndarray            # (N, 3) float64, scenes concatenated
    v: np.ndarray            # (N, 3) float64
    mat: np.ndarray          # (N,) uint8 index into `materials`
    scene_counts: list       # particles per scene, in order
    gravity: tuple = (0.0, -9.8, 0.0)
    bound: int = 3
    checkpoint_every: int = 0
    substeps_per_action: int = 10
    # kinematic box tool (one per scene)
    tool_enabled: bool = False
    tool_half: tuple = (0.05, 0.01, 0.05)
    tool_pose0: Optional[np.ndarray] = None   # (S, 7): p (3), q (w, x, y, z)
    tool_actions: Optional[np.ndarray] = None  # (S, T_a, 6): pdot (3), omega (3)
    contact_eps: float = 0.0
    contact_soft: float = 0.0
    friction: float = 0.5
    # loss definition
    loss: dict = dataclasses.field(default_factory=dict)
    seed: int = 0

    @property
    def n_particles(self) -> int:
        return int(self.x.shape[0])

    @property
    def n_scenes(self) -> int:
        return len(self.scene_counts)

    @property
    def dx(self) -> float:
        return 1.0 / self.grid_n

    def particle_mass(self) -> np.ndarray:
        rho = np.array([m.rho for m in self.materials])
        vol = np.array([m.volume for m in self.materials])
        return rho[self.mat] * vol[self.mat]


# ----------------------------------------------------------------------------
# particle placement
# ----------------------------------------------------------------------------
def jittered_cells(rng, lo_cell, hi_cell, dx, ppc):
    """`ppc` uniform points inside every grid cell of the integer cell box
    [lo_cell, hi_cell) (stratified jitter)."""
    lo_cell = np.asarray(lo_cell)
    hi_cell = np.asarray(hi_cell)
    dims = hi_cell - lo_cell
    ii, jj, kk = np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")
    cells = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1) + lo_cell
    cells = np.repeat(cells, ppc, axis=0).astype(np.float64)
    return (cells + rng.random(cells.shape)) * dx


def uniform_box(rng, lo, hi, count):
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return lo + rng.random((count, 3)) * (hi - lo)


def smooth_actions(rng, n_actions, frame_dt, trans_amp, rot_amp, trans_bias=(0.0, 0.0, 0.0),
                   freq_range=(10.0, 40.0), n_terms=3):
    """Seeded smooth 6-DoF action sequence: each component is a sum of
    `n_terms` sinusoids with random amplitude, frequency and phase, sampled at
    the action times t_j = j * frame_dt."""
    t = np.arange(n_actions) * frame_dt
    out = np.zeros((n_actions, 6))
    for c in range(6):
        amp = trans_amp if c < 3 else rot_amp
        for _ in range(n_terms):
            a = amp * rng.uniform(0.3, 1.0) / n_terms
            f = rng.uniform(*freq_range)
            ph = rng.uniform(0.0, 2.0 * math.pi)
            out[:, c] += a * np.sin(2.0 * math.pi * f * t + ph)
    out[:, :3] += np.asarray(trans_bias)
    return out


def box_target(grid_n, center, half, total_mass):
    """Grid-mass loss target: total_mass spread uniformly over the grid nodes
    inside an axis-aligned box, and every node's Euclidean distance to that box
    (0 inside). Node i sits at i * dx. Arrays are flattened (i, j, k) row-major."""
    dx = 1.0 / grid_n
    g = np.arange(grid_n) * dx
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    P = np.stack([X, Y, Z], axis=-1).reshape(-1, 3)
    d = np.abs(P - np.asarray(center)) - np.asarray(half)
    inside = np.all(d <= 0.0, axis=1)
    dist = np.linalg.norm(np.maximum(d, 0.0), axis=1)
    m = np.zeros(P.shape[0])
    m[inside] = total_mass / max(int(inside.sum()), 1)
    return m, dist


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
WATER_BULK = 1.0e4
WATER_RHO = 1.0e3
SOLID_E = 5.0e3
SOLID_NU = 0.2


def water_material(volume):
    return Material(kind=LIQUID, rho=WATER_RHO, volume=volume, bulk=WATER_BULK)


def von_mises_material(volume, yield_stress=50.0):
    return Material(kind=VON_MISES, rho=WATER_RHO, volume=volume, E=SOLID_E, nu=SOLID_NU,
                    yield_stress=yield_stress)


def sand_material(volume, friction_deg=30.0):
    return Material(kind=DRUCKER_PRAGER, rho=WATER_RHO, volume=volume, E=SOLID_E, nu=SOLID_NU,
                    friction_deg=friction_deg)


def box_yield_material(volume, crit_compress=2.5e-2, crit_stretch=7.5e-3):
    return Material(kind=BOX_YIELD, rho=WATER_RHO, volume=volume, E=SOLID_E, nu=SOLID_NU,
                    crit_compress=crit_compress, crit_stretch=crit_stretch)


def viscous_material(volume, shear=1.0e3):
    return Material(kind=VISCOUS_LIQUID, rho=WATER_RHO, volume=volume, bulk=WATER_BULK, shear=shear)


def rigid_material(volume, rho=5.0 * WATER_RHO):
    """Particle-represented rigid object (its particles of one scene form one
    body); density 5x water as the transported object of the paper's material
    table."""
    return Material(kind=RIGID, rho=rho, volume=volume, E=SOLID_E, nu=SOLID_NU)


def water_cube(seed=1, n_steps=50, on_floor=False, v_down=0.0):
    """8,192 water particles, 16 jittered per cell in the 8^3 cells of the cube
    [0.375, 0.625]^3, on a 32^3 grid; dt = 2e-4; final-position loss.
    `on_floor` moves the cube down to rest on the sticky floor layer (cells
    3..10 in y) and `v_down` gives it a uniform initial downward speed, so that
    it is compressed against the wall from the first step."""
    n = 32
    dx = 1.0 / n
    rng = np.random.Generator(np.random.PCG64(seed))
    lo_y = 3 if on_floor else 12
    x = jittered_cells(rng, (12, lo_y, 12), (20, lo_y + 8, 20), dx, 16)
    N = x.shape[0]
    vol = 0.25 ** 3 / N
    v = np.zeros_like(x)
    v[:, 1] = -float(v_down)
    name = "water_cube_8k_32" + ("_floor" if on_floor else "")
    return Scene(name=name, grid_n=n, dt=2e-4, n_steps=n_steps,
                 materials=[water_material(vol)], x=x, v=v,
                 mat=np.zeros(N, np.uint8), scene_counts=[N],
                 loss={"kind": "position", "target": (0.5, 0.35, 0.5), "weight": 1.0},
                 seed=seed)


def _three_material_layout(rng, n, n_liq, n_ep, n_sand, ppc=8, origin=(0.0, 0.0, 0.0), span=1.0):
    """Liquid slab on the floor, an elastoplastic cube resting on its middle
    and a sand cube on the floor beside it. All particles have volume dx^3/ppc.
    `origin`/`span` place the layout in a sub-box of the unit domain."""
    dx = 1.0 / n
    vp = dx ** 3 / ppc
    o = np.asarray(origin, dtype=np.float64)
    floor_y = 0.03
    # liquid slab: fixed x/z extent, height from the count
    lx = 0.30 * span
    h_liq = n_liq * vp / (lx * lx) if n_liq else 0.0
    c = o + span * np.array([0.5, 0.0, 0.5])
    liq = uniform_box(rng, (c[0] - lx / 2, floor_y, c[2] - lx / 2),
                      (c[0] + lx / 2, floor_y + h_liq, c[2] + lx / 2), n_liq)
    a_ep = (n_ep * vp) ** (1.0 / 3.0) if n_ep else 0.0
    ep_lo = np.array([c[0] - a_ep / 2, floor_y + h_liq, c[2] - a_ep / 2])
    ep = uniform_box(rng, ep_lo, ep_lo + a_ep, n_ep)
    a_sd = (n_sand * vp) ** (1.0 / 3.0) if n_sand else 0.0
    sd_lo = np.array([o[0] + 0.15 * span, floor_y, o[2] + 0.15 * span])
    sd = uniform_box(rng, sd_lo, sd_lo + a_sd, n_sand)
    x = np.concatenate([liq, ep, sd], axis=0)
    mat = np.concatenate([np.full(n_liq, 0), np.full(n_ep, 1), np.full(n_sand, 2)]).astype(np.uint8)
    top = floor_y + h_liq + a_ep
    return x, mat, vp, top, c


def multi_material(seed=2, scale=1.0, n_steps=200, grid_n=128, checkpoint_every=20):
    """Liquid / von Mises / Drucker-Prager split 50/30/20 of 200k*scale
    particles on a grid_n^3 grid, a kinematic box tool pressing on the top of
    the elastoplastic cube with a seeded smooth 6-DoF trajectory, and a
    grid-mass (Chamfer-style) loss on the final state."""
    n = grid_n
    total = int(round(200_000 * scale))
    n_liq, n_ep = total // 2, (3 * total) // 10
    n_sand = total - n_liq - n_ep
    rng = np.random.Generator(np.random.PCG64(seed))
    x, mat, vp, top, c = _three_material_layout(rng, n, n_liq, n_ep, n_sand)
    N = x.shape[0]
    mats = [water_material(vp), von_mises_material(vp), sand_material(vp)]
    dt = 1e-4
    spa = 10
    n_actions = (n_steps + spa - 1) // spa
    half = (0.05, 0.01, 0.05)
    pose0 = np.array([[c[0], top + half[1] + 0.25 / n, c[2], 1.0, 0.0, 0.0, 0.0]])
    actions = smooth_actions(rng, n_actions, spa * dt, trans_amp=0.6, rot_amp=3.0,
                             trans_bias=(0.0, -0.8, 0.0))[None]
    mass_total = float(np.sum(np.array([m.rho * m.volume for m in mats])[mat]))
    tgt_m, tgt_d = box_target(n, center=(c[0] + 0.04, 0.08, c[2] - 0.02), half=(0.12, 0.05, 0.12),
                              total_mass=mass_total)
    return Scene(name=f"multi_material_{N // 1000}k_{n}", grid_n=n, dt=dt, n_steps=n_steps,
                 materials=mats, x=x, v=np.zeros_like(x), mat=mat, scene_counts=[N],
                 checkpoint_every=checkpoint_every, substeps_per_action=spa,
                 tool_enabled=True, tool_half=half, tool_pose0=pose0, tool_actions=actions,
                 contact_eps=2.0 / n, contact_soft=1.0 / n, friction=0.5,
                 loss={"kind": "grid_mass", "target_mass": tgt_m, "target_dist": tgt_d,
                       "total_mass": mass_total},
                 seed=seed)


def batched_scenes(seed=3, n_scenes=64, grid_n=64, n_steps=100, lo=10_000, hi=150_000):
    """`n_scenes` independent scenes on grid_n^3 grids; particle counts drawn
    log-uniform in [lo, hi]; material fractions ~ Dirichlet(5, 3, 2); each a
    three-material layout with its own seeded tool trajectory; final-position
    loss per scene."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = grid_n
    counts = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), n_scenes))).astype(int)
    xs, mats_, poses, acts = [], [], [], []
    vp = None
    spa = 10
    dt = 1e-4
    n_actions = (n_steps + spa - 1) // spa
    for s in range(n_scenes):
        frac = rng.dirichlet((5.0, 3.0, 2.0))
        nl = int(counts[s] * frac[0])
        ne = int(counts[s] * frac[1])
        nd = int(counts[s]) - nl - ne
        x, mat, vp, top, c = _three_material_layout(rng, n, nl, ne, nd)
        xs.append(x)
        mats_.append(mat)
        poses.append([c[0], top + 0.01 + 0.25 / n, c[2], 1.0, 0.0, 0.0, 0.0])
        acts.append(smooth_actions(rng, n_actions, spa * dt, trans_amp=0.6, rot_amp=3.0,
                                   trans_bias=(0.0, -0.8, 0.0)))
    x = np.concatenate(xs)
    mat = np.concatenate(mats_)
    mats = [water_material(vp), von_mises_material(vp), sand_material(vp)]
    return Scene(name=f"batched_{n_scenes}x{n}", grid_n=n, dt=dt, n_steps=n_steps,
                 materials=mats, x=x, v=np.zeros_like(x), mat=mat,
                 scene_counts=[int(a.shape[0]) for a in xs], checkpoint_every=n_steps,
                 substeps_per_action=spa, tool_enabled=True, tool_half=(0.05, 0.01, 0.05),
                 tool_pose0=np.array(poses), tool_actions=np.array(acts),
                 contact_eps=2.0 / n, contact_soft=1.0 / n, friction=0.5,
                 loss={"kind": "position", "target": (0.5, 0.2, 0.5), "weight": 1.0},
                 seed=seed)


def dam_break(seed=4, scale=1.0, grid_n=256, n_steps=1000, checkpoint_every=50):
    """2M*scale particles, 70% water in a dam-break column against the -x wall
    and 30% von Mises blocks on the floor downstream; final-position loss."""
    n = grid_n
    rng = np.random.Generator(np.random.PCG64(seed))
    total = int(round(2_000_000 * scale))
    n_liq = (7 * total) // 10
    n_ep = total - n_liq
    dx = 1.0 / n
    vp = dx ** 3 / 8
    lo = 4.0 * dx
    depth = 1.0 - 8.0 * dx          # z extent of the column
    width = 0.25                     # x extent of the column
    h = n_liq * vp / (width * depth)
    liq = uniform_box(rng, (lo, lo, lo), (lo + width, lo + h, lo + depth), n_liq)
    per = n_ep // 4
    blocks = []
    a = (per * vp) ** (1.0 / 3.0)
    for b in range(4):
        zc = lo + (b + 0.5) * depth / 4
        cnt = per if b < 3 else n_ep - 3 * per
        blocks.append(uniform_box(rng, (0.62, lo, zc - a / 2), (0.62 + a, lo + a, zc + a / 2), cnt))
    x = np.concatenate([liq] + blocks)
    mat = np.concatenate([np.zeros(n_liq), np.ones(n_ep)]).astype(np.uint8)
    mats = [water_material(vp), von_mises_material(vp)]
    return Scene(name=f"dam_break_{x.shape[0] // 1000}k_{n}", grid_n=n, dt=1e-4, n_steps=n_steps,
                 materials=mats, x=x, v=np.zeros_like(x), mat=mat, scene_counts=[x.shape[0]],
                 checkpoint_every=checkpoint_every,
                 loss={"kind": "position", "target": (0.5, 0.1, 0.5), "weight": 1.0}, seed=seed)


def small_block(seed, grid_n, kinds, ppc=2, lo_cell=None, size_cells=4, v0=(0.0, 0.0, 0.0),
                spin=0.0, n_steps=10, dt=None, gravity=(0.0, -9.8, 0.0), bound=3, tool=False,
                yield_stress=50.0, friction_deg=30.0, bulk=WATER_BULK, E=SOLID_E):
    """Small test scene: a block of `size_cells`^3 cells of jittered particles,
    split along x into one slab per entry of `kinds`. Optional uniform velocity
    v0, rigid spin about the block's y axis, and a box tool above the block."""
    n = grid_n
    dx = 1.0 / n
    rng = np.random.Generator(np.random.PCG64(seed))
    if lo_cell is None:
        lo_cell = ((n - size_cells) // 2,) * 3
    lo_cell = np.asarray(lo_cell)
    x = jittered_cells(rng, lo_cell, lo_cell + size_cells, dx, ppc)
    N = x.shape[0]
    vp = dx ** 3 / ppc
    mats = []
    for k in kinds:
        if k == LIQUID:
            m = water_material(vp)
            m.bulk = bulk
        elif k == VON_MISES:
            m = von_mises_material(vp, yield_stress)
            m.E = E
        elif k == BOX_YIELD:
            m = box_yield_material(vp)
            m.E = E
        elif k == VISCOUS_LIQUID:
            m = viscous_material(vp)
            m.bulk = bulk
        elif k == RIGID:
            m = rigid_material(vp)
        else:
            m = sand_material(vp, friction_deg)
            m.E = E
        mats.append(m)
    # slab index from x position
    rel = (x[:, 0] / dx - lo_cell[0]) / size_cells
    mat = np.minimum((rel * len(kinds)).astype(int), len(kinds) - 1).astype(np.uint8)
    center = (lo_cell + size_cells / 2.0) * dx
    v = np.tile(np.asarray(v0, dtype=np.float64), (N, 1))
    if spin != 0.0:
        r = x - center
        v += spin * np.stack([r[:, 2], np.zeros(N), -r[:, 0]], axis=1)
    if dt is None:
        dt = 2e-4 * 32.0 / n
    sc = Scene(name=f"block_{n}_{N}", grid_n=n, dt=dt, n_steps=n_steps, materials=mats, x=x,
               v=v, mat=mat, scene_counts=[N], gravity=tuple(gravity), bound=bound,
               loss={"kind": "position", "target": tuple(center - np.array([0.0, 2 * dx, 0.0])),
                     "weight": 1.0}, seed=seed)
    if tool:
        top = (lo_cell[1] + size_cells) * dx
        sc.tool_enabled = True
        sc.tool_half = (size_cells * dx * 0.4, 0.5 * dx, size_cells * dx * 0.4)
        sc.tool_pose0 = np.array([[center[0] + 0.3 * dx, top + 0.2 * dx, center[2] - 0.2 * dx,
                                   math.cos(0.1), 0.0, math.sin(0.1), 0.0]])
        n_act = (n_steps + sc.substeps_per_action - 1) // sc.substeps_per_action
        sc.tool_actions = smooth_actions(rng, n_act, sc.substeps_per_action * dt,
                                         trans_amp=0.5, rot_amp=4.0,
                                         trans_bias=(0.1, -1.0, 0.0))[None]
        sc.contact_eps = 2.0 * dx
        sc.contact_soft = dx
        sc.friction = 0.5
    return sc


def merge_scenes(scenes):
    """Concatenate independent single-scene inputs (same grid, dt, materials
    and tool geometry) into one batched scene."""
    s0 = scenes[0]
    out = dataclasses.replace(
        s0, name=f"batch_of_{len(scenes)}",
        x=np.concatenate([s.x for s in scenes]), v=np.concatenate([s.v for s in scenes]),
        mat=np.concatenate([s.mat for s in scenes]),
        scene_counts=[c for s in scenes for c in s.scene_counts])
    if s0.tool_enabled:
        out.tool_pose0 = np.concatenate([s.tool_pose0 for s in scenes])
        out.tool_actions = np.concatenate([s.tool_actions for s in scenes])
    return out
