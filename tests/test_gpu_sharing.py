"""GPU parity of gradient sharing and the attraction loss (Sec. 5.1) against
the FP64 oracle, through the C-ABI: the loss and the shared gradients on the
library's own positions, and the attraction loss's gradient carried back to
the initial state by the adjoint against autograd through the oracle MPM."""
import numpy as np
import pytest
import torch

import scenes
from gpu_util import rel
from oracle import mpm as omp
from oracle import sharing as S

pytestmark = pytest.mark.gpu

DT = torch.float64
TAU = 0.5


def _scene(T=4):
    # two independent water blocks of 512 particles (8 per cell), 32^3 grid
    blocks = [scenes.small_block(seed=40 + i, grid_n=32, kinds=[0], ppc=8, size_cells=4,
                                 v0=(0.1 * i, -0.05, 0.0), spin=2.0, n_steps=T) for i in range(2)]
    return scenes.merge_scenes(blocks)


def _sim(sc, **kw):
    from paper_2303_02346_gb300.simulator import Simulator
    s = Simulator(sc, **kw)
    s.reset()
    return s


def _scene_ids(sc):
    return np.repeat(np.arange(len(sc.scene_counts)), sc.scene_counts)


def test_attraction_loss_and_shared_gradients_on_current_positions():
    sc = _scene()
    h = 0.8 / sc.grid_n
    sim = _sim(sc, checkpoint_every=2, max_steps=4)
    sim.step(4)
    x = sim.state()[0].cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(1)
    ell = rng.random(sc.n_particles).astype(np.float32)
    L = sim.attraction_loss(ell, h, TAU, weight=1.0)
    Lo = float(S.attraction_loss(x, _scene_ids(sc), ell.astype(np.float64), h, TAU))
    assert Lo > 0.0
    assert abs(L - Lo) / Lo < 1e-5
    g = rng.normal(size=(sc.n_particles, 3)).astype(np.float32)
    out = sim.share_gradients(ell, g, h, TAU)
    ref = S.share_gradients(x, _scene_ids(sc), ell.astype(np.float64), h, TAU, g.astype(np.float64)).numpy()
    assert rel(out.cpu(), ref) < 1e-5


def test_attraction_one_scene_addressed():
    sc = _scene()
    h = 1.0 / sc.grid_n
    sim = _sim(sc, checkpoint_every=2, max_steps=4)
    sim.step(4)
    x = sim.state(scene=1)[0].cpu().numpy().astype(np.float64)
    ell = np.linspace(0.0, 2.0, sc.scene_counts[1]).astype(np.float32)
    L = sim.attraction_loss(ell, h, TAU, scene=1)
    Lo = float(S.attraction_loss(x, np.zeros(len(x), int), ell.astype(np.float64), h, TAU))
    assert abs(L - Lo) / Lo < 1e-5
    g = np.ones((sc.scene_counts[1], 3), np.float32)
    out = sim.share_gradients(ell, g, h, TAU, scene=1)
    ref = S.share_gradients(x, np.zeros(len(x), int), ell.astype(np.float64), h, TAU, g.astype(np.float64))
    assert rel(out.cpu(), ref.numpy()) < 1e-5


def test_attraction_gradient_through_the_adjoint_matches_oracle():
    """L = w * L_att(x_T) + position loss; dL/dx0 and dL/dv0 through 4 steps
    (checkpoints every 2) against autograd through the oracle."""
    T = 4
    sc = _scene(T)
    h, w = 0.8 / sc.grid_n, 0.3
    ids = _scene_ids(sc)
    rng = np.random.default_rng(2)
    ell = rng.random(sc.n_particles)
    target = np.array(sc.loss["target"])
    sim = _sim(sc, checkpoint_every=2, max_steps=T)
    sim.step(T)
    L = sim.attraction_loss(ell.astype(np.float32), h, TAU, weight=w)
    sim.position_loss(target, 1.0)
    gx, gv, _ = sim.backward(want_actions=False)
    gx_ref, gv_ref, L_ref = [], [], 0.0
    for si in range(len(sc.scene_counts)):
        lo = int(sum(sc.scene_counts[:si]))
        hi = lo + int(sc.scene_counts[si])
        x0 = torch.tensor(sc.x[lo:hi], dtype=DT, requires_grad=True)
        v0 = torch.tensor(sc.v[lo:hi], dtype=DT, requires_grad=True)
        x, v, C, F = omp.rollout(sc, n_steps=T, x0=x0, v0=v0, scene_index=si)
        La = S.attraction_loss(x, ids[lo:hi], ell[lo:hi], h, TAU)
        Lp = ((x - torch.tensor(target, dtype=DT)) ** 2).sum()
        (w * La + Lp).backward()
        gx_ref.append(x0.grad.numpy())
        gv_ref.append(v0.grad.numpy())
        L_ref += float(w * La.detach())
    assert abs(L - L_ref) / L_ref < 1e-4
    assert rel(gx.cpu(), np.concatenate(gx_ref)) < 1e-3
    assert rel(gv.cpu(), np.concatenate(gv_ref)) < 1e-3


def test_sharing_rejects_bad_arguments():
    from paper_2303_02346_gb300.binding import SimError
    sc = _scene()
    sim = _sim(sc, checkpoint_every=2, max_steps=4)
    ell = np.zeros(sc.n_particles, np.float32)
    with pytest.raises(SimError):  # before any step
        sim.attraction_loss(ell, 0.5 / sc.grid_n, TAU)
    sim.step(2)
    for radius, tau in [(2.0 / sc.grid_n, TAU), (0.0, TAU), (0.5 / sc.grid_n, 0.0)]:
        with pytest.raises(SimError):
            sim.attraction_loss(ell, radius, tau)
    with pytest.raises(SimError):
        sim.attraction_loss(ell, 0.5 / sc.grid_n, TAU, scene=7)
