"""Pins of the oracle's reverse mode (Sec. 3.3, App. A: gradients through the
whole simulation, the SVD gradient written by hand) against central finite
differences of the oracle's forward rollout, on tiny scenes away from branch
switches: directional derivatives <grad L, u> for random directions u."""
import numpy as np
import pytest
import torch

import scenes
from oracle import mpm

DT = torch.float64


def _directional_check(f, params, n_dirs=3, h=1e-6, seed=0, tol=2e-5):
    rng = np.random.default_rng(seed)
    ps = [p.detach().clone().requires_grad_(True) for p in params]
    L = f(*ps)
    grads = torch.autograd.grad(L, ps)
    for _ in range(n_dirs):
        us = [torch.tensor(rng.normal(size=p.shape), dtype=DT) for p in params]
        an = sum((g * u).sum() for g, u in zip(grads, us)).item()
        with torch.no_grad():
            lp = f(*[p + h * u for p, u in zip(params, us)]).item()
            lm = f(*[p - h * u for p, u in zip(params, us)]).item()
        fd = (lp - lm) / (2 * h)
        assert abs(an - fd) <= tol * max(abs(fd), 1e-8 * abs(L.item())), (an, fd)


@pytest.mark.parametrize("kinds", [[0], [1], [2], [3], [4], [0, 1, 2, 3, 4]])
def test_rollout_gradient_wrt_initial_state(kinds):
    sc = scenes.small_block(11, 12, kinds, ppc=2, size_cells=4, lo_cell=(4, 3, 4), n_steps=12,
                            v0=(0.2, -0.3, 0.1), spin=8.0, dt=2e-4, yield_stress=5.0, E=2e4)
    x0 = torch.tensor(sc.x, dtype=DT)
    v0 = torch.tensor(sc.v, dtype=DT)

    def f(x, v):
        xs, vs, C, F = mpm.rollout(sc, x0=x, v0=v)
        return mpm.scene_loss(sc, xs) + 0.1 * (vs ** 2).sum()

    _directional_check(f, [x0, v0], h=1e-7)


def test_rollout_gradient_wrt_tool_actions():
    sc = scenes.small_block(12, 16, [0, 1, 2], ppc=2, size_cells=6, lo_cell=(5, 3, 5), n_steps=30,
                            dt=2e-4, tool=True, yield_stress=20.0)
    acts = torch.tensor(sc.tool_actions[0], dtype=DT)

    def f(a):
        xs, vs, C, F = mpm.rollout(sc, actions=a)
        return mpm.scene_loss(sc, xs)

    # the tool must actually touch the material for this test to mean anything
    a = acts.clone().requires_grad_(True)
    g, = torch.autograd.grad(f(a), a)
    assert g.abs().max().item() > 0.0
    _directional_check(f, [acts], h=1e-6, tol=1e-4)


def test_grid_mass_loss_gradient():
    sc = scenes.multi_material(scale=0.002, grid_n=32, n_steps=5)
    model = mpm.Model(sc)
    mass, _ = model.particle_mass_volume(sc.mat)
    x0 = torch.tensor(sc.x, dtype=DT)
    L = sc.loss

    def f(x):
        return mpm.grid_mass_loss(x, mass, model, L["target_mass"], L["target_dist"], L["total_mass"])

    _directional_check(f, [x0], h=1e-7)


def test_grid_mass_loss_zero_at_target():
    """With the target equal to the particles' own mass field and d* = 0 the
    loss is exactly zero."""
    sc = scenes.multi_material(scale=0.002, grid_n=32, n_steps=5)
    model = mpm.Model(sc)
    mass, _ = model.particle_mass_volume(sc.mat)
    x = torch.tensor(sc.x, dtype=DT)
    W, _, lin = mpm.stencil(x, model)
    m = torch.zeros(model.n ** 3, dtype=DT).index_add(0, lin.reshape(-1), (W * mass[:, None]).reshape(-1))
    val = mpm.grid_mass_loss(x, mass, model, m, torch.zeros_like(m), float(mass.sum()))
    assert val.item() == 0.0


def test_checkpointed_rollout_gives_the_same_gradients():
    """The oracle's per-step recompute (activation checkpointing, used for long
    full-size horizons) returns the gradients of the plain rollout: the
    recomputed steps are the same FP64 operations."""
    sc = scenes.small_block(17, 16, [0, 1, 2], ppc=2, size_cells=5, lo_cell=(5, 3, 5), n_steps=12,
                            dt=2e-4, tool=True, yield_stress=20.0)
    out = []
    for ck in (False, True):
        x0 = torch.tensor(sc.x, dtype=DT, requires_grad=True)
        v0 = torch.tensor(sc.v, dtype=DT, requires_grad=True)
        act = torch.tensor(sc.tool_actions[0], dtype=DT, requires_grad=True)
        x, _, _, _ = mpm.rollout(sc, x0=x0, v0=v0, actions=act, checkpoint_steps=ck)
        L = mpm.scene_loss(sc, x)
        L.backward()
        out.append((L.item(), x0.grad, v0.grad, act.grad))
    (L0, gx0, gv0, ga0), (L1, gx1, gv1, ga1) = out
    assert L0 == L1
    assert torch.abs(ga0).max() > 0
    for a, b in ((gx0, gx1), (gv0, gv1), (ga0, ga1)):
        assert torch.allclose(a, b, rtol=1e-12, atol=1e-12 * a.abs().max())
