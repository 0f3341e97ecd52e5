"""The no-allocation grid-mass loss entry point against the handle-based one.

sim_grid_mass_loss_static exists for callers that cannot call cudaMalloc (an
application that owns all device memory through its own pool, a real-time loop
that must not enter the allocator, a process under a hard memory cap). Its
results must match sim_grid_mass_loss, which works through a simulation
handle: the loss value directly, and the particle gradient through the same
reverse sweep of the trajectory. It is called twice in a row because every
call reuses one static device array that keeps the previous call's contents,
and then once more on a smaller grid (32^3), whose call clears and reads only
the first 32^3 entries of each field while the 64^3 call's values stay behind
the rest.
This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import scenes
from gpu_util import rel

pytestmark = pytest.mark.gpu

TOL_X = 1e-4
TOL_G = 1e-3


def test_static_grid_mass_loss_matches_handle_entry_point():
    from paper_2303_02346_gb300 import binding as B
    from paper_2303_02346_gb300.simulator import Simulator

    sc = scenes.multi_material(scale=0.02, grid_n=64, n_steps=20, checkpoint_every=10)
    L = sc.loss
    dev = torch.device("cuda", 0)
    sim = Simulator(sc)
    sim.reset()
    sim.step(sc.n_steps)
    x_T, _ = sim.state()
    loss_handle = sim.grid_mass_loss(L["target_mass"], L["target_dist"], L["total_mass"])
    gx_h, _, ga_h = sim.backward()

    tm = torch.tensor(L["target_mass"], dtype=torch.float32, device=dev)
    td = torch.tensor(L["target_dist"], dtype=torch.float32, device=dev)
    mass = torch.tensor(sc.particle_mass(), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    results = []
    for _ in range(2):
        dLdx = torch.full_like(x_T, float("nan"))
        loss = torch.zeros(1, dtype=torch.float64, device=dev)
        B.sim_grid_mass_loss_static(x_T.contiguous(), mass, sc.grid_n, tm, td, L["total_mass"], dLdx,
                                    loss, stream=stream)
        torch.cuda.synchronize()
        results.append((float(loss.item()), dLdx.clone()))
    for loss_s, dLdx in results:
        assert torch.isfinite(dLdx).all()
        assert abs(loss_s - loss_handle) / abs(loss_handle) < TOL_X
    assert rel(results[1][1].cpu(), results[0][1].cpu()) < 1e-6

    # right after the 64^3 calls: a 32^3 grid against a 32^3 handle
    sc32 = scenes.multi_material(scale=0.01, grid_n=32, n_steps=10, checkpoint_every=5)
    L32 = sc32.loss
    sim32 = Simulator(sc32)
    sim32.reset()
    sim32.step(sc32.n_steps)
    x32, _ = sim32.state()
    loss32_handle = sim32.grid_mass_loss(L32["target_mass"], L32["target_dist"], L32["total_mass"])
    gx32_h, _, ga32_h = sim32.backward()
    dLdx32 = torch.full_like(x32, float("nan"))
    loss32 = torch.zeros(1, dtype=torch.float64, device=dev)
    B.sim_grid_mass_loss_static(x32.contiguous(),
                                torch.tensor(sc32.particle_mass(), dtype=torch.float32, device=dev), 32,
                                torch.tensor(L32["target_mass"], dtype=torch.float32, device=dev),
                                torch.tensor(L32["target_dist"], dtype=torch.float32, device=dev),
                                L32["total_mass"], dLdx32, loss32, stream=stream)
    torch.cuda.synchronize()
    assert torch.isfinite(dLdx32).all()
    assert abs(float(loss32.item()) - loss32_handle) / abs(loss32_handle) < TOL_X
    sim32.reset()
    sim32.step(sc32.n_steps)
    sim32.add_loss_grad(dLdx32.contiguous(), None)
    gx32_s, _, ga32_s = sim32.backward()
    assert rel(gx32_s.cpu(), gx32_h.cpu()) < TOL_G
    assert rel(ga32_s.cpu(), ga32_h.cpu()) < TOL_G
    sim32.close()

    # the particle gradient through the same reverse sweep as the handle path
    sim.reset()
    sim.step(sc.n_steps)
    sim.add_loss_grad(results[1][1].contiguous(), None)
    gx_s, _, ga_s = sim.backward()
    assert rel(gx_s.cpu(), gx_h.cpu()) < TOL_G
    assert rel(ga_s.cpu(), ga_h.cpu()) < TOL_G
    sim.close()


def test_static_grid_mass_loss_rejects_large_grid():
    from paper_2303_02346_gb300 import binding as B
    lib = B.load()
    one = ctypes.c_void_p(1)
    # grid_n above the static array's capacity is refused before any device work
    assert lib.sim_grid_mass_loss_static(one, one, 1, 128, one, one, 1.0, one, one, None) == 1
    assert lib.sim_grid_mass_loss_static(one, one, 1, 64, one, one, 0.0, one, one, None) == 1
