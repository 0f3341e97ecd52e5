"""Scene-level wrapper over the C-ABI and the torch.autograd.Function that puts
the library's forward and hand-written adjoint behind PyTorch autograd.

Argument marshalling only: every computation is a call into the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def materials_of(scene):
    return [dict(kind=m.kind, rho=m.rho, volume=m.volume, E=m.E, nu=m.nu, bulk=m.bulk,
                 yield_stress=m.yield_stress, friction_deg=m.friction_deg,
                 crit_compress=getattr(m, "crit_compress", 0.0), crit_stretch=getattr(m, "crit_stretch", 0.0),
                 shear=getattr(m, "shear", 0.0))
            for m in scene.materials]


class Simulator:
    """One library handle configured from a `scenes.Scene`.

    checkpoint_every: 0 = forward only; k > 0 keeps a checkpoint every k steps
    for `backward` (default: the scene's own value, else the whole horizon).
    """

    def __init__(self, scene, checkpoint_every=None, max_steps=None, stream=None, resort_every=0,
                 device="cuda", graphs=True):
        self.scene = scene
        self.device = torch.device(device)
        T = int(max_steps if max_steps is not None else scene.n_steps)
        k = scene.checkpoint_every or T if checkpoint_every is None else int(checkpoint_every)
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.cfg = B.make_config(
            grid_n=scene.grid_n, dt=scene.dt, materials=materials_of(scene),
            scene_counts=scene.scene_counts, gravity=scene.gravity, bound=scene.bound,
            substeps_per_action=scene.substeps_per_action, checkpoint_every=k, max_steps=T,
            tool_enabled=scene.tool_enabled, tool_half=scene.tool_half,
            contact_eps=scene.contact_eps, contact_soft=scene.contact_soft,
            friction=scene.friction, cuda_stream=stream, resort_every=resort_every,
            no_graphs=not graphs)
        self.k = k
        self.max_steps = T
        self.N = int(scene.n_particles)
        self.S = int(scene.n_scenes)
        self.h = B.sim_create(self.cfg)

    # -- inputs -------------------------------------------------------------
    def set_particles(self, x=None, v=None, mat=None, scene=-1):
        sc = self.scene
        if x is None:
            x = torch.tensor(sc.x, dtype=torch.float32, device=self.device)
        if v is None:
            v = torch.tensor(sc.v, dtype=torch.float32, device=self.device)
        if mat is None:
            mat = torch.tensor(sc.mat, dtype=torch.uint8, device=self.device)
        B.sim_set_particles(self.h, scene, x.contiguous(), v.contiguous(), mat.contiguous())

    def set_tool(self, pose0=None, actions=None, scene=-1):
        sc = self.scene
        if pose0 is None:
            pose0 = torch.tensor(sc.tool_pose0, dtype=torch.float32, device=self.device)
        if actions is None:
            actions = torch.tensor(sc.tool_actions, dtype=torch.float32, device=self.device)
        # actions beyond the configured horizon never act: pass only those that can
        n_max = -(-self.max_steps // max(int(sc.substeps_per_action), 1))
        if actions.shape[-2] > n_max:
            actions = actions[..., :n_max, :]
        n_act = actions.shape[-2]
        B.sim_set_tool(self.h, scene, pose0.contiguous(), actions.contiguous(), n_act)

    def reset(self):
        self.set_particles()
        if self.scene.tool_enabled:
            self.set_tool()

    # -- stepping and state -------------------------------------------------
    def step(self, n):
        B.sim_step(self.h, n)

    @property
    def current_step(self):
        return B.sim_current_step(self.h)

    def state(self, scene=-1, with_CF=False, step=-1):
        cnt = self.N if scene < 0 else int(self.scene.scene_counts[scene])
        x = torch.empty(cnt, 3, dtype=torch.float32, device=self.device)
        v = torch.empty(cnt, 3, dtype=torch.float32, device=self.device)
        C = F = None
        if with_CF:
            C = torch.empty(cnt, 3, 3, dtype=torch.float32, device=self.device)
            F = torch.empty(cnt, 3, 3, dtype=torch.float32, device=self.device)
        B.sim_get_state(self.h, scene, step, x, v, C, F)
        return (x, v, C, F) if with_CF else (x, v)

    # -- losses and gradients -----------------------------------------------
    def position_loss(self, target, weight=1.0, scene=-1, step=-1):
        return B.sim_position_loss(self.h, scene, target, weight, n_out=self.S if scene < 0 else 1, step=step)

    def attraction_loss(self, ell, radius, tau, weight=1.0, scene=-1):
        """Attraction loss of Sec. 5.1 on the current positions (ell: the
        particles' previous losses, caller order); seeds its gradient."""
        e = torch.as_tensor(np.asarray(ell) if not isinstance(ell, torch.Tensor) else ell,
                            dtype=torch.float32, device=self.device).contiguous()
        return B.sim_attraction_loss(self.h, scene, e, radius, tau, weight)

    def share_gradients(self, ell, g, radius, tau, scene=-1):
        """Gradient sharing of Sec. 5.1: returns sum_j c_j k(d_aj / h) g_j per
        particle (caller order) on the current positions."""
        dev = self.device
        e = torch.as_tensor(ell, dtype=torch.float32, device=dev).contiguous()
        gg = torch.as_tensor(g, dtype=torch.float32, device=dev).reshape(-1, 3).contiguous()
        out = torch.empty_like(gg)
        B.sim_share_gradients(self.h, scene, e, radius, tau, gg, out)
        return out

    def grid_mass_loss(self, target_mass, target_dist, total_mass, scene=0, step=-1):
        tm = torch.as_tensor(np.asarray(target_mass), dtype=torch.float32, device=self.device).contiguous()
        td = torch.as_tensor(np.asarray(target_dist), dtype=torch.float32, device=self.device).contiguous()
        return B.sim_grid_mass_loss(self.h, scene, tm, td, total_mass, step=step)

    def add_loss_grad(self, dLdx=None, dLdv=None, scene=-1, step=-1):
        B.sim_add_loss_grad(self.h, scene, dLdx, dLdv, step=step)

    def tool_pose(self, step, scene=-1):
        """(S or 1, 13) tool pose at the start of `step`: position, quaternion
        (w, x, y, z), linear and angular velocity."""
        out = torch.empty(self.S if scene < 0 else 1, 13, dtype=torch.float32, device=self.device)
        B.sim_get_tool_pose(self.h, scene, step, out)
        return out

    def backward(self, want_actions=True):
        gx = torch.empty(self.N, 3, dtype=torch.float32, device=self.device)
        gv = torch.empty(self.N, 3, dtype=torch.float32, device=self.device)
        ga = None
        if want_actions and self.scene.tool_enabled:
            n_max = -(-self.max_steps // max(int(self.scene.substeps_per_action), 1))
            n_act = min(self.scene.tool_actions.shape[-2], n_max)
            ga = torch.empty(self.S, n_act, 6, dtype=torch.float32, device=self.device)
        B.sim_backward(self.h, gx, gv, ga)
        return gx, gv, ga

    def profile(self, enable=True):
        B.sim_profile_enable(self.h, enable)

    def profile_read(self):
        return B.sim_profile_read(self.h)

    def close(self):
        if self.h is not None:
            B.sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MPMRollout(torch.autograd.Function):
    """(x0, v0, actions) -> (x_T, v_T) through `n_steps` library steps.

    Forward calls sim_set_particles / sim_set_tool / sim_step; backward seeds the
    library with dL/dx_T, dL/dv_T (sim_add_loss_grad) and runs sim_backward, the
    hand-written adjoint with checkpoint + recompute (paper App. A)."""

    @staticmethod
    def forward(ctx, sim, n_steps, x0, v0, actions):
        sim.set_particles(x0.detach().float().contiguous(), v0.detach().float().contiguous())
        if sim.scene.tool_enabled:
            a = actions.detach().float().contiguous()
            sim.set_tool(actions=a)
        sim.step(n_steps)
        x, v = sim.state()
        ctx.sim = sim
        ctx.has_tool = sim.scene.tool_enabled
        ctx.act_shape = actions.shape
        return x, v

    @staticmethod
    def backward(ctx, gx, gv):
        sim = ctx.sim
        gx = torch.zeros(sim.N, 3, device=sim.device) if gx is None else gx.float().contiguous()
        gv = torch.zeros(sim.N, 3, device=sim.device) if gv is None else gv.float().contiguous()
        sim.add_loss_grad(gx, gv)
        dx0, dv0, da = sim.backward(want_actions=ctx.has_tool)
        if da is not None and tuple(da.shape) != tuple(ctx.act_shape):
            # actions past the horizon have zero gradient
            full = torch.zeros(ctx.act_shape, dtype=da.dtype, device=da.device)
            full[..., : da.shape[-2], :] = da
            da = full
        return None, None, dx0, dv0, da


def rollout(sim, n_steps, x0, v0, actions=None):
    if actions is None:
        actions = torch.zeros(1, device=sim.device)
    return MPMRollout.apply(sim, n_steps, x0, v0, actions)
