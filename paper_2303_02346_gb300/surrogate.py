"""Learned grid-space surrogate of the MLS-MPM step (include/mpm_surrogate.h):
handle wrapper, frame generation from the simulator's own rollouts, training
loop and the error-gated predictor that falls back to the full simulation.

Argument marshalling and orchestration only: features, network, loss,
gradients and Adam all run in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B
from .simulator import Simulator

FRAME_CHANNELS = 8


def frame_scales(scene):
    """(m_ref, v_ref): the mass of a grid cell filled at the first material's
    density, and 0.1 m/s (the order of the tool and free-fall speeds over a
    rollout of 10^2 steps of 10^-4 s)."""
    dx = 1.0 / scene.grid_n
    return float(scene.materials[0].rho * dx ** 3), 0.1


def particle_masses(scene):
    return [float(m.rho * m.volume) for m in scene.materials]


def param_count(channels=32, blocks=4, cin=FRAME_CHANNELS):
    c = channels
    return c * cin + c + blocks * 2 * (27 * c * c + c) + 3 * c + 3


def init_params(seed, blocks=4, channels=32, cin=FRAME_CHANNELS):
    """Initial flat parameter vector (layout of include/mpm_surrogate.h):
    He-normal lift and first convolutions; second convolutions and projection
    scaled by 0.1 so that each residual block and the network start near the
    identity (pred = input momentum); zero biases."""
    rng = np.random.default_rng(seed)
    c = channels
    parts = [rng.normal(0.0, np.sqrt(2.0 / cin), (c, cin)), np.zeros(c)]
    for _ in range(blocks):
        parts += [rng.normal(0.0, np.sqrt(2.0 / (27 * c)), (27, c, c)), np.zeros(c),
                  rng.normal(0.0, 0.1 * np.sqrt(2.0 / (27 * c)), (27, c, c)), np.zeros(c)]
    parts += [rng.normal(0.0, 0.1 * np.sqrt(1.0 / c), (3, c)), np.zeros(3)]
    return np.concatenate([np.ravel(a) for a in parts]).astype(np.float32)


class Surrogate:
    """One surrogate handle: parameters, Adam state and activations for up to
    `max_batch` frames of an n^3 grid."""

    def __init__(self, grid_n, m_ref, v_ref, max_batch=8, blocks=4, channels=32, device="cuda", stream=None):
        self.device = torch.device(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.cfg = B.make_sur_config(grid_n=grid_n, channels=channels, blocks=blocks, max_batch=max_batch,
                                     m_ref=m_ref, v_ref=v_ref, cuda_stream=stream)
        self.n = int(grid_n)
        self.n3 = self.n ** 3
        self.blocks = int(blocks)
        self.max_batch = int(max_batch)
        self.m_ref, self.v_ref = float(m_ref), float(v_ref)
        self.n_params = B.sur_param_count(self.cfg)
        self.h = B.sur_create(self.cfg)

    # -- parameters ------------------------------------------------------------
    def set_params(self, flat):
        t = torch.as_tensor(np.asarray(flat), dtype=torch.float32).contiguous()
        if t.numel() != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {t.numel()}")
        B.sur_set_params(self.h, t.to(self.device))

    def get_params(self):
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        B.sur_get_params(self.h, out)
        return out

    # -- frames ----------------------------------------------------------------
    def empty_frames(self, count):
        return torch.zeros(int(count), self.n3, FRAME_CHANNELS, dtype=torch.int16, device=self.device)

    def features(self, x, v, C, mat, material_mass, out):
        """One frame from a particle state (all device tensors); `out` is an
        (n^3, 8) int16 view that receives the BF16 bit patterns."""
        B.sur_features(self.h, x.contiguous(), v.contiguous(), C.contiguous(), mat.contiguous(),
                       material_mass, out)

    def features_vjp(self, x, v, C, mat, material_mass, g_frame):
        """(dL/dx, dL/dv, dL/dC) of the mass and momentum channels of the
        features for a cotangent g_frame (n^3, 8)."""
        n = x.shape[0]
        out = [torch.empty(n, k, dtype=torch.float32, device=self.device) for k in (3, 3, 9)]
        B.sur_features_vjp(self.h, x.contiguous(), v.contiguous() if v is not None else None,
                           C.reshape(n, 9).contiguous() if C is not None else None, mat.contiguous(),
                           material_mass, g_frame.contiguous(), *out)
        return out[0], out[1], out[2].reshape(n, 3, 3)

    def vjp(self, frames, idx, g_pred):
        """(d pred / d frame)^T g_pred for frames[idx], g_pred (batch, n^3, 3)."""
        batch = int(idx.numel())
        gf = torch.empty(batch, self.n3, FRAME_CHANNELS, dtype=torch.float32, device=self.device)
        B.sur_vjp(self.h, batch, frames, idx, g_pred.contiguous(), gf)
        return gf

    # -- network ---------------------------------------------------------------
    def predict(self, frames, idx=None, out=None):
        """Predicted normalised momentum (batch, n^3, 3) of frames[idx] (all
        frames when idx is None), max_batch frames per library call."""
        if idx is None:
            idx = torch.arange(frames.shape[0], dtype=torch.int32, device=self.device)
        batch = int(idx.numel())
        if out is None:
            out = torch.empty(batch, self.n3, 3, dtype=torch.float32, device=self.device)
        for k in range(0, batch, self.max_batch):
            i = idx[k:k + self.max_batch].contiguous()
            B.sur_predict(self.h, int(i.numel()), frames, i, out[k:k + i.numel()])
        return out

    def loss_grad(self, frames, idx, tgt, want_frame_grad=False):
        batch = int(idx.numel())
        grad = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        gf = (torch.empty(batch, self.n3, FRAME_CHANNELS, dtype=torch.float32, device=self.device)
              if want_frame_grad else None)
        loss = B.sur_loss_grad(self.h, batch, frames, idx, tgt, grad, gf)
        return loss, grad, gf

    def train_step(self, frames, idx, tgt, lr):
        return B.sur_train_step(self.h, int(idx.numel()), frames, idx, tgt, lr)

    def eval(self, frames, idx, tgt):
        """Relative L2 error of the predicted momentum per frame."""
        s = B.sur_eval(self.h, int(idx.numel()), frames, idx, tgt)
        return np.sqrt(s[:, 0] / np.maximum(s[:, 1], 1e-300))

    def profile(self, enable=True):
        B.sur_profile_enable(self.h, enable)

    def profile_read(self):
        return B.sur_profile_read(self.h)

    def close(self):
        if self.h is not None:
            B.sur_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def frames_of_state(sur, sim, scene, out, step_index=None):
    """Write the current frame of every scene of `sim` into out[s] (out: (S, n^3, 8))."""
    mm = particle_masses(scene)
    offs = np.concatenate([[0], np.cumsum(scene.scene_counts)])
    mat_all = torch.as_tensor(np.asarray(scene.mat), dtype=torch.uint8, device=sur.device)
    for s in range(scene.n_scenes):
        x, v, C, _ = sim.state(scene=s, with_CF=True)
        sur.features(x, v, C, mat_all[offs[s]:offs[s + 1]], mm, out[s])


def generate_frames(sur, scene, n_steps, horizon=10, out=None, first=0, timer=None):
    """Roll the (batched) scene forward n_steps with the simulator and keep the
    frame of every scene at every step 0..n_steps, in out[first + t * S + s]
    (a new tensor when out is None). Returns (frames, idx, tgt, scene_of_pair):
    training pairs are (frame of scene s at step t, frame at step t + horizon),
    as indices into `frames`. `timer` (a list) receives the milliseconds the
    simulation steps took, measured with CUDA events."""
    S = scene.n_scenes
    sim = Simulator(scene, checkpoint_every=0, max_steps=n_steps)
    sim.reset()
    if out is None:
        out = sur.empty_frames((n_steps + 1) * S)
        first = 0
    frames_of_state(sur, sim, scene, out[first:first + S])
    ev = []
    for t in range(1, n_steps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        sim.step(1)
        b.record()
        ev.append((a, b))
        frames_of_state(sur, sim, scene, out[first + t * S:first + (t + 1) * S])
    torch.cuda.synchronize()
    if timer is not None:
        timer.append(sum(a.elapsed_time(b) for a, b in ev))
    sim.close()
    t = np.arange(n_steps + 1 - horizon)
    s = np.arange(S)
    tt, ss = np.meshgrid(t, s, indexing="ij")
    idx = first + (tt * S + ss).ravel()
    tgt = first + ((tt + horizon) * S + ss).ravel()
    return out, idx.astype(np.int32), tgt.astype(np.int32), ss.ravel().astype(np.int32)


def train(sur, frames, idx, tgt, steps, batch, lr, seed=0, lr_final=None, log_every=0):
    """Adam on random minibatches of (idx, tgt) pairs, cosine learning-rate
    decay to lr_final. Returns the loss history."""
    rng = np.random.default_rng(seed)
    idx_d = torch.as_tensor(idx, dtype=torch.int32, device=sur.device)
    tgt_d = torch.as_tensor(tgt, dtype=torch.int32, device=sur.device)
    lr_final = lr * 0.05 if lr_final is None else lr_final
    hist = []
    for k in range(int(steps)):
        sel = torch.as_tensor(rng.choice(len(idx), size=batch, replace=False), dtype=torch.long,
                              device=sur.device)
        a = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * k / max(steps, 1)))
        loss = sur.train_step(frames, idx_d[sel].contiguous(), tgt_d[sel].contiguous(), a)
        hist.append(loss)
        if log_every and k % log_every == 0:
            print(f"step {k} loss {loss:.4e} lr {a:.2e}", flush=True)
    return np.asarray(hist)


def evaluate(sur, frames, idx, tgt, batch=None):
    """Relative L2 error per pair."""
    batch = batch or sur.max_batch
    out = []
    for k in range(0, len(idx), batch):
        i = torch.as_tensor(idx[k:k + batch], dtype=torch.int32, device=sur.device)
        t = torch.as_tensor(tgt[k:k + batch], dtype=torch.int32, device=sur.device)
        out.append(sur.eval(frames, i, t))
    return np.concatenate(out)


def cotangent_field(n, S, seed, kind, device):
    """(S, n^3, 8) seeded field on the momentum channels: "smooth" = a sum of 4
    plane waves per component with integer wave numbers in [-3, 3] (wavelength
    at least n / 3 nodes), "white" = independent normal values per node."""
    w = torch.zeros(S, n ** 3, FRAME_CHANNELS, dtype=torch.float32, device=device)
    if kind == "white":
        gen = torch.Generator(device=device).manual_seed(seed)
        w[..., 1:4] = torch.randn(S, n ** 3, 3, generator=gen, device=device)
        return w
    rng = np.random.default_rng(seed)
    ii = torch.arange(n, dtype=torch.float32, device=device)
    I, J, K = torch.meshgrid(ii, ii, ii, indexing="ij")
    for s in range(S):
        for c in range(3):
            acc = torch.zeros(n, n, n, dtype=torch.float32, device=device)
            for _ in range(4):
                f = rng.integers(-3, 4, size=3)
                while not f.any():
                    f = rng.integers(-3, 4, size=3)
                ph = rng.uniform(0, 2 * np.pi)
                acc += float(rng.normal()) * torch.cos(2 * np.pi * (f[0] * I + f[1] * J + f[2] * K) / n + ph)
            w[s, :, 1 + c] = acc.reshape(-1)
    return w


def compare_gradients(sur, scene, t, horizon=10, seed=0, field="smooth"):
    """Gradients of L = <w, momentum at t + horizon> (w a seeded field on the
    normalised momentum channels of the grid, `cotangent_field`) w.r.t. the particle
    velocities at step t, per scene, through the surrogate (features at t ->
    network -> adjoint) and through the simulation (restart from the state at
    t, `horizon` steps, adjoint seeded through the feature transfer at
    t + horizon). Also the same gradient for the no-change predictor (pred =
    input momentum). Returns per-scene relative L2 and cosine against the
    simulation."""
    S = scene.n_scenes
    dev = sur.device
    spa = int(scene.substeps_per_action)
    if t % spa:
        raise ValueError("t must start an action")
    mm = particle_masses(scene)
    offs = np.concatenate([[0], np.cumsum(scene.scene_counts)]).astype(int)
    mat_all = torch.as_tensor(np.asarray(scene.mat), dtype=torch.uint8, device=dev)
    # max_steps = t + 1 so that the library holds the tool pose of step t
    sim = Simulator(scene, checkpoint_every=0, max_steps=t + 1)
    sim.reset()
    if t:
        sim.step(t)
    x, v, C, F = sim.state(with_CF=True)
    pose = sim.tool_pose(t)[:, :7].contiguous() if scene.tool_enabled else None
    sim.close()
    sim2 = Simulator(scene, checkpoint_every=horizon, max_steps=horizon)
    B.sim_set_state(sim2.h, -1, x, v, C.reshape(-1, 9).contiguous(), F.reshape(-1, 9).contiguous(), mat_all)
    if scene.tool_enabled:
        a0 = t // spa
        acts = np.asarray(scene.tool_actions, dtype=np.float32)[:, a0:a0 + -(-horizon // spa)]
        acts = torch.tensor(np.ascontiguousarray(acts), device=dev)
        B.sim_set_tool(sim2.h, -1, pose.contiguous(), acts.contiguous(), acts.shape[1])
    sim2.step(horizon)
    w = cotangent_field(sur.n, S, seed, field, dev)
    for s in range(S):
        xs, vs, Cs, _ = sim2.state(scene=s, with_CF=True)
        gx, gv, gC = sur.features_vjp(xs, vs, Cs, mat_all[offs[s]:offs[s + 1]], mm, w[s])
        B.sim_add_state_grad(sim2.h, s, gx, gv, gC.reshape(-1, 9).contiguous())
    _, g_sim, _ = sim2.backward(want_actions=False)
    sim2.close()
    frames = sur.empty_frames(S)
    for s in range(S):
        sl = slice(offs[s], offs[s + 1])
        sur.features(x[sl], v[sl], C[sl], mat_all[sl], mm, frames[s])
    g_sur = torch.empty_like(g_sim)
    g_id = torch.empty_like(g_sim)
    ids = torch.arange(S, dtype=torch.int32, device=dev)
    for k in range(0, S, sur.max_batch):
        i = ids[k:k + sur.max_batch].contiguous()
        gf = sur.vjp(frames, i, w[i.long()][..., 1:4].contiguous())
        for j, s in enumerate(i.tolist()):
            sl = slice(offs[s], offs[s + 1])
            g_sur[sl] = sur.features_vjp(x[sl], v[sl], C[sl], mat_all[sl], mm, gf[j])[1]
            g_id[sl] = sur.features_vjp(x[sl], v[sl], C[sl], mat_all[sl], mm, w[s])[1]

    def metrics(g):
        r, c = [], []
        for s in range(S):
            a, b = g[offs[s]:offs[s + 1]].double().ravel(), g_sim[offs[s]:offs[s + 1]].double().ravel()
            r.append(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)))
            c.append(float(a @ b / (torch.linalg.norm(a) * torch.linalg.norm(b))))
        return np.array(r), np.array(c)

    rs, cs = metrics(g_sur)
    ri, ci = metrics(g_id)
    return {"rel_l2": rs, "cosine": cs, "identity_rel_l2": ri, "identity_cosine": ci,
            "g_sim": g_sim, "g_surrogate": g_sur, "w": w, "state": (x, v, C, F)}


class GatedPredictor:
    """Surrogate prediction of the grid momentum `horizon` steps ahead with the
    full simulation as fallback and as the reference for its error: every
    `check_every`-th call (and the first) also advances the simulation and
    measures the surrogate's relative L2 error against it; while the last
    measured error of a scene exceeds `bound`, that scene's prediction is the
    simulated frame."""

    def __init__(self, sur, bound, check_every=4):
        self.sur, self.bound, self.check_every = sur, float(bound), int(check_every)
        self.calls = 0
        self.fallback = None
        self.last_error = None

    def step(self, sim, scene, frames_now, frames_next, horizon=10):
        """frames_now: (S, n^3, 8) frames of the current state. Returns the
        predicted normalised momentum (S, n^3, 3) and the per-scene source
        ('surrogate' or 'mpm'). Advances `sim` by `horizon` steps only on a
        check call or when some scene is on the fallback."""
        S = scene.n_scenes
        pred = self.sur.predict(frames_now)
        check = self.calls % self.check_every == 0 or (self.fallback is not None and self.fallback.any())
        self.calls += 1
        if self.fallback is None:
            self.fallback = np.zeros(S, dtype=bool)
        if check:
            sim.step(horizon)
            frames_of_state(self.sur, sim, scene, frames_next)
            both = torch.cat([frames_now, frames_next])
            idx = torch.arange(S, dtype=torch.int32, device=self.sur.device)
            err = np.concatenate([self.sur.eval(both, idx[k:k + self.sur.max_batch],
                                                idx[k:k + self.sur.max_batch] + S)
                                  for k in range(0, S, self.sur.max_batch)])
            self.last_error = err
            self.fallback = err > self.bound
            if self.fallback.any():
                mpm = frames_next.view(torch.bfloat16)[..., 1:4].float()
                sel = torch.as_tensor(np.nonzero(self.fallback)[0], device=pred.device)
                pred[sel] = mpm[sel]
        return pred, np.where(self.fallback, "mpm", "surrogate")
