"""Shared helpers of the GPU parity tests: run the CUDA library and the FP64
oracle on the same seeded scene and compare."""
import numpy as np
import torch

from oracle import mpm as omp

DT = torch.float64


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_forward(sc, n_steps=None, scene_index=0):
    with torch.no_grad():
        x, v, C, F = omp.rollout(sc, n_steps=n_steps, scene_index=scene_index)
    return x.numpy(), v.numpy(), C.numpy(), F.numpy()


def oracle_grad(sc, n_steps=None, scene_index=0, want_actions=False, checkpoint=False):
    """Loss and gradients (x0, v0[, actions]) of the scene's loss through the oracle."""
    lo = int(sum(sc.scene_counts[:scene_index]))
    hi = lo + int(sc.scene_counts[scene_index])
    x0 = torch.tensor(sc.x[lo:hi], dtype=DT, requires_grad=True)
    v0 = torch.tensor(sc.v[lo:hi], dtype=DT, requires_grad=True)
    act = None
    if want_actions:
        act = torch.tensor(sc.tool_actions[scene_index], dtype=DT, requires_grad=True)
    x, v, C, F = omp.rollout(sc, n_steps=n_steps, x0=x0, v0=v0, actions=act, scene_index=scene_index,
                             checkpoint_steps=checkpoint)
    L = omp.scene_loss(sc, x, scene_index=scene_index)
    L.backward()
    out = dict(loss=L.item(), x0=x0.grad.numpy(), v0=v0.grad.numpy())
    if want_actions:
        out["actions"] = act.grad.numpy()
    return out
