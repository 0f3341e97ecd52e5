"""Gas solver handle (include/mpm_gas.h): the grid-based incompressible gas
of Sec. 3.2 (after Stam 1999) and its adjoint, on torch device buffers."""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class GasSolver:
    """One gas handle. solid: (n, n, n) bool/uint8 obstacle mask (cells outside
    the grid count as solid). Fields are (3, n, n, n) velocity and (n, n, n)
    smoke density, FP32 on `device`."""

    def __init__(self, n, dt, buoyancy, jacobi_iters, max_steps, solid, device="cuda", stream=None):
        self.n = int(n)
        self.device = torch.device(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.h = B.gas_create(n, dt, buoyancy, jacobi_iters, max_steps, np.asarray(solid, dtype=np.uint8), stream)

    def _f(self, a, shape):
        return torch.as_tensor(a, dtype=torch.float32, device=self.device).reshape(shape).contiguous()

    def set_state(self, u, d):
        n = self.n
        B.gas_set_state(self.h, self._f(u, (3, n, n, n)), self._f(d, (n, n, n)))

    def step(self, n_steps):
        B.gas_step(self.h, n_steps)

    def state(self):
        n = self.n
        u = torch.empty(3, n, n, n, device=self.device)
        d = torch.empty(n, n, n, device=self.device)
        B.gas_get_state(self.h, u, d)
        return u, d

    def add_grad(self, dLdu=None, dLdd=None):
        n = self.n
        B.gas_add_grad(self.h, None if dLdu is None else self._f(dLdu, (3, n, n, n)),
                       None if dLdd is None else self._f(dLdd, (n, n, n)))

    def backward(self):
        n = self.n
        gu = torch.empty(3, n, n, n, device=self.device)
        gd = torch.empty(n, n, n, device=self.device)
        B.gas_backward(self.h, gu, gd)
        return gu, gd

    def launches(self):
        return B.gas_kernel_launches(self.h)

    def close(self):
        if self.h is not None:
            B.gas_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
