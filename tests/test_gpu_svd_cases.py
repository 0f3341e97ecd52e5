"""GPU parity where the FP32 3x3 SVD and the return mappings are least
comfortable (Sec. 3.2 constitutive step, App. A SVD gradient): elastoplastic
and granular particles whose deformation gradient starts nearly singular
(det F -> 0+), with two singular values nearly or exactly equal, inverted
(det F < 0), or a hair away from a rotation. The state is set through the
C-ABI (sim_set_state); x, v after the steps and the gradients of a position
loss w.r.t. the initial x and v are compared with the FP64 oracle stepping
from the same state (tolerances of the other parity tests: 1e-4 relative L2 on
x and v, 1e-3 on gradients). The loss is linear in the final v and C with
seeded random weights, L = sum_p a_p . v_p + B_p : C_p: in these states the
stress term of the affine momentum outweighs m_p C_p, so C and the gradients
carry the constitutive model and its SVD adjoint rather than the free
motion."""
import math

import numpy as np
import pytest
import torch

import scenes
from gpu_util import rel
from oracle import mpm as omp

pytestmark = pytest.mark.gpu
DT = torch.float64
TOL_X, TOL_G = 1e-4, 1e-3

# singular values of the initial F, one case per particle (cyclic)
CASES = {
    "near_singular": (1.3, 1.0, 0.02),
    "coincident_pair": (1.02, 1.02 + 1e-6, 0.97),
    "exact_rotation": (1.0, 1.0, 1.0),
    "inverted": (1.05, 0.98, -0.1),
    "near_identity": (1.0 + 1e-6, 1.0, 1.0 - 1e-6),
    "strong_shear": (1.6, 0.9, 0.7),
}


def _rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def initial_F(n, seed, which=None):
    rng = np.random.default_rng(seed)
    names = list(CASES) if which is None else [which]
    F = np.empty((n, 3, 3))
    for p in range(n):
        s = CASES[names[p % len(names)]]
        F[p] = _rotation(rng) @ np.diag(s) @ _rotation(rng).T
    return F


def _scene(kinds, seed):
    return scenes.small_block(seed=seed, grid_n=16, kinds=kinds, ppc=2, size_cells=6, v0=(0.1, 0.0, -0.05),
                              n_steps=3, gravity=(0.0, -9.8, 0.0))


def _weights(n, seed=11):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, 3)), rng.normal(size=(n, 3, 3))


def _oracle(sc, F0, T):
    model = omp.Model(sc)
    mass, vol = model.particle_mass_volume(sc.mat)
    x0 = torch.tensor(sc.x, dtype=DT, requires_grad=True)
    v0 = torch.tensor(sc.v, dtype=DT, requires_grad=True)
    x, v = x0, v0
    C = torch.zeros(sc.n_particles, 3, 3, dtype=DT)
    F = torch.tensor(F0, dtype=DT)
    for _ in range(T):
        x, v, C, F = omp.step(x, v, C, F, sc.mat, mass, vol, model)
    a, Bw = (torch.tensor(t, dtype=DT) for t in _weights(sc.n_particles))
    L = (a * v).sum() + (Bw * C).sum()
    L.backward()
    return x.detach(), v.detach(), C.detach(), float(L.detach()), x0.grad, v0.grad


@pytest.mark.parametrize("kinds", [[1], [2], [1, 2]], ids=["von_mises", "drucker_prager", "both"])
@pytest.mark.parametrize("which", [None, "near_singular", "inverted"])
def test_degenerate_deformation_gradients_forward_and_gradient(kinds, which):
    from paper_2303_02346_gb300 import binding as B
    from paper_2303_02346_gb300.simulator import Simulator
    sc = _scene(kinds, seed=31 + len(kinds))
    T = sc.n_steps
    F0 = initial_F(sc.n_particles, seed=7, which=which)
    xo, vo, Co, Lo, gxo, gvo = _oracle(sc, F0, T)
    assert torch.isfinite(xo).all() and torch.isfinite(gxo).all()
    sim = Simulator(sc, checkpoint_every=T, max_steps=T)
    f32 = lambda t: torch.as_tensor(t, dtype=torch.float32).contiguous().cuda()
    B.sim_set_state(sim.h, -1, f32(sc.x), f32(sc.v), f32(np.zeros((sc.n_particles, 9))),
                    f32(F0.reshape(-1, 9)), torch.tensor(sc.mat, dtype=torch.uint8).cuda())
    sim.step(T)
    x, v, C, _ = sim.state(with_CF=True)
    a, Bw = _weights(sc.n_particles)
    B.sim_add_state_grad(sim.h, -1, None, f32(a), f32(Bw.reshape(-1, 9)))
    gx, gv, _ = sim.backward()
    sim.close()
    assert rel(x.cpu(), xo) < TOL_X
    assert rel(v.cpu(), vo) < TOL_X
    assert rel(C.cpu(), Co) < TOL_X
    assert rel(gx.cpu(), gxo) < TOL_G
    assert rel(gv.cpu(), gvo) < TOL_G
