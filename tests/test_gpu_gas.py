"""GPU parity of the gas solver (Sec. 3.2, Stam 1999) against the FP64 oracle
through the C-ABI: states after several steps, and the gradient of a linear
loss on the final state w.r.t. the initial state against autograd through the
oracle (the projection's adjoint is hand-written in the library)."""
import numpy as np
import pytest
import torch

from gpu_util import rel
from oracle import gas as G

pytestmark = pytest.mark.gpu
DT = torch.float64


def _case(n, seed=0, obstacle=True):
    solid = np.zeros((n, n, n), dtype=bool)
    solid[0, :, :] = solid[-1, :, :] = solid[:, 0, :] = solid[:, -1, :] = solid[:, :, 0] = solid[:, :, -1] = True
    if obstacle:
        c = n // 2
        solid[c - 2:c + 1, c + 1:c + 3, c - 2:c + 2] = True
    rng = np.random.default_rng(seed)
    f = ~solid
    idx = np.arange(n) / n
    X, Y, Z = np.meshgrid(idx, idx, idx, indexing="ij")
    u = np.stack([np.sin(2 * np.pi * Y) * np.cos(2 * np.pi * Z), 0.5 * np.sin(2 * np.pi * X),
                  np.cos(2 * np.pi * X) * np.sin(2 * np.pi * Y)]) * 0.5
    u = u + 0.1 * rng.normal(size=u.shape)
    d = np.exp(-((X - 0.5) ** 2 + (Y - 0.3) ** 2 + (Z - 0.5) ** 2) / 0.01)
    return solid, (u * f).astype(np.float32), (d * f).astype(np.float32)


def _solver(n, solid, T, K, dt=0.01, beta=4.0):
    from paper_2303_02346_gb300.gas import GasSolver
    return GasSolver(n, dt, beta, K, T, solid)


@pytest.mark.parametrize("n,T,K", [(16, 4, 20), (33, 3, 40)])
def test_forward_matches_oracle(n, T, K):
    solid, u0, d0 = _case(n)
    gs = _solver(n, solid, T, K)
    gs.set_state(u0, d0)
    gs.step(T)
    u, d = gs.state()
    uo, do = G.rollout(u0.astype(np.float64), d0.astype(np.float64), solid, T, 0.01, 4.0, K)
    assert rel(u.cpu(), uo) < 1e-4
    assert rel(d.cpu(), do) < 1e-4
    gs.close()


def test_gradient_matches_oracle_autograd():
    n, T, K = 16, 3, 20
    solid, u0, d0 = _case(n, seed=1)
    rng = np.random.default_rng(2)
    wu = rng.normal(size=(3, n, n, n)).astype(np.float32)
    wd = rng.normal(size=(n, n, n)).astype(np.float32)
    gs = _solver(n, solid, T, K)
    gs.set_state(u0, d0)
    gs.step(T)
    gs.add_grad(wu, wd)
    gu, gd = gs.backward()
    f = torch.tensor(~solid, dtype=DT)
    ur = torch.tensor(u0, dtype=DT, requires_grad=True)
    dr = torch.tensor(d0, dtype=DT, requires_grad=True)
    uT, dT = G.rollout(ur * f, dr * f, solid, T, 0.01, 4.0, K)
    L = (torch.tensor(wu, dtype=DT) * uT).sum() + (torch.tensor(wd, dtype=DT) * dT).sum()
    ru, rd = torch.autograd.grad(L, (ur, dr))
    assert rel(gu.cpu(), ru) < 1e-3
    assert rel(gd.cpu(), rd) < 1e-3
    # a second trajectory on the same handle (graphs replayed) gives the same gradient
    gs.set_state(u0, d0)
    gs.step(T)
    gs.add_grad(wu, wd)
    gu2, gd2 = gs.backward()
    assert rel(gu2.cpu(), gu.cpu()) < 1e-5 and rel(gd2.cpu(), gd.cpu()) < 1e-5
    gs.close()


def test_gas_rejects_bad_calls():
    from paper_2303_02346_gb300.binding import SimError
    n = 8
    solid, u0, d0 = _case(n, obstacle=False)
    with pytest.raises(SimError):
        _solver(4, np.zeros((4, 4, 4), bool), 2, 4)  # n below 8
    gs = _solver(n, solid, 2, 4)
    with pytest.raises(SimError):
        gs.step(1)  # no state
    gs.set_state(u0, d0)
    with pytest.raises(SimError):
        gs.backward()  # no step taken
    with pytest.raises(SimError):
        gs.step(3)  # beyond max_steps
    gs.step(2)
    u, d = gs.state()
    assert float(u[:, torch.as_tensor(solid)].abs().max()) == 0.0
    gs.close()


def test_full_size_256_forward_and_64_gradient():
    """The bench's size (256^3, 60 sweeps): two steps against the oracle; the
    adjoint at 64^3 (vector sweeps) against autograd."""
    n, T, K = 256, 2, 60
    solid, u0, d0 = _case(n, seed=3)
    gs = _solver(n, solid, T, K, dt=0.002)
    gs.set_state(u0, d0)
    gs.step(T)
    u, d = gs.state()
    gs.close()
    uo, do = G.rollout(u0.astype(np.float64), d0.astype(np.float64), solid, T, 0.002, 4.0, K)
    assert rel(u.cpu(), uo) < 1e-4
    assert rel(d.cpu(), do) < 1e-4
    n, T, K = 64, 2, 30
    solid, u0, d0 = _case(n, seed=4)
    rng = np.random.default_rng(5)
    wu = rng.normal(size=(3, n, n, n)).astype(np.float32)
    gs = _solver(n, solid, T, K)
    gs.set_state(u0, d0)
    gs.step(T)
    gs.add_grad(wu, None)
    gu, gd = gs.backward()
    gs.close()
    f = torch.tensor(~solid, dtype=DT)
    ur = torch.tensor(u0, dtype=DT, requires_grad=True)
    dr = torch.tensor(d0, dtype=DT, requires_grad=True)
    uT, _ = G.rollout(ur * f, dr * f, solid, T, 0.01, 4.0, K)
    ru, rd = torch.autograd.grad((torch.tensor(wu, dtype=DT) * uT).sum(), (ur, dr))
    assert rel(gu.cpu(), ru) < 1e-3
    assert rel(gd.cpu(), rd) < 1e-3
