"""Thin ctypes binding of the C-ABI declared in include/mpm_sim.h and
include/mpm_surrogate.h.

Functions keep the C names (sim_create, sim_step, ...). They only marshal
arguments: tensors and arrays become pointers plus an `on_device` flag, config
dicts become the C struct, and non-zero status codes become `SimError`. Every
computation runs in the CUDA library; if the library cannot be loaded, every
call raises (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SIM_MAX_MATERIALS = 8
STATUS = {0: "SIM_OK", 1: "SIM_E_ARG", 2: "SIM_E_OOM", 3: "SIM_E_CUDA", 4: "SIM_E_DOMAIN",
          5: "SIM_E_NAN", 6: "SIM_E_STATE", 7: "SIM_E_TIMEOUT"}

# Every symbol include/mpm_sim.h declares.
EXPORTS = ["sim_create", "sim_destroy", "sim_set_particles", "sim_set_tool", "sim_step",
           "sim_current_step", "sim_get_state", "sim_add_loss_grad", "sim_position_loss",
           "sim_grid_mass_loss", "sim_backward", "sim_sync", "sim_last_error",
           "sim_profile_enable", "sim_profile_read", "sim_kernel_launches", "sim_version",
           "sim_grid_mass_loss_static", "sim_autotune", "sim_set_launch", "sim_set_state",
           "sim_add_state_grad", "sim_attraction_loss", "sim_share_gradients", "sim_get_tool_pose",
           "sim_selftest_grid_barrier"]

# Every symbol include/mpm_surrogate.h declares.
SUR_EXPORTS = ["sur_param_count", "sur_create", "sur_destroy", "sur_set_params", "sur_get_params",
               "sur_features", "sur_features_vjp", "sur_predict", "sur_loss_grad", "sur_vjp", "sur_train_step",
               "sur_eval", "sur_profile_enable", "sur_profile_read", "sur_kernel_launches",
               "sur_last_error", "sur_selftest_mma", "sur_mn_major_swap"]


# Every symbol include/mpm_gas.h declares.
GAS_EXPORTS = ["gas_create", "gas_destroy", "gas_set_state", "gas_step", "gas_get_state", "gas_add_grad",
               "gas_backward", "gas_kernel_launches", "gas_last_error"]


class SimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class sim_material(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("rho", ctypes.c_float), ("volume", ctypes.c_float),
                ("E", ctypes.c_float), ("nu", ctypes.c_float), ("bulk", ctypes.c_float),
                ("yield_stress", ctypes.c_float), ("friction_deg", ctypes.c_float),
                ("crit_compress", ctypes.c_float), ("crit_stretch", ctypes.c_float),
                ("shear", ctypes.c_float)]


class gas_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("dt", ctypes.c_float), ("buoyancy", ctypes.c_float),
                ("jacobi_iters", ctypes.c_int), ("max_steps", ctypes.c_int), ("cuda_stream", ctypes.c_void_p)]


class sim_config(ctypes.Structure):
    _fields_ = [("grid_n", ctypes.c_int), ("dt", ctypes.c_float), ("gravity", ctypes.c_float * 3),
                ("bound", ctypes.c_int), ("substeps_per_action", ctypes.c_int),
                ("checkpoint_every", ctypes.c_int), ("max_steps", ctypes.c_int),
                ("n_materials", ctypes.c_int), ("materials", sim_material * SIM_MAX_MATERIALS),
                ("tool_enabled", ctypes.c_int), ("tool_half", ctypes.c_float * 3),
                ("contact_eps", ctypes.c_float), ("contact_soft", ctypes.c_float),
                ("friction", ctypes.c_float), ("n_scenes", ctypes.c_int),
                ("scene_counts", ctypes.POINTER(ctypes.c_int)), ("cuda_stream", ctypes.c_void_p),
                ("resort_every", ctypes.c_int), ("no_graphs", ctypes.c_int)]


class sur_config(ctypes.Structure):
    _fields_ = [("grid_n", ctypes.c_int), ("channels", ctypes.c_int), ("blocks", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("m_ref", ctypes.c_float), ("v_ref", ctypes.c_float),
                ("adam_beta1", ctypes.c_float), ("adam_beta2", ctypes.c_float),
                ("adam_eps", ctypes.c_float), ("cuda_stream", ctypes.c_void_p)]


_LIB = None


def load(path: str | None = None):
    """Load the CUDA library (building it first if it is missing)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.lib_path()
    if not os.path.exists(path):
        _build.build()
    lib = ctypes.CDLL(path)
    V, I, F, D, P = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_void_p
    sig = {
        "sim_create": (I, [ctypes.POINTER(sim_config), ctypes.POINTER(V)]),
        "sim_destroy": (I, [V]),
        "sim_set_particles": (I, [V, I, P, P, P, I]),
        "sim_set_tool": (I, [V, I, P, P, I, I]),
        "sim_step": (I, [V, I]),
        "sim_current_step": (I, [V]),
        "sim_get_state": (I, [V, I, I, P, P, P, P, I]),
        "sim_add_loss_grad": (I, [V, I, I, P, P, I]),
        "sim_position_loss": (I, [V, I, I, P, F, P]),
        "sim_grid_mass_loss": (I, [V, I, I, P, P, F, I, P]),
        "sim_get_tool_pose": (I, [V, I, I, P, I]),
        "sim_backward": (I, [V, P, P, P, I]),
        "sim_sync": (I, [V]),
        "sim_last_error": (ctypes.c_char_p, [V]),
        "sim_profile_enable": (I, [V, I]),
        "sim_profile_read": (I, [V, I, P, P, P, P]),
        "sim_kernel_launches": (ctypes.c_longlong, [V]),
        "sim_version": (ctypes.c_char_p, []),
        "sim_grid_mass_loss_static": (I, [P, P, I, I, P, P, F, P, P, V]),
        "sim_autotune": (I, [V, I, P]),
        "sim_set_launch": (I, [V, P]),
        "sim_selftest_grid_barrier": (I, [I, I, I, D, P]),
        "sim_set_state": (I, [V, I, P, P, P, P, P, I]),
        "sim_add_state_grad": (I, [V, I, I, P, P, P, I]),
        "sim_attraction_loss": (I, [V, I, P, F, F, F, I, P]),
        "sim_share_gradients": (I, [V, I, P, F, F, P, P, I]),
        "sur_param_count": (ctypes.c_longlong, [ctypes.POINTER(sur_config)]),
        "sur_create": (I, [ctypes.POINTER(sur_config), ctypes.POINTER(V)]),
        "sur_destroy": (I, [V]),
        "sur_set_params": (I, [V, P, I]),
        "sur_get_params": (I, [V, P, I]),
        "sur_features": (I, [V, I, P, P, P, P, P, I, P]),
        "sur_features_vjp": (I, [V, I, P, P, P, P, P, I, P, P, P, P]),
        "sur_vjp": (I, [V, I, P, P, P, P]),
        "sur_predict": (I, [V, I, P, P, P]),
        "sur_loss_grad": (I, [V, I, P, P, P, P, P, P]),
        "sur_train_step": (I, [V, I, P, P, P, F, P]),
        "sur_eval": (I, [V, I, P, P, P, P]),
        "sur_profile_enable": (I, [V, I]),
        "sur_profile_read": (I, [V, I, P, P, P, P]),
        "sur_kernel_launches": (ctypes.c_longlong, [V]),
        "sur_last_error": (ctypes.c_char_p, [V]),
        "sur_selftest_mma": (I, [P, P, P, I]),
        "sur_mn_major_swap": (ctypes.c_longlong, []),
        "gas_create": (I, [ctypes.POINTER(gas_config), P, ctypes.POINTER(V)]),
        "gas_destroy": (I, [V]),
        "gas_set_state": (I, [V, P, P, I]),
        "gas_step": (I, [V, I]),
        "gas_get_state": (I, [V, P, P, I]),
        "gas_add_grad": (I, [V, P, P, I]),
        "gas_backward": (I, [V, P, P, I]),
        "gas_kernel_launches": (ctypes.c_longlong, [V]),
        "gas_last_error": (ctypes.c_char_p, [V]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


# ----------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------
def _ptr(a):
    """(pointer, on_device) of a torch tensor or numpy array (contiguous)."""
    if a is None:
        return None, 0
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda)
    except ImportError:  # pragma: no cover
        pass
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data), 0
    raise TypeError(f"unsupported buffer type {type(a)}")


def _check(h, status):
    if status != 0:
        lib = load()
        msg = lib.sim_last_error(h)
        raise SimError(status, msg.decode() if msg else "")


def _same_place(*arrays):
    places = {(_ptr(a)[1]) for a in arrays if a is not None}
    if len(places) > 1:
        raise ValueError("all buffers of one call must be on the same side (host or device)")
    return places.pop() if places else 0


def make_config(grid_n, dt, materials, scene_counts, gravity=(0.0, -9.8, 0.0), bound=3,
                substeps_per_action=10, checkpoint_every=0, max_steps=0, tool_enabled=False,
                tool_half=(0.05, 0.01, 0.05), contact_eps=0.0, contact_soft=0.0, friction=0.5,
                cuda_stream=None, resort_every=0, no_graphs=False):
    """Build a sim_config. `materials` is a list of dicts with keys kind, rho,
    volume, E, nu, bulk, yield_stress, friction_deg."""
    cfg = sim_config()
    cfg.grid_n = int(grid_n)
    cfg.dt = float(dt)
    cfg.gravity[:] = [float(g) for g in gravity]
    cfg.bound = int(bound)
    cfg.substeps_per_action = int(substeps_per_action)
    cfg.checkpoint_every = int(checkpoint_every)
    cfg.max_steps = int(max_steps)
    if len(materials) > SIM_MAX_MATERIALS:
        raise ValueError("too many materials")
    cfg.n_materials = len(materials)
    for i, m in enumerate(materials):
        sm = cfg.materials[i]
        sm.kind = int(m["kind"])
        for key in ("rho", "volume", "E", "nu", "bulk", "yield_stress", "friction_deg", "crit_compress",
                    "crit_stretch", "shear"):
            setattr(sm, key, float(m.get(key, 0.0)))
    cfg.tool_enabled = int(bool(tool_enabled))
    cfg.tool_half[:] = [float(h) for h in tool_half]
    cfg.contact_eps = float(contact_eps)
    cfg.contact_soft = float(contact_soft)
    cfg.friction = float(friction)
    counts = (ctypes.c_int * len(scene_counts))(*[int(c) for c in scene_counts])
    cfg._counts_keepalive = counts
    cfg.n_scenes = len(scene_counts)
    cfg.scene_counts = ctypes.cast(counts, ctypes.POINTER(ctypes.c_int))
    cfg.cuda_stream = ctypes.c_void_p(cuda_stream) if cuda_stream else None
    cfg.resort_every = int(resort_every)
    cfg.no_graphs = int(bool(no_graphs))
    return cfg


# ----------------------------------------------------------------------------
# C-ABI functions (same names)
# ----------------------------------------------------------------------------
def sim_create(config: sim_config):
    lib = load()
    h = ctypes.c_void_p()
    st = lib.sim_create(ctypes.byref(config), ctypes.byref(h))
    if st != 0:
        raise SimError(st, "sim_create failed")
    return h


def sim_destroy(h):
    _check(h, load().sim_destroy(h))


def sim_set_particles(h, scene, x, v, material):
    dev = _same_place(x, v, material)
    _check(h, load().sim_set_particles(h, int(scene), _ptr(x)[0], _ptr(v)[0], _ptr(material)[0], dev))


def sim_set_state(h, scene, x, v, C, F, material):
    """Initial state with C and F (None: 0 and I); see sim_set_particles."""
    od = _same_place(x, v, C, F, material)
    _check(h, load().sim_set_state(h, int(scene), _ptr(x)[0], _ptr(v)[0], _ptr(C)[0], _ptr(F)[0],
                                   _ptr(material)[0], od))


def sim_add_state_grad(h, scene, dLdx=None, dLdv=None, dLdC=None, step=-1):
    """Seeds dL/dx, dL/dv, dL/dC of the state at `step` (-1: the current step)."""
    od = _same_place(dLdx, dLdv, dLdC)
    _check(h, load().sim_add_state_grad(h, int(scene), int(step), _ptr(dLdx)[0], _ptr(dLdv)[0], _ptr(dLdC)[0],
                                         od))


def sim_set_tool(h, scene, pose0, actions, n_actions):
    dev = _same_place(pose0, actions)
    _check(h, load().sim_set_tool(h, int(scene), _ptr(pose0)[0], _ptr(actions)[0], int(n_actions), dev))


def sim_step(h, n_steps):
    _check(h, load().sim_step(h, int(n_steps)))


def sim_current_step(h):
    return int(load().sim_current_step(h))


def sim_get_state(h, scene, step, x=None, v=None, C=None, F=None):
    dev = _same_place(x, v, C, F)
    _check(h, load().sim_get_state(h, int(scene), int(step), _ptr(x)[0], _ptr(v)[0], _ptr(C)[0],
                                    _ptr(F)[0], dev))


def sim_add_loss_grad(h, scene, dLdx=None, dLdv=None, step=-1):
    """Seeds dL/dx, dL/dv of the state at `step` (-1: the current step)."""
    dev = _same_place(dLdx, dLdv)
    _check(h, load().sim_add_loss_grad(h, int(scene), int(step), _ptr(dLdx)[0], _ptr(dLdv)[0], dev))


def sim_position_loss(h, scene, target, weight, n_out=1, step=-1):
    t = np.ascontiguousarray(np.asarray(target, dtype=np.float32))
    out = np.zeros(n_out, dtype=np.float64)
    _check(h, load().sim_position_loss(h, int(scene), int(step), _ptr(t)[0], float(weight), _ptr(out)[0]))
    return out


def sim_grid_mass_loss(h, scene, target_mass, target_dist, total_mass, step=-1):
    dev = _same_place(target_mass, target_dist)
    out = np.zeros(1, dtype=np.float64)
    _check(h, load().sim_grid_mass_loss(h, int(scene), int(step), _ptr(target_mass)[0], _ptr(target_dist)[0],
                                         float(total_mass), dev, _ptr(out)[0]))
    return float(out[0])


def sim_get_tool_pose(h, scene, step, pose):
    """Tool pose at the start of `step` into pose ([S or 1] x 13: position,
    quaternion w x y z, linear and angular velocity)."""
    _check(h, load().sim_get_tool_pose(h, int(scene), int(step), *_ptr(pose)))


def sim_attraction_loss(h, scene, ell, radius, tau, weight=1.0):
    """Attraction loss (Sec. 5.1) at the current state; accumulates its
    gradient into the backward seeds and returns the loss."""
    out = np.zeros(1, dtype=np.float64)
    p, dev = _ptr(ell)
    _check(h, load().sim_attraction_loss(h, int(scene), p, float(radius), float(tau), float(weight), dev,
                                          _ptr(out)[0]))
    return float(out[0])


def sim_share_gradients(h, scene, ell, radius, tau, g, out):
    """Gradient sharing (Sec. 5.1) of g (count x 3, caller order) into out."""
    dev = _same_place(ell, g, out)
    _check(h, load().sim_share_gradients(h, int(scene), _ptr(ell)[0], float(radius), float(tau), _ptr(g)[0],
                                          _ptr(out)[0], dev))


def sim_backward(h, dLdx0=None, dLdv0=None, dLdactions=None):
    dev = _same_place(dLdx0, dLdv0, dLdactions)
    _check(h, load().sim_backward(h, _ptr(dLdx0)[0], _ptr(dLdv0)[0], _ptr(dLdactions)[0], dev))


def sim_sync(h):
    _check(h, load().sim_sync(h))


def sim_last_error(h):
    m = load().sim_last_error(h)
    return m.decode() if m else ""


def sim_profile_enable(h, enable):
    _check(h, load().sim_profile_enable(h, int(bool(enable))))


def sim_profile_read(h, cap=32):
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_double * cap)()
    cnt = (ctypes.c_longlong * cap)()
    n = ctypes.c_int()
    _check(h, load().sim_profile_read(h, cap, ctypes.cast(names, ctypes.c_void_p),
                                       ctypes.cast(ms, ctypes.c_void_p),
                                       ctypes.cast(cnt, ctypes.c_void_p), ctypes.byref(n)))
    return {names[i].decode(): (ms[i], cnt[i]) for i in range(min(n.value, cap))}


def sim_kernel_launches(h):
    return int(load().sim_kernel_launches(h))


def sim_grid_mass_loss_static(x, mass, grid_n, target_mass, target_dist, total_mass, dLdx, loss,
                              stream=None):
    """No-allocation grid-mass loss: every argument is a CUDA tensor; dLdx and
    loss (one float64) are written. Enqueued on `stream` (a cudaStream_t
    handle; default: the legacy default stream).

    The kernels trust the sizes they are given, so every buffer is checked
    here first: x and dLdx float32 [N, 3], mass float32 [N], target_mass and
    target_dist float32 with grid_n^3 entries, loss float64 with one entry,
    all contiguous and on the current CUDA device (ValueError otherwise)."""
    import torch
    names = ("x", "mass", "target_mass", "target_dist", "dLdx", "loss")
    bufs = (x, mass, target_mass, target_dist, dLdx, loss)
    for nm, a in zip(names, bufs):
        if not isinstance(a, torch.Tensor):
            raise ValueError(f"sim_grid_mass_loss_static: {nm} must be a torch tensor")
        if not a.is_contiguous():
            raise ValueError(f"sim_grid_mass_loss_static: {nm} must be contiguous")
    if x.dim() != 2 or x.shape[1] != 3:
        raise ValueError(f"sim_grid_mass_loss_static: x must be [N, 3], got {tuple(x.shape)}")
    N = int(x.shape[0])
    n3 = int(grid_n) ** 3
    want = {"x": (torch.float32, 3 * N), "mass": (torch.float32, N), "target_mass": (torch.float32, n3),
            "target_dist": (torch.float32, n3), "dLdx": (torch.float32, 3 * N), "loss": (torch.float64, 1)}
    for nm, a in zip(names, bufs):
        dt, count = want[nm]
        if a.dtype != dt:
            raise ValueError(f"sim_grid_mass_loss_static: {nm} must be {dt}, got {a.dtype}")
        if a.numel() != count:
            raise ValueError(f"sim_grid_mass_loss_static: {nm} must have {count} entries, got {a.numel()}")
    if tuple(dLdx.shape) != (N, 3):
        raise ValueError(f"sim_grid_mass_loss_static: dLdx must be [{N}, 3], got {tuple(dLdx.shape)}")
    for nm, a in zip(names, bufs):
        if not a.is_cuda:
            raise ValueError("sim_grid_mass_loss_static takes device buffers only")
    cur = torch.cuda.current_device()
    for nm, a in zip(names, bufs):
        if a.device.index != cur:
            raise ValueError(f"sim_grid_mass_loss_static: {nm} is on cuda:{a.device.index}, "
                             f"the current device is cuda:{cur}")
    st = load().sim_grid_mass_loss_static(_ptr(x)[0], _ptr(mass)[0], int(x.shape[0]), int(grid_n),
                                          _ptr(target_mass)[0], _ptr(target_dist)[0],
                                          float(total_mass), _ptr(dLdx)[0], _ptr(loss)[0],
                                          ctypes.c_void_p(stream) if stream else None)
    if st != 0:
        raise SimError(st, "sim_grid_mass_loss_static failed")


def sim_autotune(h, n_steps=0):
    """Time launch-shape candidates on the handle's scene; returns the choices
    (scatter threads, gather threads, grid blocks per CTA, re-sort period,
    adjoint fusion, persistent forward, staged gather, scatter CTAs per SM)."""
    out = (ctypes.c_int * 8)()
    _check(h, load().sim_autotune(h, int(n_steps), ctypes.cast(out, ctypes.c_void_p)))
    return tuple(out)


def sim_set_launch(h, scatter_threads, gather_threads, grid_blocks, resort_every, fuse_adjoint=0, persistent=0,
                   stage_gather=0, scatter_ctas=3):
    c = (ctypes.c_int * 8)(int(scatter_threads), int(gather_threads), int(grid_blocks), int(resort_every),
                           int(fuse_adjoint), int(persistent), int(stage_gather), int(scatter_ctas))
    _check(h, load().sim_set_launch(h, ctypes.cast(c, ctypes.c_void_p)))


def sim_selftest_grid_barrier(blocks, extra_arrivals, rounds, timeout_ms):
    """Run the persistent forward's grid barrier alone; returns (status, passed)
    without raising (status SIM_E_TIMEOUT = 7 is the expected outcome when
    extra_arrivals > 0)."""
    passed = ctypes.c_int(-1)
    st = load().sim_selftest_grid_barrier(int(blocks), int(extra_arrivals), int(rounds), float(timeout_ms),
                                          ctypes.byref(passed))
    return int(st), int(passed.value)


def sim_version():
    return load().sim_version().decode()


# ----------------------------------------------------------------------------
# surrogate (include/mpm_surrogate.h)
# ----------------------------------------------------------------------------
def _sur_check(h, status):
    if status != 0:
        msg = load().sur_last_error(h)
        raise SimError(status, msg.decode() if msg else "")


def _dev(*arrays):
    for a in arrays:
        if a is not None and _ptr(a)[1] != 1:
            raise ValueError("surrogate calls take device tensors")
    return [(_ptr(a)[0] if a is not None else None) for a in arrays]


def make_sur_config(grid_n=64, channels=32, blocks=4, max_batch=8, m_ref=1.0, v_ref=1.0,
                    adam_beta1=0.9, adam_beta2=0.999, adam_eps=1e-8, cuda_stream=0):
    return sur_config(int(grid_n), int(channels), int(blocks), int(max_batch), float(m_ref), float(v_ref),
                      float(adam_beta1), float(adam_beta2), float(adam_eps),
                      ctypes.c_void_p(cuda_stream) if cuda_stream else None)


def sur_param_count(cfg: sur_config):
    return int(load().sur_param_count(ctypes.byref(cfg)))


def sur_create(cfg: sur_config):
    h = ctypes.c_void_p()
    st = load().sur_create(ctypes.byref(cfg), ctypes.byref(h))
    if st != 0:
        raise SimError(st, "sur_create failed (invalid config, out of memory or tensor-core self-test)")
    return h


def sur_destroy(h):
    load().sur_destroy(h)


def sur_set_params(h, params):
    p, on_dev = _ptr(params)
    _sur_check(h, load().sur_set_params(h, p, on_dev))


def sur_get_params(h, out):
    p, on_dev = _ptr(out)
    _sur_check(h, load().sur_get_params(h, p, on_dev))


def sur_features(h, x, v, C, mat, material_mass, frame):
    mm = (ctypes.c_float * len(material_mass))(*[float(m) for m in material_mass])
    px, pv, pC, pm, pf = _dev(x, v, C, mat, frame)
    _sur_check(h, load().sur_features(h, int(x.shape[0]), px, pv, pC, pm, ctypes.cast(mm, ctypes.c_void_p),
                                      len(material_mass), pf))


def sur_features_vjp(h, x, v, C, mat, material_mass, g_frame, dLdx=None, dLdv=None, dLdC=None):
    mm = (ctypes.c_float * len(material_mass))(*[float(m) for m in material_mass])
    px, pv, pC, pm, pg, pdx, pdv, pdC = _dev(x, v, C, mat, g_frame, dLdx, dLdv, dLdC)
    _sur_check(h, load().sur_features_vjp(h, int(x.shape[0]), px, pv, pC, pm, ctypes.cast(mm, ctypes.c_void_p),
                                          len(material_mass), pg, pdx, pdv, pdC))


def sur_vjp(h, batch, frames, idx, g_pred, g_frames):
    pf, pi, pg, pgf = _dev(frames, idx, g_pred, g_frames)
    _sur_check(h, load().sur_vjp(h, int(batch), pf, pi, pg, pgf))


def sur_predict(h, batch, frames, idx, pred):
    pf, pi, pp = _dev(frames, idx, pred)
    _sur_check(h, load().sur_predict(h, int(batch), pf, pi, pp))


def sur_loss_grad(h, batch, frames, idx, tgt, grad=None, g_frames=None):
    loss = ctypes.c_float()
    pf, pi, pt, pg, pgf = _dev(frames, idx, tgt, grad, g_frames)
    _sur_check(h, load().sur_loss_grad(h, int(batch), pf, pi, pt, ctypes.byref(loss), pg, pgf))
    return loss.value


def sur_train_step(h, batch, frames, idx, tgt, lr):
    loss = ctypes.c_float()
    pf, pi, pt = _dev(frames, idx, tgt)
    _sur_check(h, load().sur_train_step(h, int(batch), pf, pi, pt, float(lr), ctypes.byref(loss)))
    return loss.value


def sur_eval(h, batch, frames, idx, tgt):
    out = (ctypes.c_double * (2 * int(batch)))()
    pf, pi, pt = _dev(frames, idx, tgt)
    _sur_check(h, load().sur_eval(h, int(batch), pf, pi, pt, ctypes.cast(out, ctypes.c_void_p)))
    return np.array(out[:], dtype=np.float64).reshape(int(batch), 2)


def sur_profile_enable(h, enable):
    _sur_check(h, load().sur_profile_enable(h, int(bool(enable))))


def sur_profile_read(h, cap=32):
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_double * cap)()
    cnt = (ctypes.c_longlong * cap)()
    n = ctypes.c_int()
    _sur_check(h, load().sur_profile_read(h, cap, ctypes.cast(names, ctypes.c_void_p),
                                          ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(cnt, ctypes.c_void_p),
                                          ctypes.byref(n)))
    return {names[i].decode(): (ms[i], cnt[i]) for i in range(min(n.value, cap))}


def sur_kernel_launches(h):
    return int(load().sur_kernel_launches(h))


def sur_last_error(h):
    m = load().sur_last_error(h)
    return m.decode() if m else ""


def sur_mn_major_swap():
    return int(load().sur_mn_major_swap())


def sur_selftest_mma(a, b, mode=0):
    """D = bf16(A) bf16(B)^T on the tensor cores; a (128, 32), b (32, 32) float32
    host arrays; mode 0 K-major operands, 1 MN-major."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    d = np.zeros((128, 32), dtype=np.float32)
    st = load().sur_selftest_mma(_ptr(a)[0], _ptr(b)[0], _ptr(d)[0], int(mode))
    if st != 0:
        raise SimError(st, "sur_selftest_mma failed")
    return d


# ----------------------------------------------------------------------------
# gas solver (include/mpm_gas.h)
# ----------------------------------------------------------------------------
def _gas_check(h, status):
    if status != 0:
        msg = load().gas_last_error(h)
        raise SimError(status, msg.decode() if msg else "")


def gas_create(n, dt, buoyancy, jacobi_iters, max_steps, solid, cuda_stream=None):
    cfg = gas_config(int(n), float(dt), float(buoyancy), int(jacobi_iters), int(max_steps),
                     ctypes.c_void_p(cuda_stream) if cuda_stream else None)
    s = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(-1))
    h = ctypes.c_void_p()
    st = load().gas_create(ctypes.byref(cfg), s.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h))
    if st != 0:
        raise SimError(st, "gas_create failed")
    return h


def gas_destroy(h):
    load().gas_destroy(h)


def gas_set_state(h, u, d):
    dev = _same_place(u, d)
    _gas_check(h, load().gas_set_state(h, _ptr(u)[0], _ptr(d)[0], dev))


def gas_step(h, n_steps):
    _gas_check(h, load().gas_step(h, int(n_steps)))


def gas_get_state(h, u=None, d=None):
    dev = _same_place(u, d)
    _gas_check(h, load().gas_get_state(h, _ptr(u)[0], _ptr(d)[0], dev))


def gas_add_grad(h, dLdu=None, dLdd=None):
    dev = _same_place(dLdu, dLdd)
    _gas_check(h, load().gas_add_grad(h, _ptr(dLdu)[0], _ptr(dLdd)[0], dev))


def gas_backward(h, dLdu0=None, dLdd0=None):
    dev = _same_place(dLdu0, dLdd0)
    _gas_check(h, load().gas_backward(h, _ptr(dLdu0)[0], _ptr(dLdd0)[0], dev))


def gas_kernel_launches(h):
    return int(load().gas_kernel_launches(h))

