"""FP64 oracle: the kinematic SDF tool, its contact model and its kinematics
(test infrastructure).

Sec. 3.2 "Inter-material coupling": a mesh object is a time-varying SDF and its
contact with particle material is computed on the grid from the SDF normal with
Coulomb friction (Stomakhin et al. 2013). Sec. 5.1 "Soft Contact Model": contact
acts within a distance threshold and the post-contact velocity v_c is blended
with the original one, v_new = alpha v_c + (1 - alpha) v, alpha = min(exp(-d), 1).
Readings used here: d is the signed distance divided by a softness length ell,
contact acts where phi < eps_c and only while the relative normal velocity is
approaching (v_n < 0). The tool here is an analytic box.

The 6-vector action (Sec. 4.2) is the tool's linear and angular velocity in the
world frame, held for `substeps_per_action` steps (App. B.1: 10 substeps per
frame); the pose integrates as p <- p + dt pdot, q <- normalize(dq(omega dt) q).
"""
from __future__ import annotations

import torch


def quat_mul(a, b):
    """Hamilton product of quaternions (w, x, y, z)."""
    aw, ax, ay, az = a.unbind(-1)
    bw, bx, by, bz = b.unbind(-1)
    return torch.stack([
        aw * bw - ax * bx - ay * by - az * bz,
        aw * bx + ax * bw + ay * bz - az * by,
        aw * by - ax * bz + ay * bw + az * bx,
        aw * bz + ax * by - ay * bx + az * bw,
    ], dim=-1)


def quat_to_rot(q):
    """Rotation matrix of a unit quaternion (w, x, y, z)."""
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], dim=-2)


def rotation_increment(omega, dt):
    """Unit quaternion of the rotation by angle |omega| dt about omega."""
    ang = torch.linalg.norm(omega) * dt
    half = 0.5 * ang
    # sin(half)/|omega| written through sinc to stay smooth at omega = 0
    sinc = torch.sinc(half / torch.pi)  # torch.sinc(x) = sin(pi x)/(pi x)
    return torch.cat([torch.cos(half)[None], 0.5 * dt * sinc * omega])


def tool_trajectory(pose0, actions, n_steps, dt, substeps_per_action):
    """Per-step tool state for steps 0..n_steps-1: p (T,3), q (T,4), pdot (T,3), omega (T,3)."""
    p = pose0[:3]
    q = pose0[3:7] / torch.linalg.norm(pose0[3:7])
    ps, qs, pds, oms = [], [], [], []
    for n in range(n_steps):
        a = actions[min(n // substeps_per_action, actions.shape[0] - 1)]
        pdot, omega = a[:3], a[3:6]
        ps.append(p)
        qs.append(q)
        pds.append(pdot)
        oms.append(omega)
        p = p + dt * pdot
        q = quat_mul(rotation_increment(omega, dt), q)
        q = q / torch.linalg.norm(q)
    return torch.stack(ps), torch.stack(qs), torch.stack(pds), torch.stack(oms)


def box_sdf(y, half):
    """Signed distance phi of local points y (M,3) to a box of half-extents
    `half` centred at the origin, and its gradient g = d phi / d y (unit length).
    Outside: phi = |max(e, 0)|, g = sign(y) max(e, 0) / phi; inside: phi = max_k e_k,
    g = sign(y_k) e_k along the axis k of largest e_k (lowest k on a tie);
    e = |y| - half, sign(0) = +1."""
    sgn = torch.where(y >= 0, 1.0, -1.0).to(y.dtype)
    e = y.abs() - half
    ep = torch.clamp(e, min=0.0)
    outside = (e > 0).any(dim=-1)
    nrm = torch.linalg.norm(ep, dim=-1)
    nrm_safe = torch.where(outside, nrm, torch.ones_like(nrm))
    emax, kmax = e.max(dim=-1)
    g_out = sgn * ep / nrm_safe[:, None]
    g_in = sgn * torch.nn.functional.one_hot(kmax, 3).to(y.dtype)
    phi = torch.where(outside, nrm, emax)
    g = torch.where(outside[:, None], g_out, g_in)
    return phi, g


def contact(u, xi, p, R, pdot, omega, half, eps_c, ell, mu_f):
    """Grid velocity after soft Coulomb contact with a moving box tool.
    u: (M,3) node velocities, xi: (M,3) node positions."""
    r = xi - p
    y = r @ R                      # R^T r for each row
    phi, g = box_sdf(y, half)
    n = g @ R.T                    # world normal R g
    vT = pdot + torch.cross(omega.expand_as(r), r, dim=-1)
    vr = u - vT
    vn = (vr * n).sum(-1)
    approach = vn < 0
    t = vr - vn[:, None] * n
    tn = torch.linalg.norm(t, dim=-1)
    stick = tn <= -mu_f * vn
    tn_safe = torch.where(stick | ~approach, torch.ones_like(tn), tn)
    slide = t * (1.0 + mu_f * vn / tn_safe)[:, None]
    vr_new = torch.where(approach[:, None], torch.where(stick[:, None], torch.zeros_like(t), slide), vr)
    vc = vr_new + vT
    alpha = torch.exp(-torch.clamp(phi, min=0.0) / ell)   # = min(exp(-phi/ell), 1)
    blended = alpha[:, None] * vc + (1.0 - alpha[:, None]) * u
    active = phi < eps_c
    return torch.where(active[:, None], blended, u)
