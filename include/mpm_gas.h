/*
 * mpm_gas.h - C-ABI of the grid-based gas solver (paper Sec. 3.2 "Gas": an
 * incompressible fluid on a Cartesian grid after Stam 1999, "Stable Fluids";
 * App. A: the gradient of the projection step is written by hand) and its
 * reverse-mode adjoint.
 *
 * Grid: n^3 cells of size dx = 1/n; velocity u (3 components) and smoke
 * density d at cell centres; a solid mask marks obstacle cells (the paper
 * treats cells occupied by meshes as the gas field's boundaries), and cells
 * outside the grid count as solid. One step:
 *   1. buoyancy        u_y += dt * buoyancy * d
 *   2. advection       semi-Lagrangian: back-trace X = i - dt u(i) / dx in
 *                      cell-index space, clamped to [0, n - 1], trilinear
 *                      interpolation of u and d; u = d = 0 in solid cells
 *   3. projection      b = central-difference divergence (solid neighbours
 *                      contribute zero velocity) minus its mean over the fluid
 *                      cells; K damped Jacobi sweeps (weight 2/3) from p = 0 on
 *                      the zero-flux Laplacian of the fluid cells; u -= the
 *                      central-difference gradient of p (p mirrored across
 *                      solid faces)
 * No diffusion (inviscid). K is fixed, so the step is a fixed differentiable
 * map; its adjoint runs the same sweeps (the sweep operator is symmetric).
 *
 * Layout: fields are FP32 arrays of n^3 in (i, j, k) row-major order (k
 * fastest); u is three such arrays back to back (u_x, u_y, u_z). solid: n^3
 * bytes (nonzero = solid), host memory, copied at creation.
 *
 * Conventions as in mpm_sim.h: every call returns a sim_status,
 * gas_last_error() describes the last failure; the handle owns its device
 * memory; work runs on config.cuda_stream and every call synchronises it.
 * The handle keeps the state of every step of the current trajectory (4 n^3
 * floats per step, max_steps + 1 states) for the adjoint.
 */
#ifndef MPM_GAS_H
#define MPM_GAS_H

#include <stdint.h>

#include "mpm_sim.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_gas* gas_h;

typedef struct {
    int n;              /* cells per axis, 8 <= n <= 512 */
    float dt;           /* time step */
    float buoyancy;     /* beta: u_y += dt * beta * d */
    int jacobi_iters;   /* K >= 1 damped Jacobi sweeps per projection */
    int max_steps;      /* longest trajectory gas_backward must cover, >= 1 */
    void* cuda_stream;  /* cudaStream_t; NULL = legacy default stream */
} gas_config;

sim_status gas_create(const gas_config* cfg, const uint8_t* solid, gas_h* out);
sim_status gas_destroy(gas_h h);

/* Start a trajectory from u [3][n^3] and d [n^3] (u and d are zeroed in solid
 * cells); clears the adjoint seeds. */
sim_status gas_set_state(gas_h h, const float* u, const float* d, int on_device);

/* Advance n_steps steps (the trajectory may not exceed max_steps). */
sim_status gas_step(gas_h h, int n_steps);

/* State of the current step (either pointer may be NULL). */
sim_status gas_get_state(gas_h h, float* u, float* d, int on_device);

/* Accumulate loss gradients dL/du [3][n^3], dL/dd [n^3] (either may be NULL)
 * with respect to the state of the current step. */
sim_status gas_add_grad(gas_h h, const float* dLdu, const float* dLdd, int on_device);

/* Reverse sweep over the trajectory since gas_set_state: writes dL/du0 and
 * dL/dd0 (either may be NULL) of the initial state and clears the seeds.
 * SIM_E_STATE before any step. */
sim_status gas_backward(gas_h h, float* dLdu0, float* dLdd0, int on_device);

/* Kernels this handle has launched (graph replays count their nodes). */
long long gas_kernel_launches(gas_h h);

const char* gas_last_error(gas_h h);

#ifdef __cplusplus
}
#endif

#endif /* MPM_GAS_H */
