/*
 * mpm_sim.h - C-ABI of the GB300 MLS-MPM step and its reverse-mode adjoint.
 *
 * The library simulates continuum material with the Moving Least Squares
 * Material Point Method, which the paper uses for every particle material,
 * solid or liquid (Sec. 3.2): particle-to-grid scatter
 * of mass, momentum and stress (P2G), a grid update with gravity, sticky walls
 * and soft Coulomb contact against a moving box SDF tool (Sec. 3.2
 * "Inter-material coupling", Sec. 5.1 "Soft Contact Model"), and a
 * grid-to-particle gather with the deformation-gradient update (G2P). Materials
 * are weakly compressible liquid, von Mises elastoplastic (fixed-corotated) and
 * Drucker-Prager sand. It computes gradients through whole trajectories with
 * hand-written adjoint kernels and checkpoint/recompute (Sec. 3.3, App. A).
 *
 * The problem statement follows Sec. 4.2: the state of every scene is an
 * N_p x 6 matrix of particle positions and velocities (plus the affine
 * velocity C and deformation gradient F), and an action is the 6-vector of the
 * tool's linear and angular velocity, held for `substeps_per_action` steps
 * (App. B.1). Losses are on the particle state or on the grid mass field
 * (App. C).
 *
 * Conventions (all entry points)
 * ------------------------------
 * - Every function returns a sim_status; no exception or abort crosses the ABI.
 *   After an error, sim_last_error() gives a message valid until the next call
 *   on the same handle.
 * - The library owns all of its device memory (allocated in sim_create, freed
 *   in sim_destroy). Caller buffers are never retained: every pointer argument
 *   is read or written during the call only.
 * - `on_device` = 1 means the pointer is a CUDA device pointer on the current
 *   device; 0 means host memory. Device-pointer transfers are enqueued on the
 *   simulation's stream; host transfers are synchronous.
 * - Work is enqueued on config.cuda_stream (a cudaStream_t; NULL = the legacy
 *   default stream). sim_step / sim_backward / the loss calls synchronise that
 *   stream before returning and report device-side errors (particle left the
 *   grid, NaN) as SIM_E_DOMAIN / SIM_E_NAN.
 * - Arrays of vectors are row-major: x[3*i + c] is component c of particle i.
 *   3x3 matrices are row-major per particle: C[9*i + 3*r + c].
 * - Particles are addressed by the caller's order inside each scene; the
 *   library re-orders them internally (sorting into grid blocks) and maps back.
 * - Liquid particles carry only the volume ratio J (the paper resets a
 *   liquid's deformation gradient every step, Sec. 3.2); their F is reported as
 *   diag(J, 1, 1).
 * - Scene s owns particles [sum(counts[:s]), sum(counts[:s+1])) of the
 *   concatenated arrays; scene = -1 addresses all scenes at once.
 */
#ifndef MPM_SIM_H
#define MPM_SIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_sim* sim_h;

typedef enum {
    SIM_OK = 0,
    SIM_E_ARG = 1,      /* invalid argument (null pointer, bad size or index) */
    SIM_E_OOM = 2,      /* device allocation failed */
    SIM_E_CUDA = 3,     /* a CUDA runtime call failed */
    SIM_E_DOMAIN = 4,   /* a particle's B-spline stencil left the grid */
    SIM_E_NAN = 5,      /* non-finite particle state */
    SIM_E_STATE = 6,    /* call not valid in the current state (e.g. backward without a trajectory) */
    SIM_E_TIMEOUT = 7   /* a bounded device-side wait gave up */
} sim_status;

typedef enum {
    SIM_LIQUID = 0,          /* weakly compressible: tau = K J (J - 1) I */
    SIM_VON_MISES = 1,       /* fixed-corotated with von Mises return map in Hencky strain */
    SIM_DRUCKER_PRAGER = 2,  /* Hencky StVK with Drucker-Prager return map (Klar et al. 2016) */
    SIM_BOX_YIELD = 3,       /* plastic (Sec. 3.2): fixed-corotated with the box yield criterion of
                                Stomakhin et al. 2013, singular values of F clamped to
                                [1 - crit_compress, 1 + crit_stretch]; no hardening */
    SIM_VISCOUS_LIQUID = 4,  /* viscous liquid (Sec. 3.2): fixed-corotated (mu = shear, lambda =
                                bulk) of the step's trial F, with F reset to J^(1/3) I every
                                step, so the shear stress acts on one step's deformation */
    SIM_RIGID = 5            /* rigid body represented by particles (Sec. 3.2 "Rigid body"): the
                                particles of this material in one scene form one object whose
                                rest shape is their positions at sim_set_particles (not all in
                                one plane). After every G2P they are set to the mass-weighted
                                least-squares rigid fit of their positions (x = c + R rbar, R the
                                polar factor of sum m (x - c) rbar^T) and velocities (v = vbar +
                                w x R rbar, keeping linear and angular momentum); C = [w]_x,
                                F = R, and the P2G stress is zero (corotated stress at F = R).
                                E and nu are not used. */
} sim_material_kind;

#define SIM_MAX_MATERIALS 8

typedef struct {
    int kind;             /* sim_material_kind */
    float rho;            /* density */
    float volume;         /* per-particle volume V_p (mass = rho * volume) */
    float E;              /* Young's modulus (solids) */
    float nu;             /* Poisson ratio (solids) */
    float bulk;           /* bulk modulus K (liquid) */
    float yield_stress;   /* von Mises yield stress tau_Y */
    float friction_deg;   /* Drucker-Prager friction angle in degrees */
    float crit_compress;  /* box yield: theta_c, 0 <= theta_c < 1 */
    float crit_stretch;   /* box yield: theta_s >= 0 */
    float shear;          /* viscous liquid: mu >= 0 */
} sim_material;

typedef struct {
    int grid_n;               /* nodes per axis of every scene's grid; node i at i/grid_n */
    float dt;                 /* time step */
    float gravity[3];
    int bound;                /* sticky walls: nodes with an index < bound or >= grid_n - bound get v = 0 */
    int substeps_per_action;  /* steps an action is held (App. B.1: 10) */
    int checkpoint_every;     /* k > 0: keep a checkpoint every k steps for sim_backward;
                                 0: forward only (no gradient memory is allocated) */
    int max_steps;            /* longest trajectory sim_backward must cover */
    int n_materials;
    sim_material materials[SIM_MAX_MATERIALS];
    int tool_enabled;
    float tool_half[3];       /* box half-extents */
    float contact_eps;        /* contact acts where the SDF < contact_eps */
    float contact_soft;       /* softness length l: alpha = min(exp(-phi / l), 1) */
    float friction;           /* Coulomb friction coefficient */
    int n_scenes;
    const int* scene_counts;  /* host array of n_scenes particle counts (read during sim_create) */
    void* cuda_stream;        /* cudaStream_t the library enqueues on; NULL = default stream */
    int resort_every;         /* forward-only runs: re-sort particles into grid blocks every this
                                 many steps (0 = library default); with checkpointing, particles
                                 are re-sorted at every checkpoint */
    int no_graphs;            /* 0: sim_step / sim_backward capture their kernel sequence in a
                                 CUDA graph on first use and replay it when called again with
                                 the same step range; 1: always launch kernels one by one */
} sim_config;

/* Create a simulation; allocates all device memory for the configured sizes.
 * Errors: SIM_E_ARG (bad config), SIM_E_OOM, SIM_E_CUDA. *out is NULL on error. */
sim_status sim_create(const sim_config* config, sim_h* out);

/* Free everything the handle owns. NULL is accepted. */
sim_status sim_destroy(sim_h h);

/* Set the initial particle state of one scene (scene = -1: all scenes).
 * x, v: [count*3]; material: [count] indices into config.materials.
 * Resets C = 0, F = I, the step counter to 0, the trajectory and all
 * accumulated loss gradients. The caller keeps ownership of the buffers. */
sim_status sim_set_particles(sim_h h, int scene, const float* x, const float* v,
                             const uint8_t* material, int on_device);

/* Like sim_set_particles, and also sets the affine velocity C [n][3][3] and
 * the deformation gradient F [n][3][3] (row-major; NULL = 0 and I). For a
 * liquid particle only F[0][0] is used, as its volume ratio J (sim_get_state
 * reports a liquid's F as diag(J, 1, 1), so its output can be passed back):
 * restarts a trajectory from a saved state. */
sim_status sim_set_state(sim_h h, int scene, const float* x, const float* v, const float* C,
                         const float* F, const uint8_t* mat, int on_device);

/* Set the tool of one scene (scene = -1: all, arrays concatenated per scene):
 * pose0 [7] = position (3) and unit quaternion (w, x, y, z); actions
 * [n_actions*6] = linear velocity (3) and world-frame angular velocity (3),
 * action j applies to steps [j*spa, (j+1)*spa). The pose integrates as
 * p <- p + dt pdot, q <- normalize(exp(omega dt / 2) q). */
sim_status sim_set_tool(sim_h h, int scene, const float* pose0, const float* actions,
                        int n_actions, int on_device);

/* Advance all scenes by n_steps (MLS-MPM steps: constitutive update and P2G,
 * grid update, G2P). With checkpointing on, the total since sim_set_particles
 * may not exceed max_steps. Loss gradients seeded at earlier steps stay
 * pending and are propagated by the one sim_backward at the end (a loss
 * summed over time, App. C: L = sum_t CD(s_t, s*_t), is evaluated step by
 * step as the trajectory advances). Synchronises; returns SIM_E_DOMAIN /
 * SIM_E_NAN if a particle left the grid or became non-finite. */
sim_status sim_step(sim_h h, int n_steps);

/* Number of steps taken since sim_set_particles. */
int sim_current_step(sim_h h);

/* Copy the particle state of a scene at step `step` in the caller's particle
 * order. Any output pointer may be NULL. x, v: [count*3]; C, F: [count*9].
 * The states the trajectory keeps are readable: step = -1 or the current step,
 * step 0 (the initial state) and, with checkpointing, every checkpoint step
 * c*checkpoint_every before the current step (App. A: one state per caching
 * step). Any other step: SIM_E_STATE. */
sim_status sim_get_state(sim_h h, int scene, int step, float* x, float* v, float* C,
                         float* F, int on_device);

/* Tool pose of a scene (scene = -1: all scenes, concatenated) at the start of
 * step `step` (0 <= step < max_steps), as the grid update of that step uses
 * it: 13 floats per scene = position (3), unit quaternion w x y z (4), linear
 * velocity (3), world-frame angular velocity (3): the kinematics of
 * sim_set_tool integrated from pose0 over the actions (Sec. 4.2).
 * SIM_E_STATE if the tool is disabled, SIM_E_ARG for a bad scene or step. */
sim_status sim_get_tool_pose(sim_h h, int scene, int step, float* pose, int on_device);

/* Loss seeds. Every seeding call below adds to the seeds of the state at one
 * step t, 1 <= t <= the current step (step = -1: the current step), which
 * sim_backward propagates together: a loss summed over the trajectory (App.
 * C: L = sum_t CD(s_t, s*_t)) takes one call per term and one backward pass.
 * Seeds need checkpointing (SIM_E_STATE otherwise, before the first step, or
 * for a step outside [1, current]); seeds of several calls at one step add up.
 * sim_set_particles / sim_set_state / sim_set_tool drop pending seeds. */

/* Add caller-computed loss gradients dL/dx, dL/dv (either may be NULL) with
 * respect to the state at step `step` (caller order). Accumulates. */
sim_status sim_add_loss_grad(sim_h h, int scene, int step, const float* dLdx, const float* dLdv,
                             int on_device);

/* As sim_add_loss_grad, with the affine velocity's gradient dLdC [n][3][3]
 * (row-major) as well; any of the three may be NULL. */
sim_status sim_add_state_grad(sim_h h, int scene, int step, const float* dLdx, const float* dLdv,
                              const float* dLdC, int on_device);

/* Point-goal loss of App. C in its squared form, on the state at step `step`
 * (-1 or the current step, or a checkpoint step before it, whose state the
 * trajectory keeps; other steps: SIM_E_STATE):
 * L_s = weight * sum_p |x_p - target|^2 per scene; writes L_s to loss_out
 * (host, one double per addressed scene) and accumulates dL/dx into the
 * seeds of that step. */
sim_status sim_position_loss(sim_h h, int scene, int step, const float* target, float weight,
                             double* loss_out);

/* Chamfer-style grid-mass loss (grid analogue of App. C's Chamfer loss) on the
 * state at step `step` (steps as for sim_position_loss): with m the P2G mass
 * field of the particles, L = sum_i (m_i - m*_i)^2 / M^2 + sum_i m_i d*_i / M,
 * M = total_mass. target_mass, target_dist: [grid_n^3] flattened (i, j, k)
 * row-major for the one addressed scene (scene >= 0). Writes L to *loss_out and
 * accumulates dL/dx into the seeds of that step. */
sim_status sim_grid_mass_loss(sim_h h, int scene, int step, const float* target_mass,
                              const float* target_dist, float total_mass, int on_device,
                              double* loss_out);

/* Attraction loss (Sec. 5.1), the paper's practical stand-in for sharing
 * gradients within a fluid body, on the positions of the current step:
 *   L_att = weight * sum_a sum_{j != a} c_j phi(|x_a - x_j|),
 *   c_j = exp(-ell_j / tau),  phi(d) = d k(d / radius),
 *   k(r) = (1 - r^2)^3 for r < 1, else 0,
 * over the pairs of particles of one scene at a nonzero distance (the kernel
 * c_j k is this library's reading of the paper's w(L_j, d_ij): neighbours
 * with a lower previous loss attract more). scene = -1 addresses every scene
 * (pairs never cross scenes). ell: the particles' losses of the previous
 * iteration, [count] in caller order for the addressed range (on_device
 * selects device or host memory); 0 < radius <= 1 / grid_n; tau > 0. Writes
 * L_att to *loss_out (host) and accumulates weight * dL_att/dx into the seeds
 * of the current step. SIM_E_STATE without checkpointing or before a step. */
sim_status sim_attraction_loss(sim_h h, int scene, const float* ell, float radius, float tau,
                               float weight, int on_device, double* loss_out);

/* Gradient sharing (Sec. 5.1) on the positions of the current step: for each
 * addressed particle a, out_a = sum_j c_j k(|x_a - x_j| / radius) g_j over the
 * addressed particles j of a's scene within the radius, a itself included
 * (k(0) = 1); c_j, k, ell, radius, tau as in sim_attraction_loss.
 * g, out: [count][3] in caller order for the addressed range, distinct
 * buffers. Works with or without checkpointing. */
sim_status sim_share_gradients(sim_h h, int scene, const float* ell, float radius, float tau,
                               const float* g, float* out, int on_device);

/* Reverse-mode sweep over the whole trajectory since sim_set_particles using
 * the loss seeds of every step (checkpoints + forward recompute every
 * checkpoint_every steps, App. A); each step's seeds join the adjoint state
 * when the sweep reaches that step. Outputs (any may be NULL), concatenated
 * over scenes in caller order: dLdx0, dLdv0 [N*3]; dLdactions [n_scenes *
 * n_actions * 6]. Consumes and clears the seeds. SIM_E_STATE if checkpointing
 * is off or no step was taken. */
sim_status sim_backward(sim_h h, float* dLdx0, float* dLdv0, float* dLdactions, int on_device);

/* Wait for all enqueued work; returns deferred device errors. */
sim_status sim_sync(sim_h h);

/* Message of the last failing call on this handle (static text if h is NULL). */
const char* sim_last_error(sim_h h);

/* The grid-mass loss of sim_grid_mass_loss as a function of caller buffers
 * only, allocating no device memory. The paper has no counterpart of this
 * entry point. It is for callers that cannot call cudaMalloc: an application
 * whose device memory all belongs to its own pool, a real-time control loop
 * that must not enter the driver's allocator (which can block), a process
 * under a hard device-memory cap. Its only working memory is one file-scope
 * device array of 2 MiB + 256 B, held by every device that loads the library
 * until the process exits; grid_n may not exceed 64 (larger: SIM_E_ARG).
 * x [n_particles*3] (row-major), mass [n_particles], target_mass and
 * target_dist [grid_n^3] (flattened (i, j, k) row-major), dLdx
 * [n_particles*3] (overwritten with dL/dx), loss [1 double]: all device
 * pointers on the current device. Work is enqueued on cuda_stream (NULL = the
 * default stream) and the call returns without waiting. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and keeps
 * it for the process; make that first call before any stream capture, and do
 * not use this entry point after a cudaDeviceReset of that device (the array
 * may move, the kept address would not). Every call shares the array and
 * clears what must start at zero before using it; calls whose work overlaps on
 * the GPU (other streams, other host threads) race, so serialise them. A
 * particle whose stencil leaves the grid uses the nearest in-grid stencil and
 * no error is reported. Errors: SIM_E_ARG (sizes, null pointers), SIM_E_CUDA
 * (device lookup or launch failure, or a CUDA error already pending on entry:
 * then nothing is launched and the pending error is left for the caller to
 * read). */
sim_status sim_grid_mass_loss_static(const float* x, const float* mass, int n_particles,
                                     int grid_n, const float* target_mass,
                                     const float* target_dist, float total_mass, float* dLdx,
                                     double* loss, void* cuda_stream);

/* Per-kernel timing with CUDA events on the simulation stream. enable = 1
 * starts recording (and clears earlier records), 0 stops. */
sim_status sim_profile_enable(sim_h h, int enable);

/* Read recorded timings: for up to `cap` kernel names, fills names (pointers to
 * static strings), total milliseconds and launch counts; *n_out = number of
 * distinct kernels recorded. Synchronises. */
sim_status sim_profile_read(sim_h h, int cap, const char** names, double* total_ms,
                            long long* launches, int* n_out);

/* Number of kernels this handle has launched since it was created (every
 * kernel of every call; memset/memcpy operations are not counted). */
long long sim_kernel_launches(sim_h h);

/* Choose launch shapes for this handle by timing candidates on its current
 * scene: particles per CTA of the two scatter kernels (128 or 256), threads
 * per CTA of the gather kernels (128, 256, 512), grid blocks per CTA of the
 * grid kernels (1, 2, 4), with checkpoints whether the P2G adjoint of step n
 * runs fused with the G2P adjoint of step n - 1 (0, 1), whether the forward's
 * steps between two re-sorts run as one persistent launch (0, 1; on devices
 * with cooperative launches and without rigid materials), whether the fused
 * G2P stages each CTA's box of grid velocities in shared memory with one
 * tensor-copy (TMA) load (0, 1), how many 256-thread CTAs of the fused step
 * and the G2P adjoint each SM holds (3 at 80 registers, 4 at 64) and, without
 * checkpoints, the re-sort period (4, 8, 16, 32 steps). Each candidate runs n_steps steps (0 = 10; at most
 * max_steps when checkpointing or a tool is on), plus the reverse sweep in
 * gradient mode, with CUDA events around the kernels it affects. The choice
 * is cached per (GPU, particle count, scenes, grid, checkpoint interval) for
 * the process. The trajectory is restarted from the initial state (pending
 * loss gradients are not allowed). choices (nullable, 8 ints) receives the
 * scatter threads, gather threads, grid blocks per CTA, re-sort period,
 * adjoint fusion flag, persistent-forward flag, staged-gather flag and
 * scatter CTAs per SM.
 *
 * Persistent forward (the batched many-scene launch; no paper counterpart):
 * the steps of one run between re-sorts are one cooperative launch with one
 * set of CTAs resident on every SM. Per step, the CTAs take tiles of
 * particles from a counter for the fused G2P -> constitutive -> P2G phase,
 * meet at a grid-wide barrier, update the step's active grid blocks, and meet
 * again. Every barrier wait is bounded (5 s): a wait that runs out makes the
 * step report SIM_E_TIMEOUT, never a hang. The backward's recompute keeps the
 * per-step kernels (it shares the GPU with the reverse sweep). */
sim_status sim_autotune(sim_h h, int n_steps, int* choices);

/* Set the launch shapes directly (same 8 values as sim_autotune returns).
 * Unsupported values (or the persistent forward on a device without
 * cooperative launches): SIM_E_ARG. Drops the handle's captured graphs. */
sim_status sim_set_launch(sim_h h, const int* choices);

/* Self-test of the persistent forward's grid-wide barrier (no paper
 * counterpart): `blocks` CTAs of 64 threads, launched cooperatively on the
 * current device, meet at `rounds` barriers that each wait for
 * blocks + extra_arrivals arrivals, every wait bounded by timeout_ms.
 * extra_arrivals = 0: every barrier completes, *passed = blocks * rounds,
 * SIM_OK. extra_arrivals > 0: no barrier can complete; each CTA gives up
 * after timeout_ms and returns, *passed = 0, SIM_E_TIMEOUT, and the CUDA
 * context stays usable. Allocates and frees 16 bytes of device memory;
 * synchronises the device. SIM_E_ARG for blocks outside [1, 4096] (or more
 * than the device holds at once: SIM_E_CUDA), rounds < 1 or a timeout outside
 * (0, 60000] ms. */
sim_status sim_selftest_grid_barrier(int blocks, int extra_arrivals, int rounds, double timeout_ms,
                                     int* passed);

/* Library build identification (static string). */
const char* sim_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MPM_SIM_H */
