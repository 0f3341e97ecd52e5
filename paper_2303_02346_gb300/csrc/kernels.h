// Host-side launchers of the library's kernels (internal interface between the
// C-ABI implementation and the .cu files that hold the kernels).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace mpm {

// Device pointers of one particle-state buffer (SoA, kStateFields * N floats).
struct StateView {
  float* st;        // field f of particle p at st[f * N + p]
  uint32_t* tag;    // material | scene << 8
};

struct GridBuffers {
  float4* acc;      // P2G accumulator (m, mvx, mvy, mvz); zero outside a step
  float4* gv;       // node velocity after the update (vx, vy, vz, m)
  float4* gstore;   // optional: (u_x, u_y, u_z, m) before contact, kept for the adjoint
  int* flags;       // active-block flags (zero outside a step)
  int* list;        // active-block list
  int* count;       // number of entries in list
  float* Fp;        // projected F of solids (9 x N), written by P2G, read by G2P
  float* svd;       // optional: SVD of the trial F of solids (21 x N: U, sigma, V)
  // optional compact copy of gv for the adjoint: the grid update also writes
  // the 64 nodes of list entry e at cgv[64 e ..] for e < cap, and sets
  // ovf_bit in *ovf when the step's list has more entries than that
  float4* cgv = nullptr;
  int cap = 0;
  int* ovf = nullptr;
  int ovf_bit = 0;
};

// Launch shapes chosen by the autotuner (sim_autotune).
struct Tuning {
  int scatter_threads = 256;  // p2g / g2p_adj: 128 or 256 particles per CTA
  int gather_threads = 256;   // g2p / p2g_adj: 128, 256 or 512 threads per CTA
  int grid_blocks = 4;        // grid_update / grid_adj: 1, 2 or 4 grid blocks (64 threads each) per CTA
  int fuse_adjoint = 0;       // 1: P2G adjoint of step n fused with the G2P adjoint of step n - 1
  int persistent = 0;         // 1: forward runs between re-sorts as one persistent cooperative launch
  int stage_gather = 0;       // 1: fused G2P stages each CTA's grid box in shared memory by a TMA load
  int scatter_ctas = 3;       // resident 256-thread CTAs per SM of the fused step and G2P adjoint (3 or 4)
};

// Carve the SM's unified L1 / shared memory out at its largest shared part
// for `kernel` (once per kernel): the 4-CTA builds of the scatter kernels need it.
void max_shared_carveout(const void* kernel);

// forward step stages
// reset_count (nullable): an active-block counter to zero for the next step
void launch_p2g(const Params& P, const Tuning& tu, const float* st_in, const uint32_t* tag, GridBuffers g,
                int* reset_count, int* err, cudaStream_t s);
// G2P of step n - 1 (reads Fp_prev, gv_prev, writes st_out) fused with P2G of
// step n into the buffers of g. lean: st_out receives only x and a liquid's J
// (enough for another fused step; v, C and a solid's trial F are left stale);
// otherwise x, v, C and field 15 (the fields a recomputed state needs: st_out
// may be a 16-field slot)
// gvmap (nullable): tensor map of gv_prev (encode_grid_map); with it and
// tu.stage_gather the kernel stages each CTA's grid box by a TMA load
void launch_g2p2g(const Params& P, const Tuning& tu, const float* st_in, float* st_out, const uint32_t* tag,
                  const float* Fp_prev, const float4* gv_prev, GridBuffers g, int* reset_count, int* err,
                  cudaStream_t s, bool lean = false, const CUtensorMap* gvmap = nullptr);
// Tiled tensor map of a grid buffer for the staged gather; false if the
// driver's encoder is unavailable or refuses the layout.
bool encode_grid_map(const Params& P, const float4* grid, CUtensorMap* out);
void launch_grid_update(const Params& P, const Tuning& tu, GridBuffers g, const float* tool_pose, int step,
                        int max_steps, cudaStream_t s);
void launch_g2p(const Params& P, const Tuning& tu, const float* st_in, float* st_out, const uint32_t* tag,
                const float* Fp, const float4* gv, int* err, cudaStream_t s);
// Persistent forward of steps [n0, n1) in one cooperative launch (one CTA set
// resident per SM): P2G of step n0 from src, fused G2P -> P2G (lean, into W)
// for the later steps, each particle phase followed by the step's grid update
// behind grid-wide barriers (bounded waits: kErrTimeout in err). lists: the
// two active-block lists (parity 0, 1) list_stride apart; count: their two
// counters; tile_ctr: 2 ints, bar: 2 unsigned of scratch. The G2P of step
// n1 - 1 is left to the caller. Returns the launch's error (e.g. cooperative
// launch unsupported), in which case nothing ran.
cudaError_t launch_forward_run(const Params& P, const Tuning& tu, const float* src, float* W, const uint32_t* tag,
                               GridBuffers g, int* lists, long long list_stride, int* count, const float* pose,
                               int n0, int n1, int max_steps, int* tile_ctr, unsigned* bar, int* err,
                               cudaStream_t s);
// `rounds` grid barriers among `blocks` CTAs of 64 threads that expect
// `expected` arrivals each; *passed counts the barriers CTAs got through.
cudaError_t launch_barrier_selftest(unsigned* bar, int blocks, unsigned expected, int rounds, int* err,
                                    unsigned long long timeout_ns, int* passed, cudaStream_t s);

// sorting of particles into grid blocks
struct SortBuffers {
  uint32_t* key;   // N
  uint32_t* rank;  // N
  uint32_t* bins;  // 2 n_bins + 1 (the particle sort keys water and the other materials apart)
  uint32_t* tile_sums;
  int n_bins;      // scenes x Morton codes per scene
};
// Sort by (class: water first, scene, Morton code of the stencil-origin cell)
void launch_sort(const Params& P, const float* st_in, const uint32_t* tag_in, const int* pid_in,
                 float* st_out, uint32_t* tag_out, int* pid_out, SortBuffers sb, cudaStream_t s);
// water particles among the tags into *out (device int)
void launch_count_water(const Params& P, const uint32_t* tag, int* out, cudaStream_t s);

// permutations between the library's particle order and the caller's
void launch_gather_rows(const float* src, float* dst, const int* pid, int N, int fields,
                        int field_stride_src, int field_stride_dst, int to_caller, cudaStream_t s);

// tool kinematics
void launch_tool_forward(const Params& P, const float* pose0, const float* actions, int n_actions,
                         int spa, int n_steps, int max_steps, float* poses, cudaStream_t s);
void launch_tool_backward(const Params& P, const float* pose0, const float* actions, int n_actions,
                          int spa, int n_steps, int max_steps, const float* poses,
                          const float* tool_grad, float* action_grad, cudaStream_t s);

// adjoint stages
// Fp_n / svd_n: the projected F and the SVD of the trial F stored by the
// recompute of step n
void launch_g2p_adj(const Params& P, const Tuning& tu, const float* st_n, const float* st_n1,
                    const uint32_t* tag, const float* Fp_n, float* adj, const float4* gv, float4* gadj_v,
                    cudaStream_t s);
void launch_grid_adj(const Params& P, const Tuning& tu, GridBuffers g, float4* gadj_v, float4* gadj_m,
                     const float* tool_pose, float* tool_grad, int step, int max_steps,
                     cudaStream_t s);
// adjoint of P2G of step n fused with the adjoint of G2P of step n - 1
void launch_adj_fused(const Params& P, const Tuning& tu, const float* st_prev, const float* st_n,
                      const float* st_n1, const uint32_t* tag, const float* svd_n, const float* Fp_prev,
                      float* adj, const float4* gadj_m, const float4* gv_prev, float4* gadj_v,
                      cudaStream_t s);
void launch_p2g_adj(const Params& P, const Tuning& tu, const float* st_n, const float* st_n1,
                    const uint32_t* tag, const float* svd_n, float* adj, const float4* gadj_m,
                    cudaStream_t s);
void launch_clear_blocks(const Params& P, float4* grid, const int* list, const int* count,
                         cudaStream_t s);
// Write the compact copy g.cgv of a step's grid values (its first min(count,
// cap) list entries) into the full-size grid gv; nodes of other blocks keep
// what they hold.
void launch_expand_grid(const Params& P, GridBuffers g, float4* gv, cudaStream_t s);

// losses
void launch_position_loss(const Params& P, const float* st, const uint32_t* tag, int scene,
                          float tx, float ty, float tz, float w, float* adj, double* loss,
                          cudaStream_t s);
void launch_mass_scatter(const Params& P, const float* st, const uint32_t* tag, int scene,
                         float* mgrid, cudaStream_t s);
void launch_mass_loss_nodes(long long n3, const float* mgrid, const float* tm, const float* td,
                            float inv_M, float* dLdm, double* loss, cudaStream_t s);
void launch_mass_loss_grad(const Params& P, const float* st, const uint32_t* tag, int scene,
                           const float* dLdm, float* adj, cudaStream_t s);

// misc
// streaming multiprocessors of the current device (queried once per device);
// grid-stride kernels size their grids as a multiple of it
int sm_count();
void launch_init_state(float* st, int N, cudaStream_t s);
void launch_init_particles(float* X0, uint32_t* tag0, const uint8_t* mat, int lo, int cnt, int N,
                           int n_mat, int* err, cudaStream_t s);
void launch_iota(int* a, int N, cudaStream_t s);
// dst[i] += src[i] for i < n; with clear_src also src[i] = 0
void launch_add_fields(float* dst, float* src, long long n, int clear_src, cudaStream_t s);
void launch_add_seed(float* adj_field, const float* seed, const int* pid, const uint32_t* tag, int scene,
                     int lo, int count, int N, cudaStream_t s, int ncomp = 3);

}  // namespace mpm
