// Forward MLS-MPM step kernels: constitutive prologue + P2G scatter, active
// block compaction, grid update (gravity, tool contact, sticky walls), G2P
// gather with the deformation-gradient update.
//
// Paper Sec. 3.2 (MLS-MPM, Hu et al. 2018): stress enters in P2G, boundary
// conditions and SDF contact in the grid operations. One step n -> n+1:
//   (F_p, tau) = Phi(F_trial); A = -dt V_p (4/dx^2) tau + m_p C_p;
//   m_i += W m_p;  mv_i += W (m_p v_p + A (x_i - x_p));
//   u_i = mv_i / m_i + dt g; contact; sticky walls;
//   v_p = sum W v_i; C_p = (4/dx^2) sum W v_i (x_i - x_p)^T; x_p += dt v_p;
//   F_trial <- (I + dt C_p) F_p   (liquid: J <- J det(I + dt C_p)).
#include <cuda.h>  // CUtensorMap (encoded through the runtime's driver entry point)

#include <cstring>

#include "common.cuh"
#include "constitutive.cuh"
#include "kernels.h"
#include "scatter.cuh"
#include "sur_ptx.cuh"
#include "tool.cuh"

namespace mpm {

// field offsets in the SoA state
constexpr int fX = 0, fV = 3, fC = 6, fF = 15;

// ---------------------------------------------------------------------------
// P2G of one particle from its state in registers: constitutive prologue
// (writes F_p and, if requested, the SVD of the trial F), affine matrix A and
// stencil. F holds the trial F (solids) or J in F[0] (liquid).
// ---------------------------------------------------------------------------
template <bool kExt>
__device__ inline void p2g_prologue(const Params& P, int p, const MatParams& M, const float* x,
                                    const float* C, const float* F, float* __restrict__ Fp_out,
                                    float* __restrict__ svd_out, int* __restrict__ err, float* A,
                                    Stencil& sc) {
  const int N = P.N;
  float tau[9];
  if (kExt && M.kind == kViscousLiquid) {
    // the trial F of the step: the reset J_n^(1/3) I of the previous step
    // advanced by G = I + dt C, i.e. (J / det G)^(1/3) G with J = J_n det G;
    // fixed-corotated stress of it (the reset drops it after this step)
    float G[9], Ft[9], Fp[9], usv[21];
#pragma unroll
    for (int k = 0; k < 9; ++k) G[k] = ((k % 4 == 0) ? 1.0f : 0.0f) + P.dt * C[k];
    const float a = cbrtf(F[0] / det3(G));
#pragma unroll
    for (int k = 0; k < 9; ++k) Ft[k] = a * G[k];
    solid_forward<kExt>(M, Ft, Fp, tau, usv);
    if (svd_out) {
#pragma unroll
      for (int k = 0; k < 21; ++k) svd_out[sslot(P, k, p)] = usv[k];
    }
  } else if (kExt && M.kind == kRigid) {
    // F is the object's rotation (set by the rigidity projection), where the
    // corotated stress vanishes: tau = 0, F_p = F
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      tau[k] = 0.0f;
      Fp_out[sslot(P, k, p)] = F[k];
    }
  } else if (M.kind == kLiquid) {
    const float J = F[0];
    const float pr = M.lam * J * (J - 1.0f);
#pragma unroll
    for (int k = 0; k < 9; ++k) tau[k] = (k % 4 == 0) ? pr : 0.0f;
  } else {
    float Fp[9], usv[21];
    solid_forward<kExt>(M, F, Fp, tau, usv);
#pragma unroll
    for (int k = 0; k < 9; ++k) Fp_out[sslot(P, k, p)] = Fp[k];
    if (svd_out) {
#pragma unroll
      for (int k = 0; k < 21; ++k) svd_out[sslot(P, k, p)] = usv[k];
    }
  }
  const float coef = -P.dt * M.vol * 4.0f * P.inv_dx * P.inv_dx;
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = coef * tau[k] + M.mass * C[k];
  if (!make_stencil(x, P, sc)) atomicOr(err, kErrDomain);
}

// Block-level scatter of the CTA's particles (every thread must call it).
template <int NT>
__device__ inline void p2g_scatter(ScatterTile<NT>& T, const Params& P, bool valid, int scene,
                                   const Stencil& sc, float m, const float* v, const float* A,
                                   float4* __restrict__ acc, int* __restrict__ flags,
                                   int* __restrict__ list, int* __restrict__ count) {
  scatter_setup(T, valid, sc.base, scene);
  if (T.box[7]) {
    // cell-binned tile: records sorted by cell, then per-(cell, o_x, o_y) accumulation
    const int rank = scatter_count(T, valid, sc.base);
    __syncthreads();
    scan_cells(T);
    if (valid) {
      const float mv[3] = {m * v[0], m * v[1], m * v[2]};
      scatter_record(T, rank, sc, m, mv, A, P.dx);
    }
    __syncthreads();
    scatter_accumulate<true, NT>(T);
  } else if (valid) {
    const float mv0 = m * v[0], mv1 = m * v[1], mv2 = m * v[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float da = (a - sc.f[0]) * P.dx;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float db = (b - sc.f[1]) * P.dx;
        const float wab = sc.w[0][a] * sc.w[1][b];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float dc = (c - sc.f[2]) * P.dx;
          const float W = wab * sc.w[2][c];
          const float q0 = mv0 + A[0] * da + A[1] * db + A[2] * dc;
          const float q1 = mv1 + A[3] * da + A[4] * db + A[5] * dc;
          const float q2 = mv2 + A[6] * da + A[7] * db + A[8] * dc;
          red_add_v4(acc + node_index(P, scene, sc.base[0] + a, sc.base[1] + b, sc.base[2] + c), W * m,
                     W * q0, W * q1, W * q2);
        }
      }
    }
    mark_stencil_blocks(P, scene, sc.base, flags, list, count);
  }
  scatter_flush(T, acc, P, flags, list, count);
}

// reset_count: the active-block counter of the other step parity (consumed by
// the previous grid update) is zeroed for the next step.
template <int NT, bool kExt>
__global__ void __launch_bounds__(NT)
p2g_kernel(Params P, const float* __restrict__ st, const uint32_t* __restrict__ tag,
           float* __restrict__ Fp_out, float* __restrict__ svd_out, float4* __restrict__ acc,
           int* __restrict__ flags, int* __restrict__ list, int* __restrict__ count,
           int* __restrict__ reset_count, int* __restrict__ err) {
  __shared__ ScatterTile<NT> T;
  const int N = P.N;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && reset_count) *reset_count = 0;
  const bool valid = p < N;
  float x[3] = {0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f}, A[9];
  float m = 0.0f;
  int scene = 0;
  Stencil sc;
  sc.base[0] = sc.base[1] = sc.base[2] = 0;
  if (valid) {
    float C[9], F[9];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      x[d] = st[(fX + d) * N + p];
      v[d] = st[(fV + d) * N + p];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) C[k] = st[(fC + k) * N + p];
    const uint32_t tg = tag[p];
    scene = tag_scene(tg);
    const MatParams& M = P.mat[tag_mat(tg)];
    m = M.mass;
    F[0] = st[fF * N + p];
    if (!is_liquid(M.kind)) {
#pragma unroll
      for (int k = 1; k < 9; ++k) F[k] = st[(fF + k) * N + p];
    }
    p2g_prologue<kExt>(P, p, M, x, C, F, Fp_out, svd_out, err, A, sc);
  }
  p2g_scatter<NT>(T, P, valid, scene, sc, m, v, A, acc, flags, list, count);
}

__device__ inline void node_of(const Params& P, int blk, int l, int& scene, int& i, int& j, int& k) {
  scene = blk / P.NB;
  int bl = blk - scene * P.NB;
  int bx = bl / (P.nb * P.nb), by = (bl / P.nb) % P.nb, bz = bl % P.nb;
  i = bx * kBlockEdge + (l >> 4);
  j = by * kBlockEdge + ((l >> 2) & 3);
  k = bz * kBlockEdge + (l & 3);
}

// 64 threads per active block; zeroes the accumulator after reading it. A
// group of 64 threads takes kGridItems blocks of the list at a time (strided by
// the grid's groups): their list entries and node accumulators are loaded
// before any of them is processed, so each thread keeps kGridItems independent
// load chains in flight instead of walking them one after the other.
// kTool: built with the tool contact. group / n_groups: this thread's group of
// 64 and the number of groups sharing the list.
constexpr int kGridItems = 4;
template <bool kTool>
__device__ inline void grid_update_items(const Params& P, float4* __restrict__ acc, float4* __restrict__ gv,
                                         float4* __restrict__ gstore, int* __restrict__ flags,
                                         const int* __restrict__ list, int cnt, const float* __restrict__ pose,
                                         int step, int max_steps, int group, int n_groups,
                                         float4* __restrict__ cgv = nullptr, int cap = 0, int* ovf = nullptr,
                                         int ovf_bit = 0) {
  const int l = threadIdx.x & 63;
  const int stride = n_groups;
  for (int item0 = group; item0 < cnt; item0 += stride * kGridItems) {
    int blk[kGridItems];
    float4 a[kGridItems];
    unsigned ok = 0u;  // bit u: node of item u inside the grid
#pragma unroll
    for (int u = 0; u < kGridItems; ++u) {
      const int item = item0 + u * stride;
      blk[u] = item < cnt ? list[item] : -1;
    }
#pragma unroll
    for (int u = 0; u < kGridItems; ++u) {
      if (blk[u] < 0) continue;
      int scene, i, j, k;
      node_of(P, blk[u], l, scene, i, j, k);
      if (i >= P.n || j >= P.n || k >= P.n) continue;
      ok |= 1u << u;
      a[u] = acc[node_index(P, scene, i, j, k)];
    }
#pragma unroll
    for (int u = 0; u < kGridItems; ++u) {
      if (l == 0 && blk[u] >= 0) flags[blk[u]] = 0;
      // compact copy: list entry `item` -> cgv[64 item + l]
      const int item = item0 + u * stride;
      const bool keep = cgv != nullptr && item < cap;
      if (cgv != nullptr && item >= cap && l == 0 && blk[u] >= 0) atomicOr(ovf, ovf_bit);
      if (!(ok & (1u << u))) continue;
      int scene, i, j, k;
      node_of(P, blk[u], l, scene, i, j, k);
      const long long idx = node_index(P, scene, i, j, k);
      acc[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (a[u].x > 0.0f) {
        float inv = 1.0f / a[u].x;
        float uu[3] = {a[u].y * inv + P.dt * P.g[0], a[u].z * inv + P.dt * P.g[1], a[u].w * inv + P.dt * P.g[2]};
        if (gstore) gstore[idx] = make_float4(uu[0], uu[1], uu[2], a[u].x);
        float vv[3] = {uu[0], uu[1], uu[2]};
        if (kTool) {
          ToolState T;
          load_tool(pose + ((long long)scene * max_steps + step) * kToolFields, T);
          float xi[3] = {i * P.dx, j * P.dx, k * P.dx};
          contact_forward(P, T, xi, vv);
        }
        bool wall = i < P.bound || j < P.bound || k < P.bound || i >= P.n - P.bound ||
                    j >= P.n - P.bound || k >= P.n - P.bound;
        if (wall) vv[0] = vv[1] = vv[2] = 0.0f;
        gv[idx] = make_float4(vv[0], vv[1], vv[2], a[u].x);
        if (keep) cgv[(long long)item * 64 + l] = make_float4(vv[0], vv[1], vv[2], a[u].x);
      } else {
        gv[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (keep) cgv[(long long)item * 64 + l] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gstore) gstore[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
}

template <bool kTool>
__global__ void __launch_bounds__(256)
grid_update_kernel(Params P, float4* __restrict__ acc, float4* __restrict__ gv,
                   float4* __restrict__ gstore, int* __restrict__ flags, const int* __restrict__ list,
                   const int* __restrict__ count, const float* __restrict__ pose, int step,
                   int max_steps, float4* __restrict__ cgv, int cap, int* __restrict__ ovf, int ovf_bit) {
  const int per = blockDim.x >> 6;
  grid_update_items<kTool>(P, acc, gv, gstore, flags, list, *count, pose, step, max_steps,
                           blockIdx.x * per + (threadIdx.x >> 6), gridDim.x * per, cgv, cap, ovf, ovf_bit);
}

// Compact copy of a step's grid values back into a full-size grid: list entry
// e's 64 nodes to their places, nodes outside the grid skipped.
__global__ void __launch_bounds__(256)
expand_grid_kernel(Params P, const float4* __restrict__ cgv, const int* __restrict__ list,
                   const int* __restrict__ count, int cap, float4* __restrict__ gv) {
  const long long n = (long long)min(*count, cap) * 64;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    int scene, i, j, k;
    node_of(P, list[t >> 6], int(t & 63), scene, i, j, k);
    if (i >= P.n || j >= P.n || k >= P.n) continue;
    gv[node_index(P, scene, i, j, k)] = cgv[t];
  }
}

__device__ inline bool in_domain(const float* x, const Params& P) {
  bool ok = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float bf = base_floor(grid_coord(x[d], P));
    ok = ok && (bf >= 0.0f) && (bf <= float(P.n - 3));
  }
  return ok;
}

// G2P of one particle: gathers the grid velocities of step n, updates x, v, C
// and the trial F (J for liquid), writes them to st_out and returns them in
// registers. kStore: kStoreFull writes x, v, C and the trial F (J for water);
// kStoreLean only x and a water particle's J (what the next fused step reads;
// another material's next step starts from the F_p its P2G writes), for
// forward steps whose v, C and trial F nobody reads; kStoreChunk x, v, C and
// field 15 (J, or F[0][0]), the fields the adjoint kernels read from a
// recomputed state (they take the other materials' trial F from the stored
// SVD), for states kept in 16-field slots.
// stage (nullable): the CTA's grid box of kStageBox^3 nodes in shared memory,
// with its origin node (so, oy, oz) in stage_org; the gather reads there
// once `stage_bar` has completed (bounded wait: on timeout the particle reads
// global memory and kErrTimeout is set).
constexpr int kStageBox = 8;
enum : int { kStoreFull = 0, kStoreLean = 1, kStoreChunk = 2 };
template <int kStore = kStoreFull, bool kNC = true>
__device__ inline void g2p_particle(const Params& P, int p, const MatParams& M, int scene,
                                    const float* __restrict__ st_in, float* __restrict__ st_out,
                                    const float* __restrict__ Fp_in, const float4* __restrict__ gv,
                                    int* __restrict__ err, float* xn, float* vn, float* C, float* Fn,
                                    const float4* stage = nullptr, const int* stage_org = nullptr,
                                    uint64_t* stage_bar = nullptr) {
  const int N = P.N;
  float x[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) x[d] = st_in[(fX + d) * N + p];
  Stencil sc;
  make_stencil(x, P, sc);
  // B = sum_o W v_o dpos^T with dpos = (o - f) dx for the stencil offset o:
  // B = dx (S - v f^T), S = sum_o W v_o o^T (integer o: zero terms drop out).
  // W = w0[a] w1[b] w2[c] factorises, so each (a, b) column of three nodes is
  // first reduced over c: t = sum_c w2[c] v, tc = sum_c c w2[c] v; then
  // v += wab t, S[:, 0] += a wab t, S[:, 1] += b wab t, S[:, 2] += wab tc.
  // The sums run on the lane pairs (x, y) and (z, w) of the node values with
  // packed two-lane FP32 instructions (the w lane is carried along unused):
  // vp[h] holds lanes h of v, Sp[j][h] lanes h of the column S[:, j].
  float2 vp[2], Sp[3][2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    vp[h] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < 3; ++j) Sp[j][h] = make_float2(0.0f, 0.0f);
  }
  const float2 w20 = make_float2(sc.w[2][0], sc.w[2][0]), w21 = make_float2(sc.w[2][1], sc.w[2][1]),
               w22 = make_float2(sc.w[2][2], sc.w[2][2]);
  const float2 w2c2 = make_float2(2.0f * sc.w[2][2], 2.0f * sc.w[2][2]);
  int srow = -1;  // staged: the particle's stencil origin in the box
  if (stage != nullptr) {
    if (sur::mbar_wait(stage_bar, 0, nullptr)) {
      const int r0 = sc.base[0] - stage_org[0], r1 = sc.base[1] - stage_org[1], r2 = sc.base[2] - stage_org[2];
      // the box covers every stencil of the CTA; a particle outside it (none
      // is expected) reads global memory
      if (r0 >= 0 && r1 >= 0 && r2 >= 0 && r0 <= kStageBox - 3 && r1 <= kStageBox - 3 && r2 <= kStageBox - 3)
        srow = (r0 * kStageBox + r1) * kStageBox + r2;
    } else {
      atomicOr(err, kErrTimeout);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      float4 g0, g1, g2;
      if (srow >= 0) {
        const float4* col = stage + srow + (a * kStageBox + b) * kStageBox;
        g0 = col[0];
        g1 = col[1];
        g2 = col[2];
      } else {
        const float4* col = gv + node_index(P, scene, sc.base[0] + a, sc.base[1] + b, sc.base[2]);
        // kNC: the read-only path; a kernel that wrote gv itself (the persistent
        // forward) reads it with coherent loads
        g0 = kNC ? __ldg(col) : col[0];
        g1 = kNC ? __ldg(col + 1) : col[1];
        g2 = kNC ? __ldg(col + 2) : col[2];
      }
      const float2 gp[3][2] = {{make_float2(g0.x, g0.y), make_float2(g0.z, g0.w)},
                               {make_float2(g1.x, g1.y), make_float2(g1.z, g1.w)},
                               {make_float2(g2.x, g2.y), make_float2(g2.z, g2.w)}};
      const float wab = sc.w[0][a] * sc.w[1][b];
      const float2 wab2 = make_float2(wab, wab);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 t = __ffma2_rn(w22, gp[2][h], __ffma2_rn(w21, gp[1][h], __fmul2_rn(w20, gp[0][h])));
        const float2 tc = __ffma2_rn(w2c2, gp[2][h], __fmul2_rn(w21, gp[1][h]));
        const float2 u = __fmul2_rn(wab2, t);
        vp[h] = __fadd2_rn(vp[h], u);
        if (a == 1) Sp[0][h] = __fadd2_rn(Sp[0][h], u);
        if (a == 2) Sp[0][h] = __ffma2_rn(make_float2(2.0f, 2.0f), u, Sp[0][h]);
        if (b == 1) Sp[1][h] = __fadd2_rn(Sp[1][h], u);
        if (b == 2) Sp[1][h] = __ffma2_rn(make_float2(2.0f, 2.0f), u, Sp[1][h]);
        Sp[2][h] = __ffma2_rn(wab2, tc, Sp[2][h]);
      }
    }
  }
  vn[0] = vp[0].x;
  vn[1] = vp[0].y;
  vn[2] = vp[1].x;
  float S[9];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    S[j] = Sp[j][0].x;
    S[3 + j] = Sp[j][0].y;
    S[6 + j] = Sp[j][1].x;
  }
  const float s4d = 4.0f * P.inv_dx * P.inv_dx * P.dx;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[3 * i + j] = s4d * (S[3 * i + j] - vn[i] * sc.f[j]);
#pragma unroll
  for (int d = 0; d < 3; ++d) xn[d] = x[d] + P.dt * vn[d];
  const bool fin = isfinite(xn[0]) && isfinite(xn[1]) && isfinite(xn[2]);
  if (!fin) atomicOr(err, kErrNaN);
  else if (!in_domain(xn, P)) atomicOr(err, kErrDomain);
  float G[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) G[k] = ((k % 4 == 0) ? 1.0f : 0.0f) + P.dt * C[k];
  if (is_liquid(M.kind)) {
    Fn[0] = st_in[fF * N + p] * det3(G);
    st_out[fF * N + p] = Fn[0];
  } else {
    float Fp[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Fp[k] = Fp_in[sslot(P, k, p)];
    mat_mul(G, Fp, Fn);
    if (kStore == kStoreFull) {
#pragma unroll
      for (int k = 0; k < 9; ++k) st_out[(fF + k) * N + p] = Fn[k];
    } else if (kStore == kStoreChunk) {
      st_out[fF * N + p] = Fn[0];
    }
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) st_out[(fX + d) * N + p] = xn[d];
  if (kStore != kStoreLean) {
#pragma unroll
    for (int d = 0; d < 3; ++d) st_out[(fV + d) * N + p] = vn[d];
#pragma unroll
    for (int k = 0; k < 9; ++k) st_out[(fC + k) * N + p] = C[k];
  }
}

__global__ void __launch_bounds__(512)
g2p_kernel(Params P, const float* __restrict__ st_in, float* __restrict__ st_out,
           const uint32_t* __restrict__ tag, const float* __restrict__ Fp_in,
           const float4* __restrict__ gv, int* __restrict__ err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.N) return;
  const uint32_t tg = tag[p];
  float x[3], v[3], C[9], F[9];
  g2p_particle(P, p, P.mat[tag_mat(tg)], tag_scene(tg), st_in, st_out, Fp_in, gv, err, x, v, C, F);
}

// Tensor-copy staging of the gather (kStage): the CTA reduces the bounding box
// of its particles' G2P stencil origins; if the box's nodes fit in
// kStageBox^3 and the particles share one scene, one thread issues a tiled
// TMA load of that box of the previous step's grid velocities into the
// scatter tile's accumulator storage (unused until the scatter), and the
// gathers read shared memory instead of issuing 27 global loads a particle.
template <int NT>
__device__ inline bool stage_gather_box(ScatterTile<NT>& T, const Params& P, const CUtensorMap* gvmap, bool valid,
                                        const float* x, int scene, int* org, uint64_t* bar) {
  int b[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float bf = base_floor(grid_coord(x[d], P));
    b[d] = valid ? int(fminf(fmaxf(bf, 0.0f), float(P.n - 3))) : 0;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const int v = d < 3 ? b[d] : scene;
    const int mn = __reduce_min_sync(0xffffffffu, valid ? v : INT_MAX);
    const int mx = __reduce_max_sync(0xffffffffu, valid ? v : INT_MIN);
    if (lane == 0) {
      T.red[0][d][wid] = mn;
      T.red[1][d][wid] = mx;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int mn[4], mx[4];
    for (int d = 0; d < 4; ++d) {
      mn[d] = INT_MAX;
      mx[d] = INT_MIN;
      for (int w = 0; w < NT / 32; ++w) {
        mn[d] = min(mn[d], T.red[0][d][w]);
        mx[d] = max(mx[d], T.red[1][d][w]);
      }
    }
    const bool fits = mn[3] != INT_MAX && mn[3] == mx[3] && mx[0] - mn[0] + 3 <= kStageBox &&
                      mx[1] - mn[1] + 3 <= kStageBox && mx[2] - mn[2] + 3 <= kStageBox;
    org[0] = mn[0];
    org[1] = mn[1];
    org[2] = mn[2];
    org[3] = fits ? 1 : 0;
    if (fits) {
      sur::mbar_init(bar, 1);
      sur::fence_barrier_init();
      sur::fence_proxy_async_smem();
      sur::mbar_arrive_expect_tx(bar, kStageBox * kStageBox * kStageBox * 16);
      asm volatile(
          "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(sur::smem_u32(&T.acc[0][0])),
          "l"(reinterpret_cast<uint64_t>(gvmap)), "r"(0), "r"(mn[2]), "r"(mn[1]), "r"(mn[0]), "r"(mn[3]),
          "r"(sur::smem_u32(bar))
          : "memory");
    }
  }
  __syncthreads();
  return org[3] != 0;
}

// G2P of step n - 1 fused with P2G of step n: the particle state of step n is
// written once and scattered from registers without being read back (kLean:
// only the part of it the next fused step reads; otherwise the 16 fields a
// recomputed state keeps).
// Registers as the compiler chooses them (80: 3 resident CTAs of 256 per SM)
// or, with kHigh, held to 64 for 4 CTAs
template <int NT, bool kExt, bool kLean, bool kStage, bool kHigh = false>
__global__ void __launch_bounds__(NT, kHigh ? kScatterResidentThreadsHigh / NT : 0)
g2p2g_kernel(Params P, const float* __restrict__ st_in, float* __restrict__ st_out,
             const uint32_t* __restrict__ tag, const float* __restrict__ Fp_prev,
             const float4* __restrict__ gv_prev, float* __restrict__ Fp_out,
             float* __restrict__ svd_out, float4* __restrict__ acc, int* __restrict__ flags,
             int* __restrict__ list, int* __restrict__ count, int* __restrict__ reset_count,
             int* __restrict__ err, const __grid_constant__ CUtensorMap gvmap) {
  __shared__ ScatterTile<NT> T;
  __shared__ uint64_t stage_bar;
  __shared__ int stage_org[4];
  const int N = P.N;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && reset_count) *reset_count = 0;
  const bool valid = p < N;
  bool staged = false;
  if (kStage) {
    float xs[3] = {0.f, 0.f, 0.f};
    int sc0 = 0;
    if (valid) {
#pragma unroll
      for (int d = 0; d < 3; ++d) xs[d] = st_in[(fX + d) * N + p];
      sc0 = tag_scene(tag[p]);
    }
    staged = stage_gather_box(T, P, &gvmap, valid, xs, sc0, stage_org, &stage_bar);
  }
  float x[3] = {0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f}, A[9];
  float m = 0.0f;
  int scene = 0;
  Stencil sc;
  sc.base[0] = sc.base[1] = sc.base[2] = 0;
  if (valid) {
    const uint32_t tg = tag[p];
    scene = tag_scene(tg);
    const MatParams& M = P.mat[tag_mat(tg)];
    m = M.mass;
    float C[9], F[9];
    g2p_particle<kLean ? kStoreLean : kStoreChunk>(P, p, M, scene, st_in, st_out, Fp_prev, gv_prev, err, x, v,
                                                  C, F,
                        staged ? reinterpret_cast<const float4*>(&T.acc[0][0]) : nullptr, stage_org,
                        &stage_bar);
    p2g_prologue<kExt>(P, p, M, x, C, F, Fp_out, svd_out, err, A, sc);
  }
  p2g_scatter<NT>(T, P, valid, scene, sc, m, v, A, acc, flags, list, count);
}

// ---------------------------------------------------------------------------
// Persistent forward: the steps [n0, n1) between two re-sorts in one
// cooperative launch. Step n0 is a P2G of the state in src; every later step
// is the fused G2P of step n - 1 and P2G of step n (its state written to W,
// lean: x and a liquid's J). Each step's particle phase (CTAs take tiles of NT
// particles from a counter) is followed by a grid-wide barrier, the grid
// update of the step over its active blocks (all CTAs), and another barrier.
// The G2P after the last step is left to the caller.
// ---------------------------------------------------------------------------
__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch (every CTA resident). bar[0]
// counts arrivals and bar[1] is the generation, both zero at launch; the last
// of `expected` CTAs to arrive resets the count and advances the generation.
// Arrival is a release and the wait an acquire at GPU scope, so every CTA's
// writes before the barrier are visible to every CTA after it. The wait is
// bounded: after timeout_ns the CTA sets kErrTimeout in err and the function
// returns false (its caller returns; a CTA still waiting for it times out in
// turn), never hangs.
__device__ inline bool grid_barrier(unsigned* bar, unsigned expected, int* err,
                                    unsigned long long timeout_ns) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    unsigned g;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(bar + 1) : "memory");
    unsigned arrived;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
    if (arrived + 1u == expected) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
    } else {
      const unsigned long long t0 = global_ns();
      unsigned cur = g;
      while (cur == g) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(bar + 1) : "memory");
        if (cur != g) break;
        if (global_ns() - t0 > timeout_ns) {
          atomicOr(err, kErrTimeout);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
  }
  return __syncthreads_and(ok) != 0;
}

// One tile of NT particles of a persistent run's particle phase (every thread
// of the CTA calls it): mode 0 = P2G of the state in src, 1 = fused G2P -> P2G
// reading src and writing W, 2 = the same in place on W. Kept out of line so
// that its registers are allocated as in the per-step fused kernel, apart
// from the run's loop state.
template <int NT, bool kExt>
__device__ __noinline__ void forward_tile(ScatterTile<NT>& T, const Params& P, int tile, int mode, const float* src,
                                          float* W, const uint32_t* __restrict__ tag, float* Fp, float4* acc,
                                          const float4* gv, int* flags, int* list, int* count, int* err) {
  const int N = P.N;
  const int p = tile * NT + threadIdx.x;
  const bool valid = p < N;
  float x[3] = {0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f}, A[9];
  float m = 0.0f;
  int scene = 0;
  Stencil sc;
  sc.base[0] = sc.base[1] = sc.base[2] = 0;
  if (valid) {
    const uint32_t tg = tag[p];
    scene = tag_scene(tg);
    const MatParams& M = P.mat[tag_mat(tg)];
    m = M.mass;
    float C[9], F[9];
    if (mode == 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        x[d] = src[(fX + d) * N + p];
        v[d] = src[(fV + d) * N + p];
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) C[k] = src[(fC + k) * N + p];
      F[0] = src[fF * N + p];
      if (!is_liquid(M.kind)) {
#pragma unroll
        for (int k = 1; k < 9; ++k) F[k] = src[(fF + k) * N + p];
      }
    } else {
      g2p_particle<kStoreLean, false>(P, p, M, scene, mode == 1 ? src : W, W, Fp, gv, err, x, v, C, F);
    }
    p2g_prologue<kExt>(P, p, M, x, C, F, Fp, nullptr, err, A, sc);
  }
  p2g_scatter<NT>(T, P, valid, scene, sc, m, v, A, acc, flags, list, count);
}

// held to the fused step kernel's residency (3 CTAs of 256 per SM)
template <int NT, bool kExt, bool kTool>
__global__ void __launch_bounds__(NT, kScatterResidentThreads / NT)
forward_run_kernel(Params P, const float* src, float* W, const uint32_t* __restrict__ tag, float* Fp,
                   float4* acc, float4* gv, int* flags, int* lists, long long list_stride, int* count,
                   const float* __restrict__ pose, int n0, int n1, int max_steps, int* tile_ctr, unsigned* bar,
                   int* err, unsigned long long timeout_ns) {
  __shared__ ScatterTile<NT> T;
  __shared__ int tile_sh[2];
  const int ntiles = (P.N + NT - 1) / NT;
  for (int n = n0; n < n1; ++n) {
    const int q = n & 1;
    int* list = lists + q * list_stride;
    // the other parity's counters were last used by step n - 1, whose phases
    // ended at the barriers before this step
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      count[q ^ 1] = 0;
      tile_ctr[q ^ 1] = 0;
    }
    // tiles from the counter; thread 0 fetches the next tile's index while the
    // CTA works on the current one (the tile's own barriers publish it)
    if (threadIdx.x == 0) tile_sh[0] = atomicAdd(tile_ctr + q, 1);
    __syncthreads();
    for (int it = 0;; ++it) {
      const int tile = tile_sh[it & 1];
      if (tile >= ntiles) break;
      if (threadIdx.x == 0) tile_sh[(it + 1) & 1] = atomicAdd(tile_ctr + q, 1);
      forward_tile<NT, kExt>(T, P, tile, n == n0 ? 0 : (n == n0 + 1 ? 1 : 2), src, W, tag, Fp, acc, gv, flags,
                             list, count + q, err);
    }
    if (!grid_barrier(bar, gridDim.x, err, timeout_ns)) return;
    int cnt;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(cnt) : "l"(count + q) : "memory");
    grid_update_items<kTool>(P, acc, gv, nullptr, flags, list, cnt, pose, n, max_steps,
                             blockIdx.x * (NT >> 6) + (threadIdx.x >> 6), gridDim.x * (NT >> 6));
    if (n + 1 < n1 && !grid_barrier(bar, gridDim.x, err, timeout_ns)) return;
  }
}

// Self-test of the barrier's bound: `rounds` barriers among the launch's CTAs
// that wait for `expected` arrivals (more than the CTAs launched: none
// completes, every CTA times out and returns).
__global__ void barrier_selftest_kernel(unsigned* bar, unsigned expected, int rounds, int* err,
                                        unsigned long long timeout_ns, int* passed) {
  for (int r = 0; r < rounds; ++r) {
    if (!grid_barrier(bar, expected, err, timeout_ns)) return;
    if (threadIdx.x == 0) atomicAdd(passed, 1);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline int blocks_for(long long n, int t) { return int((n + t - 1) / t); }

void launch_p2g(const Params& P, const Tuning& tu, const float* st_in, const uint32_t* tag, GridBuffers g,
                int* reset_count, int* err, cudaStream_t s) {
  if (P.N == 0) {
    if (reset_count) cudaMemsetAsync(reset_count, 0, sizeof(int), s);
    return;
  }
  auto k = tu.scatter_threads == 128 ? (P.ext ? p2g_kernel<128, true> : p2g_kernel<128, false>)
                                     : (P.ext ? p2g_kernel<256, true> : p2g_kernel<256, false>);
  const int nt = tu.scatter_threads == 128 ? 128 : 256;
  k<<<blocks_for(P.N, nt), nt, 0, s>>>(P, st_in, tag, g.Fp, g.svd, g.acc, g.flags, g.list, g.count, reset_count,
                                       err);
}

template <bool kLean, bool kStage>
static auto g2p2g_variant(const Params& P, const Tuning& tu) {
  if (tu.scatter_threads == 128)
    return P.ext ? g2p2g_kernel<128, true, kLean, kStage> : g2p2g_kernel<128, false, kLean, kStage>;
  if (tu.scatter_ctas == 4)
    return P.ext ? g2p2g_kernel<256, true, kLean, kStage, true> : g2p2g_kernel<256, false, kLean, kStage, true>;
  return P.ext ? g2p2g_kernel<256, true, kLean, kStage> : g2p2g_kernel<256, false, kLean, kStage>;
}

void launch_g2p2g(const Params& P, const Tuning& tu, const float* st_in, float* st_out, const uint32_t* tag,
                  const float* Fp_prev, const float4* gv_prev, GridBuffers g, int* reset_count, int* err,
                  cudaStream_t s, bool lean, const CUtensorMap* gvmap) {
  if (P.N == 0) {
    if (reset_count) cudaMemsetAsync(reset_count, 0, sizeof(int), s);
    return;
  }
  const bool stage = gvmap != nullptr && tu.stage_gather;
  auto k = lean ? (stage ? g2p2g_variant<true, true>(P, tu) : g2p2g_variant<true, false>(P, tu))
                : (stage ? g2p2g_variant<false, true>(P, tu) : g2p2g_variant<false, false>(P, tu));
  const int nt = tu.scatter_threads == 128 ? 128 : 256;
  if (nt == 256 && tu.scatter_ctas == 4) max_shared_carveout(reinterpret_cast<const void*>(k));
  CUtensorMap none;
  std::memset(&none, 0, sizeof(none));
  k<<<blocks_for(P.N, nt), nt, 0, s>>>(P, st_in, st_out, tag, Fp_prev, gv_prev, g.Fp, g.svd, g.acc, g.flags,
                                       g.list, g.count, reset_count, err, stage ? *gvmap : none);
}

// Tiled tensor map over a grid of float4 nodes (scenes x n^3, node (i, j, k)
// at ((scene n + i) n + j) n + k) with kStageBox^3-node boxes, for the staged
// gather. The encode function is the driver's, found through the runtime.
bool encode_grid_map(const Params& P, const float4* grid, CUtensorMap* out) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  const cuuint64_t n = (cuuint64_t)P.n;
  const cuuint64_t dims[5] = {4, n, n, n, (cuuint64_t)P.S};
  const cuuint64_t strides[4] = {16, 16 * n, 16 * n * n, 16 * n * n * n};
  const cuuint32_t box[5] = {4, kStageBox, kStageBox, kStageBox, 1};
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<float4*>(grid), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Resident CTAs of 256 threads per SM of a grid-update variant (queried once).
template <class K>
static int ctas_per_sm(K kernel, int* cache) {
  if (*cache <= 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 256, 0) != cudaSuccess || b <= 0) {
      cudaGetLastError();
      b = 4;
    }
    *cache = b;
  }
  return *cache;
}

void launch_grid_update(const Params& P, const Tuning& tu, GridBuffers g, const float* tool_pose, int step,
                        int max_steps, cudaStream_t s) {
  long long nb = (long long)P.S * P.NB;
  const int per = tu.grid_blocks;
  static int occ[2] = {0, 0};
  auto k = P.tool ? grid_update_kernel<true> : grid_update_kernel<false>;
  int grid = int(nb / per + 1);
  const int cap = sm_count() * ctas_per_sm(k, &occ[P.tool ? 1 : 0]);
  if (grid > cap) grid = cap;
  k<<<grid, 64 * per, 0, s>>>(P, g.acc, g.gv, g.gstore, g.flags, g.list, g.count, tool_pose, step, max_steps,
                               g.cgv, g.cap, g.ovf, g.ovf_bit);
}

void launch_expand_grid(const Params& P, GridBuffers g, float4* gv, cudaStream_t s) {
  if (g.cgv == nullptr || g.cap <= 0) return;
  // the entry count is on the device: a grid-stride loop over up to cap entries
  const long long n = (long long)g.cap * 64;
  long long blocks = (n + 255) / 256;
  const long long most = 8LL * sm_count();
  if (blocks > most) blocks = most;
  expand_grid_kernel<<<int(blocks), 256, 0, s>>>(P, g.cgv, g.list, g.count, g.cap, gv);
}

template <int NT, bool kExt, bool kTool>
static cudaError_t forward_run_variant(const Params& P, const float* src, float* W, const uint32_t* tag,
                                       GridBuffers g, int* lists, long long list_stride, int* count,
                                       const float* pose, int n0, int n1, int max_steps, int* tile_ctr,
                                       unsigned* bar, int* err, cudaStream_t s) {
  auto kern = forward_run_kernel<NT, kExt, kTool>;
  static int occ = 0;  // resident CTAs per SM (queried once per variant)
  if (occ <= 0) {
    int b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, NT, 0);
    if (e != cudaSuccess) return e;
    if (b <= 0) return cudaErrorCooperativeLaunchTooLarge;
    occ = b;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(occ * sm_count());
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const unsigned long long timeout_ns = 5000000000ull;  // 5 s per barrier wait
  return cudaLaunchKernelEx(&cfg, kern, P, src, W, tag, g.Fp, g.acc, g.gv, g.flags, lists, list_stride, count, pose,
                            n0, n1, max_steps, tile_ctr, bar, err, timeout_ns);
}

cudaError_t launch_forward_run(const Params& P, const Tuning& tu, const float* src, float* W, const uint32_t* tag,
                               GridBuffers g, int* lists, long long list_stride, int* count, const float* pose,
                               int n0, int n1, int max_steps, int* tile_ctr, unsigned* bar, int* err,
                               cudaStream_t s) {
  if (P.N == 0 || n1 <= n0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(tile_ctr, 0, 2 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
#define MPM_RUN(NT, X, TL) \
  forward_run_variant<NT, X, TL>(P, src, W, tag, g, lists, list_stride, count, pose, n0, n1, max_steps, tile_ctr, \
                                 bar, err, s)
  const bool ext = P.ext != 0, tool = P.tool != 0;
  if (tu.scatter_threads == 128) {
    if (ext) return tool ? MPM_RUN(128, true, true) : MPM_RUN(128, true, false);
    return tool ? MPM_RUN(128, false, true) : MPM_RUN(128, false, false);
  }
  if (ext) return tool ? MPM_RUN(256, true, true) : MPM_RUN(256, true, false);
  return tool ? MPM_RUN(256, false, true) : MPM_RUN(256, false, false);
#undef MPM_RUN
}

cudaError_t launch_barrier_selftest(unsigned* bar, int blocks, unsigned expected, int rounds, int* err,
                                    unsigned long long timeout_ns, int* passed, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(64);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, barrier_selftest_kernel, bar, expected, rounds, err, timeout_ns, passed);
}

void launch_g2p(const Params& P, const Tuning& tu, const float* st_in, float* st_out, const uint32_t* tag,
                const float* Fp, const float4* gv, int* err, cudaStream_t s) {
  if (P.N == 0) return;
  const int t = tu.gather_threads;
  g2p_kernel<<<blocks_for(P.N, t), t, 0, s>>>(P, st_in, st_out, tag, Fp, gv, err);
}

}  // namespace mpm
