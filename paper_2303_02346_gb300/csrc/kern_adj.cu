// Hand-written reverse-mode kernels of one MLS-MPM step (paper Sec. 3.3 and
// App. A: gradients through the simulation, with the SVD gradient written by
// hand). One kernel per forward stage, run in reverse order:
//   g2p_adj   gather of the step's grid velocities; scatter of dL/dv_i,
//   grid_adj  adjoint of v = contact(mv/m + dt g) with walls, plus the tool's
//             pose/velocity gradients reduced per step,
//   p2g_adj   gather of dL/dm_i, dL/dmv_i; adjoint of the MLS affine
//             momentum and of the constitutive model (SVD adjoint).
// The adjoint state has the same SoA layout as the particle state
// (x, v, C, F; a liquid uses only F[0] = J).
#include "common.cuh"
#include "constitutive.cuh"
#include "kernels.h"
#include "scatter.cuh"
#include "tool.cuh"

namespace mpm {

constexpr int fX = 0, fV = 3, fC = 6, fF = 15;
static inline int blocks_for(long long n, int t) { return int((n + t - 1) / t); }

// Adjoint of G2P of step n for one particle (the gather part). Inputs: the
// adjoint (xb, vb, Cb, Fb) of the state of step n + 1 in registers, x^n and J^n
// (st_n), C^{n+1} (st_n1) and the projected F^n (Fp_n). With vb and Cb the
// total adjoints of v^{n+1} and C^{n+1}, the node offset o's share of the
// scatter is W (vb + s4 Cb dpos) = W (u + Cq o): on return u and Cq hold
// those coefficients (what the scatter needs; vb and Cb are used up) and xb
// the partial adjoint of x^n; sc is the stencil of x^n.
__device__ inline void g2p_adj_gather(const Params& P, int p, const MatParams& M, int scene,
                                      const float* __restrict__ st_n, const float* __restrict__ st_n1,
                                      const float* __restrict__ Fp_n, const float4* __restrict__ gv,
                                      float* xb, float* vb, float* Cb, const float* Fb, Stencil& sc,
                                      float* u, float* Cq) {
  const int N = P.N;
  const float s4 = 4.0f * P.inv_dx * P.inv_dx;
  float x[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) x[d] = st_n[(fX + d) * N + p];
  float G[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) G[k] = ((k % 4 == 0) ? 1.0f : 0.0f) + P.dt * st_n1[(fC + k) * N + p];
  if (is_liquid(M.kind)) {
    // J' = J det(G): Gbar = Jbar' J cof(G)
    const float J = st_n[fF * N + p];
    float K[9];
    cof3(G, K);
#pragma unroll
    for (int k = 0; k < 9; ++k) Cb[k] += P.dt * Fb[0] * J * K[k];
  } else {
    // F' = G F_p: Cbar += dt Fbar' F_p^T (F_p stored by the recompute)
    float Fp[9], t[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Fp[k] = Fp_n[sslot(P, k, p)];
    mat_mult(Fb, Fp, t);
#pragma unroll
    for (int k = 0; k < 9; ++k) Cb[k] += P.dt * t[k];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) vb[d] += P.dt * xb[d];
  make_stencil(x, P, sc);
  // xbar += sum_o grad W (v_i . (vb + s4 Cb dpos)) - s4 W Cb^T v_i, with
  // dpos = (o - f) dx for the stencil offset o: vb + s4 Cb dpos = u + Cq o
  // (u = vb - s4 dx Cb f, Cq = s4 dx Cb), so each node costs a few adds for
  // its integer offset; sum_o W v_i is accumulated once for the second term.
  const float sd = s4 * P.dx;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    u[i] = vb[i] - sd * (Cb[3 * i] * sc.f[0] + Cb[3 * i + 1] * sc.f[1] + Cb[3 * i + 2] * sc.f[2]);
#pragma unroll
    for (int j = 0; j < 3; ++j) Cq[3 * i + j] = sd * Cb[3 * i + j];
  }
  // W = w0[a] w1[b] w2[c] factorises: each (a, b) column of three nodes is
  // reduced over c first (P = sum_c w2[c] sv, Q = sum_c w2'[c] sv,
  // t = sum_c w2[c] v_i), then weighted by the column's factors.
  // Gv = sum_o W v_i runs on the lane pairs (x, y) and (z, w) of the node
  // values with packed two-lane FP32 instructions (w carried along unused).
  float xs[3] = {0.f, 0.f, 0.f};
  float2 Gp[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  const float2 w20 = make_float2(sc.w[2][0], sc.w[2][0]), w21 = make_float2(sc.w[2][1], sc.w[2][1]),
               w22 = make_float2(sc.w[2][2], sc.w[2][2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float4* col = gv + node_index(P, scene, sc.base[0] + a, sc.base[1] + b, sc.base[2]);
      const float4 g0 = __ldg(col), g1 = __ldg(col + 1), g2 = __ldg(col + 2);
      float uab[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) uab[i] = u[i] + float(a) * Cq[3 * i] + float(b) * Cq[3 * i + 1];
      // sv at offset c: v_i . (uab + c Cq[:, 2])
      const float sv0 = g0.x * uab[0] + g0.y * uab[1] + g0.z * uab[2];
      const float sv1 = g1.x * (uab[0] + Cq[2]) + g1.y * (uab[1] + Cq[5]) + g1.z * (uab[2] + Cq[8]);
      const float sv2 =
          g2.x * (uab[0] + 2.0f * Cq[2]) + g2.y * (uab[1] + 2.0f * Cq[5]) + g2.z * (uab[2] + 2.0f * Cq[8]);
      const float Pc = sc.w[2][0] * sv0 + sc.w[2][1] * sv1 + sc.w[2][2] * sv2;
      const float Qc = sc.dw[2][0] * sv0 + sc.dw[2][1] * sv1 + sc.dw[2][2] * sv2;
      const float wab = sc.w[0][a] * sc.w[1][b], dab0 = sc.dw[0][a] * sc.w[1][b], dab1 = sc.w[0][a] * sc.dw[1][b];
      xs[0] += dab0 * Pc;
      xs[1] += dab1 * Pc;
      xs[2] += wab * Qc;
      const float2 wab2 = make_float2(wab, wab);
      Gp[0] = __ffma2_rn(wab2, __ffma2_rn(w22, make_float2(g2.x, g2.y),
                                          __ffma2_rn(w21, make_float2(g1.x, g1.y),
                                                     __fmul2_rn(w20, make_float2(g0.x, g0.y)))), Gp[0]);
      Gp[1] = __ffma2_rn(wab2, __ffma2_rn(w22, make_float2(g2.z, g2.w),
                                          __ffma2_rn(w21, make_float2(g1.z, g1.w),
                                                     __fmul2_rn(w20, make_float2(g0.z, g0.w)))), Gp[1]);
    }
  }
  const float Gv[3] = {Gp[0].x, Gp[0].y, Gp[1].x};
#pragma unroll
  // s4 Cb = Cq / dx
  for (int d = 0; d < 3; ++d)
    xb[d] += P.inv_dx * (xs[d] - (Cq[d] * Gv[0] + Cq[3 + d] * Gv[1] + Cq[6 + d] * Gv[2]));
}

// Scatter part of the G2P adjoint (every thread must call it):
// vbar_i += W (u + Cq o) for the node at stencil offset o.
template <int NT>
__device__ inline void g2p_adj_scatter(ScatterTile<NT>& T, const Params& P, bool valid, int scene,
                                       const Stencil& sc, const float* u, const float* Cq,
                                       float4* __restrict__ gadj_v) {
  scatter_setup(T, valid, sc.base, scene);
  if (T.box[7]) {
    const int rank = scatter_count(T, valid, sc.base);
    __syncthreads();
    scan_cells(T);
    if (valid) scatter_record_affine(T, rank, sc, 0.0f, u, Cq);
    __syncthreads();
    scatter_accumulate<false, NT>(T);
  } else if (valid) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int b = 0; b < 3; ++b) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float W = sc.w[0][a] * sc.w[1][b] * sc.w[2][c];
          float val[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) val[i] = u[i] + float(a) * Cq[3 * i] + float(b) * Cq[3 * i + 1] + float(c) * Cq[3 * i + 2];
          red_add_v4(gadj_v + node_index(P, scene, sc.base[0] + a, sc.base[1] + b, sc.base[2] + c),
                     W * val[0], W * val[1], W * val[2], 0.0f);
        }
      }
    }
  }
  scatter_flush(T, gadj_v, P, nullptr, nullptr, nullptr);
}

// kHigh: 4 resident CTAs of 256 per SM (64 registers) instead of 3
template <int NT, bool kHigh = false>
__global__ void __launch_bounds__(NT, (kHigh ? kScatterResidentThreadsHigh : kScatterResidentThreads) / NT)
g2p_adj_kernel(Params P, const float* __restrict__ st_n, const float* __restrict__ st_n1,
               const uint32_t* __restrict__ tag, const float* __restrict__ Fp_n,
               float* __restrict__ adj, const float4* __restrict__ gv, float4* __restrict__ gadj_v) {
  __shared__ ScatterTile<NT> T;
  const int N = P.N;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = p < N;
  int scene = 0;
  Stencil sc;
  sc.base[0] = sc.base[1] = sc.base[2] = 0;
  float Cb[9], vb[3] = {0.f, 0.f, 0.f}, xb[3], Fb[9], u[3], Cq[9];
  if (valid) {
    const uint32_t tg = tag[p];
    scene = tag_scene(tg);
    const MatParams& M = P.mat[tag_mat(tg)];
#pragma unroll
    for (int k = 0; k < 9; ++k) Cb[k] = adj[(fC + k) * N + p];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      xb[d] = adj[(fX + d) * N + p];
      vb[d] = adj[(fV + d) * N + p];
    }
    Fb[0] = adj[fF * N + p];
    if (!is_liquid(M.kind)) {
#pragma unroll
      for (int k = 1; k < 9; ++k) Fb[k] = adj[(fF + k) * N + p];
    }
    g2p_adj_gather(P, p, M, scene, st_n, st_n1, Fp_n, gv, xb, vb, Cb, Fb, sc, u, Cq);
#pragma unroll
    for (int d = 0; d < 3; ++d) adj[(fX + d) * N + p] = xb[d];
  }
  g2p_adj_scatter<NT>(T, P, valid, scene, sc, u, Cq, gadj_v);
}

__device__ inline void node_of_blk(const Params& P, int blk, int l, int& scene, int& i, int& j, int& k) {
  scene = blk / P.NB;
  int bl = blk - scene * P.NB;
  int bx = bl / (P.nb * P.nb), by = (bl / P.nb) % P.nb, bz = bl % P.nb;
  i = bx * kBlockEdge + (l >> 4);
  j = by * kBlockEdge + ((l >> 2) & 3);
  k = bz * kBlockEdge + (l & 3);
}

__device__ inline void flush_tool_grad(float* acc, int scene, float* __restrict__ tool_grad, int step,
                                       int max_steps, bool warp_uniform) {
  float* dst = tool_grad + ((long long)scene * max_steps + step) * kToolGradFields;
  if (warp_uniform) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < kToolGradFields; ++q) {
      float s = warp_sum(acc[q]);
      if (lane == 0 && s != 0.0f) atomicAdd(dst + q, s);
    }
  } else {
#pragma unroll
    for (int q = 0; q < kToolGradFields; ++q)
      if (acc[q] != 0.0f) atomicAdd(dst + q, acc[q]);
  }
}

// As the grid update: each group of 64 threads loads the list entries and
// node values of kItems blocks before processing any of them. kTool: built
// with the tool-contact adjoint (its pose-gradient accumulators take
// registers, so the kernel without a tool takes more blocks at a time).
template <bool kTool, int kGridAdjItems>
__global__ void __launch_bounds__(256)
grid_adj_kernel(Params P, const float4* __restrict__ gstore, float4* __restrict__ gadj_v,
                float4* __restrict__ gadj_m, const int* __restrict__ list,
                const int* __restrict__ count, const float* __restrict__ pose,
                float* __restrict__ tool_grad, int step, int max_steps) {
  const int cnt = *count;
  const int per = blockDim.x >> 6;
  const int l = threadIdx.x & 63;
  const int stride = gridDim.x * per;
  float acc[kToolGradFields];
#pragma unroll
  for (int q = 0; q < kToolGradFields; ++q) acc[q] = 0.0f;
  int cur = -1;
  for (int item0 = blockIdx.x * per + (threadIdx.x >> 6); item0 < cnt; item0 += stride * kGridAdjItems) {
    int blk[kGridAdjItems];
    float4 vb4[kGridAdjItems], um4[kGridAdjItems];
    unsigned ok = 0u;  // bit u: node of item u inside the grid
#pragma unroll
    for (int u = 0; u < kGridAdjItems; ++u) {
      const int item = item0 + u * stride;
      blk[u] = item < cnt ? __ldg(list + item) : -1;
    }
#pragma unroll
    for (int u = 0; u < kGridAdjItems; ++u) {
      if (blk[u] < 0) continue;
      int scene, i, j, k;
      node_of_blk(P, blk[u], l, scene, i, j, k);
      if (i >= P.n || j >= P.n || k >= P.n) continue;
      ok |= 1u << u;
      const long long idx = node_index(P, scene, i, j, k);
      vb4[u] = gadj_v[idx];
      um4[u] = __ldg(gstore + idx);
    }
#pragma unroll
    for (int u = 0; u < kGridAdjItems; ++u) {
      if (!(ok & (1u << u))) continue;
      int scene, i, j, k;
      node_of_blk(P, blk[u], l, scene, i, j, k);
      const long long idx = node_index(P, scene, i, j, k);
      gadj_v[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 um = um4[u];
      if (!(um.w > 0.0f)) {
        gadj_m[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
      bool wall = i < P.bound || j < P.bound || k < P.bound || i >= P.n - P.bound ||
                  j >= P.n - P.bound || k >= P.n - P.bound;
      float vb[3] = {wall ? 0.0f : vb4[u].x, wall ? 0.0f : vb4[u].y, wall ? 0.0f : vb4[u].z};
      float uu[3] = {um.x, um.y, um.z};
      float ub[3] = {vb[0], vb[1], vb[2]};
      if (kTool && !wall) {
        if (scene != cur) {
          if (cur >= 0) flush_tool_grad(acc, cur, tool_grad, step, max_steps, false);
#pragma unroll
          for (int q = 0; q < kToolGradFields; ++q) acc[q] = 0.0f;
          cur = scene;
        }
        ToolState T;
        load_tool(pose + ((long long)scene * max_steps + step) * kToolFields, T);
        float xi[3] = {i * P.dx, j * P.dx, k * P.dx};
        contact_adjoint(P, T, xi, uu, vb, ub, acc, acc + 3, acc + 12, acc + 15);
      }
      float inv = 1.0f / um.w;
      // u = mv / m + dt g
      float mb = -(ub[0] * (uu[0] - P.dt * P.g[0]) + ub[1] * (uu[1] - P.dt * P.g[1]) +
                   ub[2] * (uu[2] - P.dt * P.g[2])) * inv;
      gadj_m[idx] = make_float4(mb, ub[0] * inv, ub[1] * inv, ub[2] * inv);
    }
  }
  if (kTool) {
    // lanes with cur == -1 hold zeros and join the warp's common scene
    int c = __reduce_max_sync(0xffffffffu, cur);
    bool uni = __all_sync(0xffffffffu, cur == c || cur == -1) && c >= 0;
    if (uni) {
      flush_tool_grad(acc, c, tool_grad, step, max_steps, true);
    } else if (cur >= 0) {
      flush_tool_grad(acc, cur, tool_grad, step, max_steps, false);
    }
  }
}

// Adjoint of a viscous liquid's stress through its trial F = a Gn,
// a = (J / det Gn)^(1/3), Gn = I + dt C^n (the reset J^(1/3) I advanced by the
// step): with Fbar the SVD adjoint of tau = corotated(F),
//   Jbar = (Fbar : Gn) a / (3 J)   (returned),
//   Cbar = dt (a Fbar - (Fbar : Gn) (a / 3) Gn^-T)   (written to Cv).
// Kept out of line: its registers stay off the paths of the other materials.
__device__ __noinline__ float viscous_liquid_adjoint(const MatParams& M, const float* U, const float* sg,
                                                     const float* V, const float* taub, const float* C, float dt,
                                                     float J, float* Cv) {
  float Gn[9], Kn[9], Fbt[9], zero[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    Gn[k] = ((k % 4 == 0) ? 1.0f : 0.0f) + dt * C[k];
    zero[k] = 0.0f;
  }
  solid_adjoint_svd<true>(M, U, sg, V, zero, taub, Fbt);
  const float dG = det3(Gn);
  const float a = cbrtf(J / dG);
  cof3(Gn, Kn);  // Gn^-T = cof(Gn) / det(Gn)
  float sFG = 0.0f;
#pragma unroll
  for (int k = 0; k < 9; ++k) sFG += Fbt[k] * Gn[k];
#pragma unroll
  for (int k = 0; k < 9; ++k) Cv[k] = dt * (a * Fbt[k] - sFG * (a / 3.0f) * Kn[k] / dG);
  return sFG * a / (3.0f * J);
}

// Adjoint of P2G of step n (with the constitutive adjoint) for one particle.
// Inputs: the state of step n (st_n), C^{n+1} (st_n1), the stored SVD of the
// trial F^n, the partial adjoint of x^n and the adjoint F' of F^{n+1} in adj,
// and the adjoint grid (mbar, mvbar) of step n. Outputs in registers: the
// adjoint (xb, vb, Cb, Fb) of the state of step n (a liquid's Jbar in Fb[0]).
template <bool kExt>
__device__ inline void p2g_adj_particle(const Params& P, int p, const MatParams& M, int scene,
                                        const float* __restrict__ st_n, const float* __restrict__ st_n1,
                                        const float* __restrict__ svd_n, const float* __restrict__ adj,
                                        const float4* __restrict__ gadj_m, float* xb, float* vb,
                                        float* Cb, float* Fb) {
  const int N = P.N;
  // the fields read after the node gather (C^{n+1} and the incoming adjoint)
  // are requested from L2 now, so that the gather's latency covers theirs
#pragma unroll
  for (int k = 0; k < 9; ++k) prefetch_l2(st_n1 + (fC + k) * N + p);
#pragma unroll
  for (int d = 0; d < 3; ++d) prefetch_l2(adj + (fX + d) * N + p);
  prefetch_l2(adj + fF * N + p);
  float x[3], v[3], C[9], tau[9], U[9], sg[3], V[9];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    x[d] = st_n[(fX + d) * N + p];
    v[d] = st_n[(fV + d) * N + p];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) C[k] = st_n[(fC + k) * N + p];
  const bool liquid = is_liquid(M.kind), viscous = kExt && M.kind == kViscousLiquid;
  const bool rigid = kExt && M.kind == kRigid;
  float J = 0.0f;
  if (rigid) {
#pragma unroll
    for (int k = 0; k < 9; ++k) tau[k] = 0.0f;
  } else if (liquid && !viscous) {
    J = st_n[fF * N + p];
    const float pr = M.lam * J * (J - 1.0f);
#pragma unroll
    for (int k = 0; k < 9; ++k) tau[k] = (k % 4 == 0) ? pr : 0.0f;
  } else {
    // SVD of the trial F stored by the recompute of this step
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      U[k] = svd_n[sslot(P, k, p)];
      V[k] = svd_n[sslot(P, 12 + k, p)];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) sg[k] = svd_n[sslot(P, 9 + k, p)];
    solid_tau_from_svd<kExt>(M, U, sg, tau);
    if (viscous) J = st_n[fF * N + p];
  }
  const float m = M.mass;
  const float coef = -P.dt * M.vol * 4.0f * P.inv_dx * P.inv_dx;
  float A[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = coef * tau[k] + m * C[k];
  Stencil sc;
  make_stencil(x, P, sc);
  // Per node o (dpos = (o - f) dx), with g = (mbar, mvbar) at the node:
  //   q = m v + A dpos = q0 + Ad o   (q0 = m v - A f dx, Ad = A dx),
  //   xbar += grad W (m mbar + mvbar . q) - W A^T mvbar,
  //   vbar += W m mvbar,   Abar += W mvbar dpos^T.
  // The sums that do not depend on o are taken once: Gv = sum_o W mvbar
  // gives vbar = m Gv and the A^T term; S = sum_o W mvbar o^T gives
  // Abar = dx (S - Gv f^T).
  const float dx = P.dx;
  float Ad[9], q0[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) Ad[k] = A[k] * dx;
#pragma unroll
  for (int i = 0; i < 3; ++i) q0[i] = m * v[i] - (Ad[3 * i] * sc.f[0] + Ad[3 * i + 1] * sc.f[1] + Ad[3 * i + 2] * sc.f[2]);
  // W = w0[a] w1[b] w2[c] factorises: each (a, b) column of three nodes is
  // reduced over c first (P = sum_c w2[c] s, Q = sum_c w2'[c] s,
  // t = sum_c w2[c] mvbar, tc = sum_c c w2[c] mvbar), then weighted by the
  // column's factors.
  // t, tc and the sums Gv, S run on the lane pairs (mbar, mvbar_x) and
  // (mvbar_y, mvbar_z) of the node values with packed two-lane FP32
  // instructions (the mbar lane is carried along unused): Gp[h] holds lanes h
  // of (-, Gv), Sp[j][h] lanes h of (-, S[:, j]).
  float xs[3] = {0.f, 0.f, 0.f};
  float2 Gp[2], Sp[3][2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    Gp[h] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < 3; ++j) Sp[j][h] = make_float2(0.0f, 0.0f);
  }
  const float2 w20 = make_float2(sc.w[2][0], sc.w[2][0]), w21 = make_float2(sc.w[2][1], sc.w[2][1]),
               w22 = make_float2(sc.w[2][2], sc.w[2][2]);
  const float2 w2c2 = make_float2(2.0f * sc.w[2][2], 2.0f * sc.w[2][2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float4* col = gadj_m + node_index(P, scene, sc.base[0] + a, sc.base[1] + b, sc.base[2]);
      const float4 g0 = __ldg(col), g1 = __ldg(col + 1), g2 = __ldg(col + 2);
      float qab[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) qab[i] = q0[i] + float(a) * Ad[3 * i] + float(b) * Ad[3 * i + 1];
      // s at offset c: m mbar + mvbar . (qab + c Ad[:, 2])
      const float s0 = m * g0.x + g0.y * qab[0] + g0.z * qab[1] + g0.w * qab[2];
      const float s1 = m * g1.x + g1.y * (qab[0] + Ad[2]) + g1.z * (qab[1] + Ad[5]) + g1.w * (qab[2] + Ad[8]);
      const float s2 = m * g2.x + g2.y * (qab[0] + 2.0f * Ad[2]) + g2.z * (qab[1] + 2.0f * Ad[5]) +
                       g2.w * (qab[2] + 2.0f * Ad[8]);
      const float Pc = sc.w[2][0] * s0 + sc.w[2][1] * s1 + sc.w[2][2] * s2;
      const float Qc = sc.dw[2][0] * s0 + sc.dw[2][1] * s1 + sc.dw[2][2] * s2;
      const float wab = sc.w[0][a] * sc.w[1][b], dab0 = sc.dw[0][a] * sc.w[1][b], dab1 = sc.w[0][a] * sc.dw[1][b];
      xs[0] += dab0 * Pc;
      xs[1] += dab1 * Pc;
      xs[2] += wab * Qc;
      const float2 gp[3][2] = {{make_float2(g0.x, g0.y), make_float2(g0.z, g0.w)},
                               {make_float2(g1.x, g1.y), make_float2(g1.z, g1.w)},
                               {make_float2(g2.x, g2.y), make_float2(g2.z, g2.w)}};
      const float2 wab2 = make_float2(wab, wab);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 t = __ffma2_rn(w22, gp[2][h], __ffma2_rn(w21, gp[1][h], __fmul2_rn(w20, gp[0][h])));
        const float2 tc = __ffma2_rn(w2c2, gp[2][h], __fmul2_rn(w21, gp[1][h]));
        const float2 ut = __fmul2_rn(wab2, t);
        Gp[h] = __fadd2_rn(Gp[h], ut);
        if (a == 1) Sp[0][h] = __fadd2_rn(Sp[0][h], ut);
        if (a == 2) Sp[0][h] = __ffma2_rn(make_float2(2.0f, 2.0f), ut, Sp[0][h]);
        if (b == 1) Sp[1][h] = __fadd2_rn(Sp[1][h], ut);
        if (b == 2) Sp[1][h] = __ffma2_rn(make_float2(2.0f, 2.0f), ut, Sp[1][h]);
        Sp[2][h] = __ffma2_rn(wab2, tc, Sp[2][h]);
      }
    }
  }
  const float Gv[3] = {Gp[0].y, Gp[1].x, Gp[1].y};
  float S[9];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    S[j] = Sp[j][0].y;
    S[3 + j] = Sp[j][1].x;
    S[6 + j] = Sp[j][1].y;
  }
  float Ab[9];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    xb[d] = adj[(fX + d) * N + p] + P.inv_dx * xs[d] - (A[d] * Gv[0] + A[3 + d] * Gv[1] + A[6 + d] * Gv[2]);
    vb[d] = m * Gv[d];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Ab[3 * i + j] = dx * (S[3 * i + j] - Gv[i] * sc.f[j]);
  float G[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) G[k] = ((k % 4 == 0) ? 1.0f : 0.0f) + P.dt * st_n1[(fC + k) * N + p];
  float taub[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) taub[k] = coef * Ab[k];
  float Cv[9];  // C^n's adjoint through a viscous liquid's trial F
#pragma unroll
  for (int k = 0; k < 9; ++k) Cv[k] = 0.0f;
  if (viscous) {
    Fb[0] = adj[fF * N + p] * det3(G) + viscous_liquid_adjoint(M, U, sg, V, taub, C, P.dt, J, Cv);
  } else if (liquid) {
    Fb[0] = adj[fF * N + p] * det3(G) + M.lam * (2.0f * J - 1.0f) * (taub[0] + taub[4] + taub[8]);
  } else if (rigid) {
    // tau = 0 and F_p = F: Fbar = G^T Fbar'
    float Fb1[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Fb1[k] = adj[(fF + k) * N + p];
    mat_tmul(G, Fb1, Fb);
  } else {
    float Fb1[9], Fpb[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Fb1[k] = adj[(fF + k) * N + p];
    mat_tmul(G, Fb1, Fpb);  // Fbar_p = G^T Fbar'
    solid_adjoint_svd<kExt>(M, U, sg, V, Fpb, taub, Fb);
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) Cb[k] = m * Ab[k] + Cv[k];
}

template <bool kExt>
__global__ void __launch_bounds__(512)
p2g_adj_kernel(Params P, const float* __restrict__ st_n, const float* __restrict__ st_n1,
               const uint32_t* __restrict__ tag, const float* __restrict__ svd_n,
               float* __restrict__ adj, const float4* __restrict__ gadj_m) {
  const int N = P.N;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const uint32_t tg = tag[p];
  const MatParams& M = P.mat[tag_mat(tg)];
  float xb[3], vb[3], Cb[9], Fb[9];
  p2g_adj_particle<kExt>(P, p, M, tag_scene(tg), st_n, st_n1, svd_n, adj, gadj_m, xb, vb, Cb, Fb);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    adj[(fX + d) * N + p] = xb[d];
    adj[(fV + d) * N + p] = vb[d];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) adj[(fC + k) * N + p] = Cb[k];
  adj[fF * N + p] = Fb[0];
  if (!is_liquid(M.kind)) {
#pragma unroll
    for (int k = 1; k < 9; ++k) adj[(fF + k) * N + p] = Fb[k];
  }
}

// Adjoint of P2G of step n fused with the adjoint of G2P of step n - 1: the
// adjoint of the state of step n stays in registers; only the partial adjoint
// of x^{n-1} and the adjoint of F^n are written back. Compiled for two CTAs
// of 256 (three of 128) per SM: at most 128 (170) registers a thread.
template <int NT, bool kExt>
__global__ void __launch_bounds__(NT, NT >= 256 ? 2 : 3)
adj_fused_kernel(Params P, const float* __restrict__ st_prev, const float* __restrict__ st_n,
                 const float* __restrict__ st_n1, const uint32_t* __restrict__ tag,
                 const float* __restrict__ svd_n, const float* __restrict__ Fp_prev,
                 float* __restrict__ adj, const float4* __restrict__ gadj_m,
                 const float4* __restrict__ gv_prev, float4* __restrict__ gadj_v) {
  __shared__ ScatterTile<NT> T;
  const int N = P.N;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = p < N;
  int scene = 0;
  Stencil sc;
  sc.base[0] = sc.base[1] = sc.base[2] = 0;
  float xb[3], vb[3] = {0.f, 0.f, 0.f}, Cb[9], Fb[9], u[3], Cq[9];
  if (valid) {
    const uint32_t tg = tag[p];
    scene = tag_scene(tg);
    const MatParams& M = P.mat[tag_mat(tg)];
    p2g_adj_particle<kExt>(P, p, M, scene, st_n, st_n1, svd_n, adj, gadj_m, xb, vb, Cb, Fb);
    g2p_adj_gather(P, p, M, scene, st_prev, st_n, Fp_prev, gv_prev, xb, vb, Cb, Fb, sc, u, Cq);
#pragma unroll
    for (int d = 0; d < 3; ++d) adj[(fX + d) * N + p] = xb[d];
    adj[fF * N + p] = Fb[0];
    if (!is_liquid(M.kind)) {
#pragma unroll
      for (int k = 1; k < 9; ++k) adj[(fF + k) * N + p] = Fb[k];
    }
  }
  g2p_adj_scatter<NT>(T, P, valid, scene, sc, u, Cq, gadj_v);
}

__global__ void clear_blocks_kernel(Params P, float4* __restrict__ grid, const int* __restrict__ list,
                                    const int* __restrict__ count) {
  const int cnt = *count;
  const int per = blockDim.x >> 6;
  const int l = threadIdx.x & 63;
  for (int item = blockIdx.x * per + (threadIdx.x >> 6); item < cnt; item += gridDim.x * per) {
    int scene, i, j, k;
    node_of_blk(P, list[item], l, scene, i, j, k);
    if (i >= P.n || j >= P.n || k >= P.n) continue;
    grid[node_index(P, scene, i, j, k)] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// ---------------------------------------------------------------------------
void launch_g2p_adj(const Params& P, const Tuning& tu, const float* st_n, const float* st_n1,
                    const uint32_t* tag, const float* Fp_n, float* adj, const float4* gv, float4* gadj_v,
                    cudaStream_t s) {
  if (P.N == 0) return;
  if (tu.scatter_threads == 128) {
    g2p_adj_kernel<128><<<blocks_for(P.N, 128), 128, 0, s>>>(P, st_n, st_n1, tag, Fp_n, adj, gv, gadj_v);
  } else if (tu.scatter_ctas == 4) {
    max_shared_carveout(reinterpret_cast<const void*>(g2p_adj_kernel<256, true>));
    g2p_adj_kernel<256, true><<<blocks_for(P.N, 256), 256, 0, s>>>(P, st_n, st_n1, tag, Fp_n, adj, gv, gadj_v);
  } else {
    g2p_adj_kernel<256><<<blocks_for(P.N, 256), 256, 0, s>>>(P, st_n, st_n1, tag, Fp_n, adj, gv, gadj_v);
  }
}

// Resident CTAs of 256 threads per SM of a grid-adjoint variant (queried once).
template <class K>
static int ctas_per_sm(K kernel, int* cache) {
  if (*cache <= 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 256, 0) != cudaSuccess || b <= 0) {
      cudaGetLastError();
      b = 2;
    }
    *cache = b;
  }
  return *cache;
}

void launch_grid_adj(const Params& P, const Tuning& tu, GridBuffers g, float4* gadj_v, float4* gadj_m,
                     const float* tool_pose, float* tool_grad, int step, int max_steps,
                     cudaStream_t s) {
  long long nb = (long long)P.S * P.NB;
  const int per = tu.grid_blocks;
  static int occ[2] = {0, 0};
  auto k = P.tool ? grid_adj_kernel<true, 2> : grid_adj_kernel<false, 4>;
  int grid = int(nb / per + 1);
  const int cap = sm_count() * ctas_per_sm(k, &occ[P.tool ? 1 : 0]);
  if (grid > cap) grid = cap;
  // without a tool the post-contact velocities stored for the gather stand in
  // for the pre-contact ones: they differ only at wall nodes, whose adjoint
  // the walls zero (and the mass in .w is the same)
  const float4* um = g.gstore ? g.gstore : g.gv;
  k<<<grid, 64 * per, 0, s>>>(P, um, gadj_v, gadj_m, g.list, g.count, tool_pose, tool_grad, step, max_steps);
}

void launch_adj_fused(const Params& P, const Tuning& tu, const float* st_prev, const float* st_n,
                      const float* st_n1, const uint32_t* tag, const float* svd_n, const float* Fp_prev,
                      float* adj, const float4* gadj_m, const float4* gv_prev, float4* gadj_v,
                      cudaStream_t s) {
  if (P.N == 0) return;
  auto k = tu.scatter_threads == 128 ? (P.ext ? adj_fused_kernel<128, true> : adj_fused_kernel<128, false>)
                                     : (P.ext ? adj_fused_kernel<256, true> : adj_fused_kernel<256, false>);
  const int nt = tu.scatter_threads == 128 ? 128 : 256;
  k<<<blocks_for(P.N, nt), nt, 0, s>>>(P, st_prev, st_n, st_n1, tag, svd_n, Fp_prev, adj, gadj_m, gv_prev, gadj_v);
}

void launch_p2g_adj(const Params& P, const Tuning& tu, const float* st_n, const float* st_n1,
                    const uint32_t* tag, const float* svd_n, float* adj, const float4* gadj_m,
                    cudaStream_t s) {
  if (P.N == 0) return;
  const int t = tu.gather_threads;
  auto k = P.ext ? p2g_adj_kernel<true> : p2g_adj_kernel<false>;
  k<<<blocks_for(P.N, t), t, 0, s>>>(P, st_n, st_n1, tag, svd_n, adj, gadj_m);
}

void launch_clear_blocks(const Params& P, float4* grid, const int* list, const int* count,
                         cudaStream_t s) {
  long long nb = (long long)P.S * P.NB;
  int g = int(nb / 4 + 1);
  if (g > sm_count() * 8) g = sm_count() * 8;
  clear_blocks_kernel<<<g, 256, 0, s>>>(P, grid, list, count);
}

}  // namespace mpm
