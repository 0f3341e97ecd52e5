// Particle-to-grid scatter through a cell-binned shared-memory tile.
//
// A CTA owns a contiguous range of particles that the block sort keeps
// spatially compact. It reduces the bounding box of their stencil origins
// ("cells"). If the box plus the 3-node stencil fits in the tile and every
// particle belongs to one scene:
//   1. each thread writes its particle's record (fractional position f and the
//      coefficients of its per-node contribution) into shared memory, counting-
//      sorted by cell;
//   2. work item (cell, o_x, o_y) over the occupied cells accumulates the
//      contributions of all particles of that cell to its 3 nodes (o_z = 0..2)
//      in registers, then adds them to the tile with one shared atomic per node
//      and value;
//   3. the CTA flushes every touched node with one global float4 reduction.
// Particles of one cell hit the same 27 nodes, so step 2 replaces one atomic
// per particle and node by one per cell and node; the 9 items of one cell sit
// in neighbouring lanes, read the same records (shared-memory broadcast) and add
// to distinct nodes. Otherwise (a range straddling scenes or spread too far)
// each particle reduces straight into global memory.
//
// The contribution of a particle with coefficients (c, M) to node x_i at
// offset dpos = x_i - x_p = (o - f) dx (o = the node's offset in the stencil,
// f = the particle's fractional position) is  W * (c + M dpos)  per value;
// P2G's first value (mass) has no dpos term. The record stores the same
// affine map in the node offset o: c + M dpos = c' + M' o with M' = M dx and
// c' = c - M' f, so that step 2 needs no per-particle offset arithmetic.
#pragma once

#include <climits>

#include "common.cuh"

namespace mpm {

constexpr int kTileCap = 1280;          // nodes (and cells) per tile (static shared memory <= 48 KB)
constexpr int kRecF4 = 5;               // float4 per particle record
// Resident threads per SM the G2P adjoint kernel is compiled for (3 CTAs of
// 256 or 6 of 128: at most 85 registers a thread, and 3 x 47 KB of shared
// memory; left to itself the compiler takes 118 registers and 2 CTAs), and,
// as a launch choice for the fused step and the G2P adjoint, 4 CTAs of 256
// at 64 registers, which needs the SM's shared memory carved out at its
// maximum (4 x 47 KB).
constexpr int kScatterResidentThreads = 768;
constexpr int kScatterResidentThreadsHigh = 1024;

// record (5 x float4): (f.x, f.y, w_z0, w_z1) (c_m, c'0, c'1, c'2) then the columns
// of M' with a zero in front, (0, M'_0j, M'_1j, M'_2j) for j = 0, 1, 2;
// value v (vector part) = c'_v + M'_v . o; P2G adds a mass value c_m.
// NT = threads per CTA = particles per CTA (one each)
// 128-byte aligned: the node accumulators double as the landing area of a
// tensor-copy (TMA) of grid values before the scatter uses them.
template <int NT>
struct alignas(128) ScatterTile {
  float acc[4][kTileCap];
  int cnt[kTileCap];
  float4 rec[NT * kRecF4];
  int occ[NT];  // occupied cells
  int red[2][4][NT / 32];
  int box[11];  // ox oy oz ex ey ez scene mode ncell nvalid nocc
  float inv[4];  // 1 / ez, 1 / (ey ez), 1 / cz, 1 / (cy cz) for div_small
};

// q = a / d for 0 <= a < 2^20 and 0 < d < 2^10 from a float reciprocal of d
// (inv = 1/d rounded): the float quotient is within 1 of the exact one, and
// the remainder test corrects it. Replaces the integer division sequence
// where tile indices are decoded.
__device__ inline int div_small(int a, int d, float inv) {
  int q = __float2int_rz(__int2float_rn(a) * inv);
  const int r = a - q * d;
  q += int(r >= d) - int(r < 0);
  return q;
}

// Block-wide bounding box of the stencil origins and tile decision. Every
// thread of the CTA must call it. On return the tile accumulators and cell
// counts are zero when the tile is used.
template <int NT>
__device__ inline void scatter_setup(ScatterTile<NT>& T, bool valid, const int* base, int scene) {
  const int nvalid = __syncthreads_count(valid);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int vmin[4], vmax[4];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    vmin[d] = valid ? base[d] : INT_MAX;
    vmax[d] = valid ? base[d] : INT_MIN;
  }
  vmin[3] = valid ? scene : INT_MAX;
  vmax[3] = valid ? scene : INT_MIN;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    int mn = __reduce_min_sync(0xffffffffu, vmin[d]);
    int mx = __reduce_max_sync(0xffffffffu, vmax[d]);
    if (lane == 0) {
      T.red[0][d][wid] = mn;
      T.red[1][d][wid] = mx;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nw = blockDim.x >> 5;
    int mn[4], mx[4];
    for (int d = 0; d < 4; ++d) {
      mn[d] = INT_MAX;
      mx[d] = INT_MIN;
      for (int w = 0; w < nw; ++w) {
        mn[d] = min(mn[d], T.red[0][d][w]);
        mx[d] = max(mx[d], T.red[1][d][w]);
      }
    }
    bool any = mn[3] != INT_MAX;
    long long cx = any ? (long long)mx[0] - mn[0] + 1 : 0, cy = any ? (long long)mx[1] - mn[1] + 1 : 0,
              cz = any ? (long long)mx[2] - mn[2] + 1 : 0;
    long long nodes = (cx + 2) * (cy + 2) * (cz + 2);
    T.box[0] = mn[0];
    T.box[1] = mn[1];
    T.box[2] = mn[2];
    T.box[3] = int(cx + 2);
    T.box[4] = int(cy + 2);
    T.box[5] = int(cz + 2);
    T.box[6] = mn[3];
    T.box[7] = (any && mn[3] == mx[3] && nodes <= kTileCap) ? 1 : 0;
    T.box[8] = int(cx * cy * cz);
    T.box[9] = nvalid;
    T.box[10] = 0;
    T.inv[0] = __frcp_rn(float(cz + 2));
    T.inv[1] = __frcp_rn(float((cy + 2) * (cz + 2)));
    T.inv[2] = __frcp_rn(float(cz > 0 ? cz : 1));
    T.inv[3] = __frcp_rn(float(cy * cz > 0 ? cy * cz : 1));
  }
  __syncthreads();
  if (T.box[7]) {
    int nt = T.box[3] * T.box[4] * T.box[5];
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
      T.acc[0][t] = 0.0f;
      T.acc[1][t] = 0.0f;
      T.acc[2][t] = 0.0f;
      T.acc[3][t] = 0.0f;
    }
    for (int t = threadIdx.x; t < T.box[8]; t += blockDim.x) T.cnt[t] = 0;
  }
  __syncthreads();
}

template <int NT>
__device__ inline int cell_of(const ScatterTile<NT>& T, const int* base) {
  int cy = T.box[4] - 2, cz = T.box[5] - 2;
  return ((base[0] - T.box[0]) * cy + (base[1] - T.box[1])) * cz + (base[2] - T.box[2]);
}

// Exclusive scan of the cell counts in place (every thread must call it).
template <int NT>
__device__ inline void scan_cells(ScatterTile<NT>& T) {
  __shared__ int wsum[NT / 32];
  const int n = T.box[8];
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int lo = threadIdx.x * per;
  int s = 0;
  for (int i = 0; i < per; ++i)
    if (lo + i < n) s += T.cnt[lo + i];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  int pre = x - s;
  for (int w = 0; w < wid; ++w) pre += wsum[w];
  for (int i = 0; i < per; ++i)
    if (lo + i < n) {
      int c = T.cnt[lo + i];
      T.cnt[lo + i] = pre;
      pre += c;
      if (c > 0) T.occ[atomicAdd(&T.box[10], 1)] = lo + i;
    }
  __syncthreads();
}

// Phase 1 (tile mode): place this particle's record, sorted by cell.
// rank = the value returned by atomicAdd on the cell count.
template <int NT>
__device__ inline int scatter_count(ScatterTile<NT>& T, bool valid, const int* base) {
  if (!valid) return -1;
  return atomicAdd(&T.cnt[cell_of(T, base)], 1);
}
template <int NT>
__device__ inline float4* scatter_slot(ScatterTile<NT>& T, const int* base, int rank) {
  return T.rec + (T.cnt[cell_of(T, base)] + rank) * kRecF4;
}

// Phase 1 (tile mode): write the record of a particle with stencil sc
// (fractional position f, weights w), mass value c_m and per-value
// coefficients (c, M) (M row-major, 3 x 3) at its cell-sorted slot. The values
// are laid out as two pairs, (mass, v0) and (v1, v2), each in one half of a
// float4, so that step 2 accumulates them with packed two-lane FP32
// instructions; the mass has no offset term (zero M' entries). The z weights
// of offsets 0 and 1 replace f_z (the third is 1 minus their sum).
// scatter_record_affine takes the coefficients already in the node-offset
// form (c', M').
template <int NT>
__device__ inline void scatter_record_affine(ScatterTile<NT>& T, int rank, const Stencil& sc, float cm,
                                             const float* cp, const float* Md) {
  float4* r = scatter_slot(T, sc.base, rank);
  r[0] = make_float4(sc.f[0], sc.f[1], sc.w[2][0], sc.w[2][1]);
  r[1] = make_float4(cm, cp[0], cp[1], cp[2]);
  r[2] = make_float4(0.0f, Md[0], Md[3], Md[6]);
  r[3] = make_float4(0.0f, Md[1], Md[4], Md[7]);
  r[4] = make_float4(0.0f, Md[2], Md[5], Md[8]);
}
template <int NT>
__device__ inline void scatter_record(ScatterTile<NT>& T, int rank, const Stencil& sc, float cm,
                                      const float* c, const float* M, float dx) {
  const float* f = sc.f;
  float Md[9], cp[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) Md[k] = M[k] * dx;
#pragma unroll
  for (int v = 0; v < 3; ++v) cp[v] = c[v] - (Md[3 * v] * f[0] + Md[3 * v + 1] * f[1] + Md[3 * v + 2] * f[2]);
  scatter_record_affine(T, rank, sc, cm, cp, Md);
}

// Quadratic B-spline weight of stencil offset o as a polynomial in the
// fractional position f in [0.5, 1.5): w_o(f) = k0 + k1 f + k2 f^2, from
// w_0 = (1.5 - f)^2 / 2, w_1 = 3/4 - (f - 1)^2, w_2 = (f - 0.5)^2 / 2.
__device__ inline void spline_poly(int o, float& k0, float& k1, float& k2) {
  k0 = o == 0 ? 1.125f : (o == 1 ? -0.25f : 0.125f);
  k1 = o == 0 ? -1.5f : (o == 1 ? 2.0f : -0.5f);
  k2 = o == 1 ? -1.0f : 0.5f;
}

// Phase 2 (tile mode, every thread must call it): per (occupied cell, o_x,
// o_y) item, accumulate the cell's particles into its 3 nodes (o_z = 0, 1, 2)
// in registers and add them to the tile. kMass: 4 values (mass first), else
// the 3 vector values (the record's mass slot is zero and is not added).
// The values travel as the pairs (mass, v0) and (v1, v2) through packed
// two-lane FP32 fused multiply-adds and adds (per lane the same rounding as
// the scalar fmaf and add).
template <bool kMass, int NT>
__device__ inline void scatter_accumulate(ScatterTile<NT>& T) {
  const int ncell = T.box[8], nocc = T.box[10];
  const int cy = T.box[4] - 2, cz = T.box[5] - 2;
  const int ey = T.box[4], ez = T.box[5];
  for (int item = threadIdx.x; item < 9 * nocc; item += blockDim.x) {
    const int oc = item / 9, sub = item - 9 * oc;
    const int oa = sub / 3, ob = sub - 3 * oa;
    const int c = T.occ[oc];
    const int start = T.cnt[c];
    const int end = (c + 1 < ncell) ? T.cnt[c + 1] : T.box[9];
    float ka0, ka1, ka2, kb0, kb1, kb2;
    spline_poly(oa, ka0, ka1, ka2);
    spline_poly(ob, kb0, kb1, kb2);
    const float2 k0 = make_float2(ka0, kb0), k1 = make_float2(ka1, kb1), k2 = make_float2(ka2, kb2);
    const float2 fa = make_float2(float(oa), float(oa)), fb = make_float2(float(ob), float(ob));
    float2 acc[3][2];
#pragma unroll
    for (int q = 0; q < 3; ++q) acc[q][0] = acc[q][1] = make_float2(0.0f, 0.0f);
    for (int s = start; s < end; ++s) {
      const float4* r = T.rec + s * kRecF4;
      const float4 r0 = r[0], r1 = r[1], m0 = r[2], m1 = r[3], m2 = r[4];
      const float2 fxy = make_float2(r0.x, r0.y);
      const float2 wab = __ffma2_rn(__ffma2_rn(k2, fxy, k1), fxy, k0);  // (w_x(o_a), w_y(o_b))
      const float wxy = wab.x * wab.y;
      const float2 W01 = __fmul2_rn(make_float2(wxy, wxy), make_float2(r0.z, r0.w));
      const float W[3] = {W01.x, W01.y, wxy - W01.x - W01.y};
      // value pairs at o_z = 0, stepped by the third column of M' per unit o_z
      float2 val[2] = {__ffma2_rn(make_float2(m1.x, m1.y), fb,
                                  __ffma2_rn(make_float2(m0.x, m0.y), fa, make_float2(r1.x, r1.y))),
                       __ffma2_rn(make_float2(m1.z, m1.w), fb,
                                  __ffma2_rn(make_float2(m0.z, m0.w), fa, make_float2(r1.z, r1.w)))};
      const float2 st[2] = {make_float2(m2.x, m2.y), make_float2(m2.z, m2.w)};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float2 w = make_float2(W[q], W[q]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          acc[q][h] = __ffma2_rn(w, val[h], acc[q][h]);
          if (q < 2) val[h] = __fadd2_rn(val[h], st[h]);
        }
      }
    }
    const int ci = div_small(c, cy * cz, T.inv[3]);
    const int cjk = c - ci * (cy * cz);
    const int cj = div_small(cjk, cz, T.inv[2]);
    const int ck = cjk - cj * cz;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int t = ((ci + oa) * ey + (cj + ob)) * ez + (ck + q);
      if (kMass) {
        atomicAdd(&T.acc[0][t], acc[q][0].x);
        atomicAdd(&T.acc[1][t], acc[q][0].y);
        atomicAdd(&T.acc[2][t], acc[q][1].x);
        atomicAdd(&T.acc[3][t], acc[q][1].y);
      } else {
        atomicAdd(&T.acc[0][t], acc[q][0].y);
        atomicAdd(&T.acc[1][t], acc[q][1].x);
        atomicAdd(&T.acc[2][t], acc[q][1].y);
      }
    }
  }
}

// Activate grid block b: the first caller to set its flag appends it to the
// active-block list (the grid update clears the flag again).
__device__ inline void activate_block(int* __restrict__ flags, int* __restrict__ list,
                                      int* __restrict__ count, long long b) {
  if (flags[b] == 0 && atomicExch(&flags[b], 1) == 0) list[atomicAdd(count, 1)] = int(b);
}

// Flush the tile to global memory (every thread must call it). If `flags` is
// given, activates the grid blocks the tile covers.
template <int NT>
__device__ inline void scatter_flush(ScatterTile<NT>& T, float4* __restrict__ grid, const Params& P,
                                     int* __restrict__ flags, int* __restrict__ list,
                                     int* __restrict__ count) {
  __syncthreads();
  if (!T.box[7]) return;
  const int ox = T.box[0], oy = T.box[1], oz = T.box[2];
  const int ex = T.box[3], ey = T.box[4], ez = T.box[5], sc = T.box[6];
  const int nt = ex * ey * ez;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    float a = T.acc[0][t], b = T.acc[1][t], c = T.acc[2][t], d = T.acc[3][t];
    if (a != 0.0f || b != 0.0f || c != 0.0f || d != 0.0f) {
      const int ti = div_small(t, ey * ez, T.inv[1]);
      const int tjk = t - ti * (ey * ez);
      const int tj = div_small(tjk, ez, T.inv[0]);
      red_add_v4(grid + node_index(P, sc, ox + ti, oy + tj, oz + tjk - tj * ez), a, b, c, d);
    }
  }
  if (flags) {
    int bx0 = ox / kBlockEdge, by0 = oy / kBlockEdge, bz0 = oz / kBlockEdge;
    int nbx = (ox + ex - 1) / kBlockEdge - bx0 + 1;
    int nby = (oy + ey - 1) / kBlockEdge - by0 + 1;
    int nbz = (oz + ez - 1) / kBlockEdge - bz0 + 1;
    int nbt = nbx * nby * nbz;
    if (threadIdx.x < nbt) {
      const float inv_yz = __frcp_rn(float(nby * nbz)), inv_z = __frcp_rn(float(nbz));
      for (int t = threadIdx.x; t < nbt; t += blockDim.x) {
        const int tx = div_small(t, nby * nbz, inv_yz);
        const int tyz = t - tx * (nby * nbz);
        const int ty = div_small(tyz, nbz, inv_z);
        const int bx = bx0 + tx, by = by0 + ty, bz = bz0 + tyz - ty * nbz;
        activate_block(flags, list, count, (long long)sc * P.NB + (bx * P.nb + by) * P.nb + bz);
      }
    }
  }
}

// Activate the blocks of one particle's stencil (used when the tile is off).
__device__ inline void mark_stencil_blocks(const Params& P, int scene, const int* base,
                                           int* __restrict__ flags, int* __restrict__ list,
                                           int* __restrict__ count) {
  int b0[3], b1[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    b0[d] = base[d] / kBlockEdge;
    b1[d] = (base[d] + 2) / kBlockEdge;
  }
  for (int bx = b0[0]; bx <= b1[0]; ++bx)
    for (int by = b0[1]; by <= b1[1]; ++by)
      for (int bz = b0[2]; bz <= b1[2]; ++bz)
        activate_block(flags, list, count, (long long)scene * P.NB + (bx * P.nb + by) * P.nb + bz);
}

}  // namespace mpm
