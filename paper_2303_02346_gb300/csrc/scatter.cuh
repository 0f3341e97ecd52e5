// Particle-to-grid scatter through a shared-memory tile.
//
// A CTA owns a contiguous range of particles that the block sort keeps
// spatially compact. It reduces the bounding box of their stencil origins;
// if the box (plus the 3-node stencil) fits in the tile and all particles
// belong to one scene, every particle adds its 27 node contributions into
// shared memory, and the CTA then flushes each touched node with one global
// float4 vector reduction. Otherwise (a range that straddles scenes or spread
// out too far) each particle reduces straight into global memory.
#pragma once

#include <climits>

#include "common.cuh"

namespace mpm {

constexpr int kTileCap = 1024;     // nodes per tile (4 x 4 KB of shared memory)
constexpr int kScatterThreads = 256;

struct Tile {
  float a[kTileCap], b[kTileCap], c[kTileCap], d[kTileCap];
  int red[2][8][kScatterThreads / 32];
  int box[8];  // ox, oy, oz, ex, ey, ez, scene, mode
};

// Block-wide setup. Every thread of the CTA must call it.
__device__ inline void tile_setup(Tile& T, bool valid, const int* base, int scene) {
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
    int ex = mx[0] - mn[0] + 3, ey = mx[1] - mn[1] + 3, ez = mx[2] - mn[2] + 3;
    bool any = mn[3] != INT_MAX;
    long long vol = (long long)ex * ey * ez;
    T.box[0] = mn[0];
    T.box[1] = mn[1];
    T.box[2] = mn[2];
    T.box[3] = ex;
    T.box[4] = ey;
    T.box[5] = ez;
    T.box[6] = mn[3];
    T.box[7] = (any && mn[3] == mx[3] && vol <= kTileCap) ? 1 : 0;
  }
  __syncthreads();
  if (T.box[7]) {
    int nt = T.box[3] * T.box[4] * T.box[5];
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
      T.a[t] = 0.0f;
      T.b[t] = 0.0f;
      T.c[t] = 0.0f;
      T.d[t] = 0.0f;
    }
  }
  __syncthreads();
}

// Add (va, vb, vc, vd) to node (i, j, k) of `scene`. kFour = false skips the 4th
// component (it is then treated as 0).
template <bool kFour>
__device__ inline void tile_add(Tile& T, float4* __restrict__ grid, const Params& P, int scene,
                                int i, int j, int k, float va, float vb, float vc, float vd) {
  if (T.box[7]) {
    int t = ((i - T.box[0]) * T.box[4] + (j - T.box[1])) * T.box[5] + (k - T.box[2]);
    atomicAdd(&T.a[t], va);
    atomicAdd(&T.b[t], vb);
    atomicAdd(&T.c[t], vc);
    if (kFour) atomicAdd(&T.d[t], vd);
  } else {
    red_add_v4(grid + node_index(P, scene, i, j, k), va, vb, vc, kFour ? vd : 0.0f);
  }
}

// Flush the tile to global memory (every thread must call it). If `flags` is
// given, marks the grid blocks the tile covers as active.
__device__ inline void tile_flush(Tile& T, float4* __restrict__ grid, const Params& P,
                                  uint8_t* __restrict__ flags) {
  __syncthreads();
  if (!T.box[7]) return;
  int ox = T.box[0], oy = T.box[1], oz = T.box[2];
  int ex = T.box[3], ey = T.box[4], ez = T.box[5], sc = T.box[6];
  int nt = ex * ey * ez;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    float a = T.a[t], b = T.b[t], c = T.c[t], d = T.d[t];
    if (a != 0.0f || b != 0.0f || c != 0.0f || d != 0.0f) {
      int i = ox + t / (ey * ez);
      int j = oy + (t / ez) % ey;
      int k = oz + t % ez;
      red_add_v4(grid + node_index(P, sc, i, j, k), a, b, c, d);
    }
  }
  if (flags) {
    int bx0 = ox / kBlockEdge, by0 = oy / kBlockEdge, bz0 = oz / kBlockEdge;
    int nbx = (ox + ex - 1) / kBlockEdge - bx0 + 1;
    int nby = (oy + ey - 1) / kBlockEdge - by0 + 1;
    int nbz = (oz + ez - 1) / kBlockEdge - bz0 + 1;
    int nbt = nbx * nby * nbz;
    for (int t = threadIdx.x; t < nbt; t += blockDim.x) {
      int bx = bx0 + t / (nby * nbz), by = by0 + (t / nbz) % nby, bz = bz0 + t % nbz;
      flags[(long long)sc * P.NB + (bx * P.nb + by) * P.nb + bz] = 1;
    }
  }
}

// Mark the blocks of one particle's stencil (used when the tile is off).
__device__ inline void mark_stencil_blocks(const Params& P, int scene, const int* base,
                                           uint8_t* __restrict__ flags) {
  int b0[3], b1[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    b0[d] = base[d] / kBlockEdge;
    b1[d] = (base[d] + 2) / kBlockEdge;
  }
  for (int bx = b0[0]; bx <= b1[0]; ++bx)
    for (int by = b0[1]; by <= b1[1]; ++by)
      for (int bz = b0[2]; bz <= b1[2]; ++bz)
        flags[(long long)scene * P.NB + (bx * P.nb + by) * P.nb + bz] = 1;
}

}  // namespace mpm
