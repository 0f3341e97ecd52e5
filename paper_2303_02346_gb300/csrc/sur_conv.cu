// 3x3x3 convolution, C = 32 -> 32 channels, as an implicit GEMM on the
// 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// tensor memory).
//
// A UMMA of M = 128, K = 16 costs the same issue time for every N up to 128,
// so the convolution is arranged to give N = 128 instead of the 32 output
// channels. Per tile of 126 output rows p0 .. p0 + 125 (padded row layout of
// sur_kernels.h) and per tap pair (a, b), one UMMA chain computes
//   D[(c, o)][j] += sum_q W[a][b][c][o][q] x[p0 - 1 + j + (a-1) P2 + (b-1) P1][q]
// with M = 128 rows (c = 0..2 the third tap index, o the output channel; rows
// 96..127 are zero), N = 128 input rows j, K = 32 input channels: the weights
// are the A operand, held in tensor memory for the whole kernel, and the input
// rows, shifted by the pair's constant offset, the B operand in shared memory.
// All 9 pairs accumulate into the same TMEM tile (18 UMMAs of 128 x 128 x 16
// per tile instead of 54 of 128 x 32 x 16), and the epilogue adds the three c
// rows at column shifts 0, 1, 2:
//   out[p0 + l][o] = D[(0, o)][l] + D[(1, o)][l + 1] + D[(2, o)][l + 2].
//
// Tiles march along i (one column of 126 rows of each i-plane at a time), so
// the three input slabs of tap plane a = 0, 1, 2 of tile i are the slabs of
// planes i-1, i, i+1 and each step loads one new slab (4 channel groups x
// (128 + 2 P1) rows, bulk asynchronous copies) into a ring of kRing slots.
// Work item = (frame, 8 consecutive planes, column); items are distributed
// round-robin over persistent CTAs (one per SM). Keeping the weights in
// tensor memory leaves shared-memory bandwidth to the B operand and the
// epilogue, which together bound the kernel.
//
// Tensor memory (512 columns): columns 0..143 the weights of the 9 pairs (16
// columns of two BF16 each per pair and lane), 256..511 two 128 x 128 FP32
// accumulators.
//
// Warp roles (416 threads):
//   warp 0       producer: the slab ring
//   warp 1       allocates the tensor memory and one lane issues the UMMAs,
//                committing to "accumulator full" and "slab free" mbarriers
//   warps 2, 4, 5  readers: warp w copies TMEM lanes 32 (w % 4) .. +31 (rows
//                c = w % 4) of a finished accumulator into one of two padded
//                shared-memory tiles
//   warps 3, 6-12 finishers: each pair of threads completes one output row of
//                a tile (16 of its 32 channels each):
//                shifted sum of the three c rows, bias, relu / residual /
//                relu-mask, BF16 rounding, coalesced 16-byte stores; the
//                residual / mask rows are loaded before the tile is awaited
// UMMAs of tile T + 1, the reader copy of tile T and the finishing of tile
// T - 1 overlap. Every wait is a bounded mbarrier wait (sur_ptx.cuh).
#include <cuda_bf16.h>

#include "sur_kernels.h"
#include "sur_ptx.cuh"

namespace sur {
namespace {

constexpr int kRing = 6;
// finisher warps: 4 x (kFinWarps / 4) threads per output row, each finishing
// kFinGroups of the 4 groups of 8 output channels
constexpr int kFinWarps = 8;
constexpr int kFinGroups = 16 / kFinWarps;
constexpr int kThreads = (5 + kFinWarps) * 32;
constexpr int kAcc = 2;
constexpr int kRed = 2;  // shared-memory tiles between readers and finishers
constexpr uint32_t kAccCol = 256;  // first TMEM column of the accumulators
constexpr uint32_t kTmemCols = 512;
// The shared-memory tile between readers and finishers holds, per tap c and
// accumulator column, the 32 output channels in a row of kRedRow floats (4 of
// padding: consecutive columns start 4 banks apart, so the finishers' 16-byte
// loads of 8 consecutive columns hit distinct banks).
constexpr int kRedRow = 36;
constexpr int kRedTile = 3 * kConvN * kRedRow;  // floats per tile
constexpr uint32_t kIdesc = idesc_bf16_f32(128, kConvN);

__device__ __forceinline__ void unpack8(const uint4& u, float (&f)[8]) {
  const __nv_bfloat162* p = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float2 t = __bfloat1622float2(p[i]);
    f[2 * i] = t.x;
    f[2 * i + 1] = t.y;
  }
}

__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
  uint4 u;
  __nv_bfloat162* p = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) p[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
  return u;
}

struct Smem {
  uint8_t* ring;    // kRing slabs of 4 x SR x 16 bytes
  float* red;       // kRed x 3 x kConvN x kRedRow
  float* bias;      // 32
  uint64_t* bars;   // full[kRing], empty[kRing], acc_full[kAcc], acc_empty[kAcc], red_full[kRed], red_empty[kRed]
  uint32_t* tmem_slot;
  int* abort_flag;
};

constexpr int kBars = 2 * kRing + 2 * kAcc + 2 * kRed;

__host__ __device__ inline int slab_rows(const SurGeom& g) { return kConvN + 2 * g.P1; }

__device__ __forceinline__ Smem carve(uint8_t* base, const SurGeom& g) {
  Smem s;
  size_t off = 0;
  s.ring = base + off;
  off += static_cast<size_t>(kRing) * 4 * slab_rows(g) * 16;
  s.red = reinterpret_cast<float*>(base + off);
  off += static_cast<size_t>(kRed) * kRedTile * 4;
  s.bias = reinterpret_cast<float*>(base + off);
  off += 128;
  s.bars = reinterpret_cast<uint64_t*>(base + off);
  off += 8 * kBars;
  s.tmem_slot = reinterpret_cast<uint32_t*>(base + off);
  s.abort_flag = reinterpret_cast<int*>(base + off + 4);
  return s;
}

struct Item {
  int f, k0, kn, c;  // frame, first plane index, planes, column
};

__device__ __forceinline__ Item item_of(int it, const SurGeom& g) {
  const int nc = (g.P2 + kConvW - 1) / kConvW;
  const int nch = (g.n + kConvChunk - 1) / kConvChunk;
  Item r;
  r.c = it % nc;
  const int rest = it / nc;
  const int kc = rest % nch;
  r.f = rest / nch;
  r.k0 = kc * kConvChunk;
  r.kn = min(kConvChunk, g.n - r.k0);
  return r;
}

__global__ void __launch_bounds__(kThreads, 1) conv3_umma_kernel(ConvArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const SurGeom g = a.g;
  Smem s = carve(smem_raw, g);
  uint64_t* full = s.bars;
  uint64_t* empty = s.bars + kRing;
  uint64_t* acc_full = s.bars + 2 * kRing;
  uint64_t* acc_empty = s.bars + 2 * kRing + kAcc;
  uint64_t* red_full = s.bars + 2 * kRing + 2 * kAcc;
  uint64_t* red_empty = s.bars + 2 * kRing + 2 * kAcc + kRed;
  volatile int* abort_flag = s.abort_flag;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n_items = a.batch * ((g.n + kConvChunk - 1) / kConvChunk) * ((g.P2 + kConvW - 1) / kConvW);
  const int SR = slab_rows(g);
  const uint32_t plane_bytes = static_cast<uint32_t>(SR) * 16;  // one channel group of one slab
  const uint32_t slab_bytes = 4 * plane_bytes;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kRing; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < kAcc; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 3);  // the three reader warps
    }
    for (int i = 0; i < kRed; ++i) {
      mbar_init(&red_full[i], 3);   // the three reader warps
      mbar_init(&red_empty[i], kFinWarps);  // the finisher warps
    }
    *s.abort_flag = 0;
    fence_barrier_init();
  }
  if (threadIdx.x < kC) s.bias[threadIdx.x] = a.bias ? a.bias[threadIdx.x] : 0.0f;
  if (warp == 1) {
    tmem_alloc(s.tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s.tmem_slot;
  if (warp >= 2 && warp <= 5) {
    // weights into tensor memory: lane quarter q holds rows 32 q .. 32 q + 31
    const int q = warp & 3, m = q * 32 + lane;
    const uint4* src = reinterpret_cast<const uint4*>(a.w) + static_cast<size_t>(m) * 9 * 4;
#pragma unroll 1
    for (int p = 0; p < 9; ++p) {
      uint32_t r[16];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint4 u = __ldg(src + p * 4 + i);
        const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) r[i * 4 + e] = a.apack ? __byte_perm(w4[e], 0, 0x1032) : w4[e];
      }
      tmem_st16(tmem + (static_cast<uint32_t>(q * 32) << 16) + p * 16, r);
    }
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  int issued_slabs = 0, issued_tiles = 0;
  if (warp == 0) {
    if (lane == 0) {
      int S = 0;
      bool ok = true;
      for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
        const Item I = item_of(it, g);
        for (int m = 0; m < I.kn + 2; ++m, ++S) {
          const int slot = S % kRing;
          if (S >= kRing && !mbar_wait(&empty[slot], ((S / kRing) - 1) & 1, abort_flag)) {
            atomicOr(a.err, kErrTimeout);
            *s.abort_flag = 1;
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[slot], slab_bytes);
          const long long row = g.G + I.f * g.V + static_cast<long long>(I.k0 + m) * g.P2 +
                                static_cast<long long>(I.c) * kConvW - (g.P1 + 1);
          uint8_t* dst = s.ring + static_cast<size_t>(slot) * slab_bytes;
#pragma unroll 1
          for (int c = 0; c < 4; ++c)
            bulk_g2s(dst + c * plane_bytes, a.in + (c * g.plane + row) * 8, plane_bytes, &full[slot]);
          issued_slabs = S + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      const uint32_t ring = smem_u32(s.ring);
      // The B descriptors of a tile differ from the ring's only in the start
      // address field (address / 16, 14 bits: every shared address here is
      // below 2^18 bytes), so each is the ring's descriptor plus a field
      // offset: (slab, dy, ks) -> slab * slab_bytes + 2 ks plane_bytes + dy P1 16.
      // The issue loop then costs a few instructions per UMMA.
      const uint64_t desc_ring = smem_desc(ring, plane_bytes, 128);
      uint32_t boff[6];
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) boff[dy * 2 + ks] = (2 * ks * plane_bytes + dy * g.P1 * 16) >> 4;
      const uint32_t slab16 = slab_bytes >> 4;
      int S0 = 0, T = 0;
      for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
        const Item I = item_of(it, g);
        int waited = 0;
        for (int k = 0; ok && k < I.kn; ++k, ++T) {
          while (ok && waited <= k + 2) {
            const int S = S0 + waited;
            ok = mbar_wait(&full[S % kRing], (S / kRing) & 1, abort_flag);
            ++waited;
          }
          const int buf = T % kAcc;
          if (ok && T >= kAcc) ok = mbar_wait(&acc_empty[buf], ((T / kAcc) - 1) & 1, abort_flag);
          if (!ok) {
            atomicOr(a.err, kErrTimeout);
            *s.abort_flag = 1;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + kAccCol + buf * kConvN;
          int sl[3];
          sl[0] = (S0 + k) % kRing;
          sl[1] = sl[0] + 1 == kRing ? 0 : sl[0] + 1;
          sl[2] = sl[1] + 1 == kRing ? 0 : sl[1] + 1;
#pragma unroll
          for (int dz = 0; dz < 3; ++dz) {
            const uint64_t ds = desc_ring + static_cast<uint64_t>(sl[dz] * slab16);
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
              const int grp = dz * 3 + dy;
#pragma unroll
              for (int ks = 0; ks < 2; ++ks)
                umma_bf16_ts(d, tmem + grp * 16 + ks * 8, ds + boff[dy * 2 + ks], kIdesc, (grp | ks) ? 1u : 0u);
            }
          }
          umma_commit(&acc_full[buf]);
          umma_commit(&empty[(S0 + k) % kRing]);  // plane k's slab is not read again
          issued_tiles = T + 1;
        }
        if (!ok) break;
        umma_commit(&empty[(S0 + I.kn) % kRing]);
        umma_commit(&empty[(S0 + I.kn + 1) % kRing]);
        S0 += I.kn + 2;
      }
    }
  } else if (warp == 2 || warp == 4 || warp == 5) {
    // readers: finished accumulator -> shared-memory tile
    const int q = warp & 3;  // TMEM lane quarter = tap c
    int T = 0;
    bool ok = true;
    for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
      const Item I = item_of(it, g);
      for (int k = 0; k < I.kn; ++k, ++T) {
        const int buf = T % kAcc, rb = T % kRed;
        ok = mbar_wait(&acc_full[buf], (T / kAcc) & 1, abort_flag);
        if (ok && T >= kRed) ok = mbar_wait(&red_empty[rb], ((T / kRed) - 1) & 1, abort_flag);
        ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
        if (!ok) {
          atomicOr(a.err, kErrTimeout);
          *s.abort_flag = 1;
          break;
        }
        tc_fence_after();
        // lane = output channel o: column j of this tap goes to row (q, j), entry o
        float* dst = s.red + static_cast<size_t>(rb) * kRedTile + q * kConvN * kRedRow + lane;
        // two 32-column loads in flight before each wait
#pragma unroll
        for (int cc = 0; cc < 4; cc += 2) {
          uint32_t v0[32], v1[32];
          const uint32_t src = tmem + (static_cast<uint32_t>(q * 32) << 16) + kAccCol + buf * kConvN + cc * 32;
          tmem_ld32(src, v0);
          tmem_ld32(src + 32, v1);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 32; ++e) dst[(cc * 32 + e) * kRedRow] = __uint_as_float(v0[e]);
#pragma unroll
          for (int e = 0; e < 32; ++e) dst[(cc * 32 + 32 + e) * kRedRow] = __uint_as_float(v1[e]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&acc_empty[buf]);
          mbar_arrive(&red_full[rb]);
        }
      }
    }
  } else {
    // finishers (warps 3 and 6 ..): output row t, channel groups c0 .. c0 + kFinGroups - 1
    const int fi = warp == 3 ? 0 : warp - 5;
    const int t = (fi % 4) * 32 + lane;  // 0..127
    const int c0 = (fi / 4) * kFinGroups;
    const int n = g.n;
    float4 bias4[2 * kFinGroups];
#pragma unroll
    for (int j = 0; j < 2 * kFinGroups; ++j) bias4[j] = reinterpret_cast<const float4*>(s.bias)[2 * c0 + j];
    // this thread's output row of tile (I, k) and whether it is an interior node
    auto row_of = [&](const Item& I, int k, long long& row) -> bool {
      const int off = I.c * kConvW + t;
      const int jj = off / g.P1, kk = off % g.P1;
      row = g.G + I.f * g.V + static_cast<long long>(I.k0 + k + 1) * g.P2 + off;
      return t < kConvW && off < g.P2 && jj >= 1 && jj <= n && kk >= 1 && kk <= n;
    };
    auto fetch = [&](bool mine, long long row, uint4 (&ad)[kFinGroups], uint4 (&mk)[kFinGroups]) {
#pragma unroll
      for (int c = 0; c < kFinGroups; ++c) {
        const long long eo = ((c0 + c) * g.plane + row) * 8;
        ad[c] = (mine && a.add) ? __ldg(reinterpret_cast<const uint4*>(a.add + eo)) : make_uint4(0, 0, 0, 0);
        mk[c] = (mine && a.mask) ? __ldg(reinterpret_cast<const uint4*>(a.mask + eo)) : make_uint4(0, 0, 0, 0);
      }
    };
    // the residual / mask rows of the next tile are loaded before this tile is
    // awaited and finished, so their latency overlaps a tile's work
    bool ok = true;
    int it = blockIdx.x, kn = 0;
    Item In;
    long long row_n = 0;
    bool mine_n = false;
    uint4 ad_n[kFinGroups], mk_n[kFinGroups];
    if (it < n_items) {
      In = item_of(it, g);
      mine_n = row_of(In, 0, row_n);
      fetch(mine_n, row_n, ad_n, mk_n);
    }
    for (int T = 0; ok && it < n_items; ++T) {
      {
        const long long row = row_n;
        const bool mine = mine_n;
        uint4 ad[kFinGroups], mk[kFinGroups];
#pragma unroll
        for (int c = 0; c < kFinGroups; ++c) {
          ad[c] = ad_n[c];
          mk[c] = mk_n[c];
        }
        if (++kn == In.kn) {
          kn = 0;
          it += gridDim.x;
          if (it < n_items) In = item_of(it, g);
        }
        if (it < n_items) {
          mine_n = row_of(In, kn, row_n);
          fetch(mine_n, row_n, ad_n, mk_n);
        }
        const int rb = T % kRed;
        ok = mbar_wait(&red_full[rb], (T / kRed) & 1, abort_flag);
        if (!ok) {
          atomicOr(a.err, kErrTimeout);
          *s.abort_flag = 1;
          break;
        }
        const float* red = s.red + static_cast<size_t>(rb) * kRedTile;
        if (mine) {
          // rows (tap, column): (0, t), (1, t + 1), (2, t + 2)
          const float4* r0 = reinterpret_cast<const float4*>(red + t * kRedRow) + 2 * c0;
          const float4* r1 = reinterpret_cast<const float4*>(red + (kConvN + t + 1) * kRedRow) + 2 * c0;
          const float4* r2 = reinterpret_cast<const float4*>(red + (2 * kConvN + t + 2) * kRedRow) + 2 * c0;
#pragma unroll
          for (int c = 0; c < kFinGroups; ++c) {
            float o8[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float4 x0 = r0[2 * c + h], x1 = r1[2 * c + h], x2 = r2[2 * c + h];
              const float4 bb = bias4[2 * c + h];
              // (tap 0 + tap 1) + tap 2 + bias, lane pairs in packed two-lane adds
              const float2 lo = __fadd2_rn(__fadd2_rn(__fadd2_rn(make_float2(x0.x, x0.y), make_float2(x1.x, x1.y)),
                                                      make_float2(x2.x, x2.y)),
                                           make_float2(bb.x, bb.y));
              const float2 hi = __fadd2_rn(__fadd2_rn(__fadd2_rn(make_float2(x0.z, x0.w), make_float2(x1.z, x1.w)),
                                                      make_float2(x2.z, x2.w)),
                                           make_float2(bb.z, bb.w));
              o8[4 * h] = lo.x;
              o8[4 * h + 1] = lo.y;
              o8[4 * h + 2] = hi.x;
              o8[4 * h + 3] = hi.y;
            }
            if (a.relu) {
#pragma unroll
              for (int e = 0; e < 8; ++e) o8[e] = fmaxf(o8[e], 0.0f);
            }
            if (a.add) {
              float ad8[8];
              unpack8(ad[c], ad8);
#pragma unroll
              for (int e = 0; e < 8; ++e) o8[e] += ad8[e];
            }
            if (a.mask) {
              float mk8[8];
              unpack8(mk[c], mk8);
#pragma unroll
              for (int e = 0; e < 8; ++e) o8[e] = mk8[e] > 0.0f ? o8[e] : 0.0f;
            }
            *reinterpret_cast<uint4*>(a.out + ((c0 + c) * g.plane + row) * 8) = pack8(o8);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&red_empty[rb]);
      }
    }
  }

  // drain: no copy or UMMA may still target this CTA's shared or tensor memory
  if (warp == 0 && lane == 0 && issued_slabs > 0 && *abort_flag) {
    for (int S = (issued_slabs > kRing ? issued_slabs - kRing : 0); S < issued_slabs; ++S)
      mbar_wait(&full[S % kRing], (S / kRing) & 1, nullptr);
  }
  if (warp == 1 && lane == 0 && issued_tiles > 0 && *abort_flag) {
    const int T = issued_tiles - 1;
    mbar_wait(&acc_full[T % kAcc], (T / kAcc) & 1, nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// One CTA of 128 threads: D (128 x 32) = A (128 x 32) B^T (B: 32 x 32) on the
// tensor cores, two K = 16 steps. mode 0: both operands K-major in shared
// memory as in the convolution's B operand (core matrices of 8 rows x 8
// K-elements; M/N groups 128 B apart, K groups 2048 / 512 B apart). mode 1:
// both MN-major as in the weight gradient (core matrices of 8 K-rows x 8
// M-elements; MN groups 512 B apart, K groups 128 B apart), descriptors built
// with `opt` = mn_swap. mode 2: A in tensor memory as in the convolution (row m
// in lane m, K in columns 32.., two elements per column: element 2i in the low
// half when opt = 0, in the high half when opt = 1), B K-major. The shared
// allocation is 64 KB and every address either assignment of the two
// descriptor offsets could form stays below 10 KB.
__global__ void __launch_bounds__(128, 1)
    selftest_mma_kernel(const float* A, const float* B, float* D, int mode, int opt, int* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __nv_bfloat16* sa = reinterpret_cast<__nv_bfloat16*>(sm);
  __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(sm + 8192);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 49152);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + 49152 + 16);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  if (mode != 2) {
    for (int i = tid; i < 128 * 32; i += 128) {
      const int row = i / 32, k = i % 32;
      const int off = mode == 0 ? (k / 8) * 128 * 8 + row * 8 + (k % 8)
                                : ((row / 8) * 512 + (k / 8) * 128 + (k % 8) * 16) / 2 + (row % 8);
      sa[off] = __float2bfloat16_rn(A[i]);
    }
  }
  for (int i = tid; i < 32 * 32; i += 128) {
    const int nn = i / 32, k = i % 32;
    const int off = mode == 1 ? ((nn / 8) * 512 + (k / 8) * 128 + (k % 8) * 16) / 2 + (nn % 8)
                              : (k / 8) * 32 * 8 + nn * 8 + (k % 8);
    sb[off] = __float2bfloat16_rn(B[i]);
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(slot, 64);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (mode == 2) {
    // each warp writes the A rows of its lane quarter into columns 32..47
    const int m = warp * 32 + lane;
    uint32_t r[16];
    for (int c = 0; c < 16; ++c) {
      const uint32_t lo = __bfloat16_as_ushort(__float2bfloat16_rn(A[m * 32 + 2 * c]));
      const uint32_t hi = __bfloat16_as_ushort(__float2bfloat16_rn(A[m * 32 + 2 * c + 1]));
      r[c] = opt ? (hi | (lo << 16)) : (lo | (hi << 16));
    }
    tmem_st16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + 32, r);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    for (int ks = 0; ks < 2; ++ks) {
      if (mode == 2) {
        const uint64_t db = smem_desc(smem_u32(sb) + 2 * ks * 512, 512, 128);
        umma_bf16_ts(tmem, tmem + 32 + ks * 8, db, idesc_bf16_f32(128, 32), ks > 0);
      } else {
        uint64_t da, db;
        if (mode == 0) {
          da = smem_desc(smem_u32(sa) + 2 * ks * 2048, 2048, 128);
          db = smem_desc(smem_u32(sb) + 2 * ks * 512, 512, 128);
        } else {
          da = smem_desc_mn(smem_u32(sa) + ks * 256, 512, 128, opt);
          db = smem_desc_mn(smem_u32(sb) + ks * 256, 512, 128, opt);
        }
        umma_bf16(tmem, da, db, idesc_bf16_f32(128, 32, mode, mode), ks > 0);
      }
    }
    umma_commit(bar);
  }
  __syncwarp();
  const bool ok = mbar_wait(bar, 0, nullptr);
  if (!ok && lane == 0) atomicOr(err, kErrTimeout);
  __syncwarp();
  tc_fence_after();
  uint32_t v[32];
  tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16), v);
  tmem_wait_ld();
  const int row = warp * 32 + lane;
  for (int c = 0; c < 32; ++c) D[row * 32 + c] = ok ? __uint_as_float(v[c]) : 0.0f;
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 64);
  }
}

}  // namespace

size_t conv_smem_bytes(const SurGeom& g) {
  return static_cast<size_t>(kRing) * 4 * slab_rows(g) * 16 + static_cast<size_t>(kRed) * kRedTile * 4 +
         128 + 8 * kBars + 16;
}

cudaError_t launch_conv(const ConvArgs& a, int num_sms, cudaStream_t st) {
  const size_t smem = conv_smem_bytes(a.g);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(conv3_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(conv_smem_bytes(make_geom(64, 1))));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int n_items =
      a.batch * ((a.g.n + kConvChunk - 1) / kConvChunk) * ((a.g.P2 + kConvW - 1) / kConvW);
  const int grid = n_items < num_sms ? n_items : num_sms;
  if (grid <= 0) return cudaSuccess;
  conv3_umma_kernel<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t selftest_mma(const float* a, const float* b, float* d, int mode, int opt) {
  int* err = nullptr;
  cudaError_t e = cudaFuncSetAttribute(selftest_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
  if (e != cudaSuccess) return e;
  if ((e = cudaMalloc(&err, sizeof(int))) != cudaSuccess) return e;
  cudaMemset(err, 0, sizeof(int));
  selftest_mma_kernel<<<1, 128, 65536>>>(a, b, d, mode, opt, err);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(err);
  if (e == cudaSuccess && h) return cudaErrorTimeout;
  return e;
}

}  // namespace sur
