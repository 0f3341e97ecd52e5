// 3x3x3 convolution, C = 32 -> 32 channels, as an implicit GEMM on the
// 5th-generation tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// tensor memory).
//
// GEMM view: D[row][o] = sum_tap sum_q A_tap[row][q] W_tap[o][q] with M = 128
// output rows per tile, N = 32 output channels, K = 27 taps x 32 channels
// (54 UMMAs of 128 x 32 x 16 per tile). In the padded row layout of
// sur_kernels.h, A_tap is the run of input rows shifted by the tap's constant
// offset, so no im2col is built: a tile stages three slabs (one per tap plane
// a = 0..2) of kTile + 2 (P1 + 1) rows x 4 channel groups into shared memory
// with bulk asynchronous copies, and each tap's A descriptor points at the
// shifted row inside its slab (16-byte granularity, no swizzle). The 27 taps'
// weights (55 KB) stay resident in shared memory for the whole kernel.
//
// Persistent warp-specialised CTA (one per SM, 192 threads):
//   warp 0   producer: bulk copies of the slabs into a 3-stage ring
//   warp 1   allocates 64 TMEM columns (two 32-column accumulators) and one
//            lane issues the UMMAs, committing to "slab free" and "accumulator
//            full" mbarriers
//   warps 2-5  epilogue: TMEM -> registers (warp w reads lanes 32 (w % 4)..),
//            bias / relu / residual / relu-mask, BF16 rounding, coalesced stores
// The epilogue of tile j overlaps the UMMAs of tile j + 1 and the copies of
// tiles j + 1 .. j + 3. All waits are bounded (sur_ptx.cuh).
#include <cuda_bf16.h>

#include "sur_kernels.h"
#include "sur_ptx.cuh"

namespace sur {
namespace {

constexpr int kStages = 3;
constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 64;
constexpr uint32_t kIdesc = idesc_bf16_f32(kTile, kC);

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
  uint8_t* w;       // kWBytes
  uint8_t* slabs;   // kStages x 12 x SR x 16
  float* bias;      // 32
  uint64_t* bars;   // w_full, slab_full[3], slab_empty[3], acc_full[2], acc_empty[2]
  uint32_t* tmem_slot;
  int* abort_flag;
};

__device__ __forceinline__ Smem carve(uint8_t* base, int SR) {
  Smem s;
  s.w = base;
  s.slabs = base + kWBytes;
  size_t off = kWBytes + static_cast<size_t>(kStages) * 12 * SR * 16;
  s.bias = reinterpret_cast<float*>(base + off);
  off += 128;
  s.bars = reinterpret_cast<uint64_t*>(base + off);
  off += 8 * 16;
  s.tmem_slot = reinterpret_cast<uint32_t*>(base + off);
  s.abort_flag = reinterpret_cast<int*>(base + off + 4);
  return s;
}

__global__ void __launch_bounds__(kThreads, 1) conv3_umma_kernel(ConvArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const SurGeom g = a.g;
  Smem s = carve(smem_raw, g.SR);
  uint64_t* w_full = s.bars;
  uint64_t* slab_full = s.bars + 1;
  uint64_t* slab_empty = s.bars + 1 + kStages;
  uint64_t* acc_full = s.bars + 1 + 2 * kStages;
  uint64_t* acc_empty = s.bars + 3 + 2 * kStages;
  volatile int* abort_flag = s.abort_flag;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int total = a.batch * g.tpf;
  const uint32_t slab_bytes = static_cast<uint32_t>(g.SR) * 16;  // one channel group of one tap plane

  if (threadIdx.x == 0) {
    mbar_init(w_full, 1);
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&slab_full[i], 1);
      mbar_init(&slab_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);
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

  int issued_loads = 0, issued_mma = 0;
  if (warp == 0) {
    if (lane == 0) {
      // resident weights, then the slab ring
      mbar_arrive_expect_tx(w_full, kWBytes);
      bulk_g2s(s.w, a.w, kWBytes, w_full);
      int j = 0;
      for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++j) {
        const int st = j % kStages;
        if (j >= kStages && !mbar_wait(&slab_empty[st], ((j / kStages) - 1) & 1, abort_flag)) {
          atomicOr(a.err, kErrTimeout);
          *abort_flag = 1;
          break;
        }
        mbar_arrive_expect_tx(&slab_full[st], 12 * slab_bytes);
        const int f = tile / g.tpf, t = tile % g.tpf;
        const long long row0 = g.G + f * g.V + g.P2 + static_cast<long long>(t) * kTile - (g.P1 + 1);
        uint8_t* dst = s.slabs + static_cast<size_t>(st) * 12 * slab_bytes;
#pragma unroll 1
        for (int dz = 0; dz < 3; ++dz) {
          const long long r = row0 + static_cast<long long>(dz - 1) * g.P2;
#pragma unroll 1
          for (int c = 0; c < 4; ++c) {
            const __nv_bfloat16* src = a.in + (c * g.plane + r) * 8;
            bulk_g2s(dst + (dz * 4 + c) * slab_bytes, src, slab_bytes, &slab_full[st]);
          }
        }
        issued_loads = j + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = mbar_wait(w_full, 0, abort_flag);
      if (!ok) {
        atomicOr(a.err, kErrTimeout);
        *abort_flag = 1;
      }
      const uint32_t w_base = smem_u32(s.w);
      int j = 0;
      for (int tile = blockIdx.x; ok && tile < total; tile += gridDim.x, ++j) {
        const int st = j % kStages, acc = j & 1;
        if (!mbar_wait(&slab_full[st], (j / kStages) & 1, abort_flag) ||
            (j >= 2 && !mbar_wait(&acc_empty[acc], ((j >> 1) - 1) & 1, abort_flag))) {
          atomicOr(a.err, kErrTimeout);
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t slab = smem_u32(s.slabs + static_cast<size_t>(st) * 12 * slab_bytes);
        const uint32_t d = tmem + acc * kC;
        uint32_t accumulate = 0;
#pragma unroll 1
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll 1
          for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
              const int tap = dz * 9 + dy * 3 + dx;
              const uint32_t a_row = slab + dz * 4 * slab_bytes + (dy * g.P1 + dx) * 16;
#pragma unroll
              for (int ks = 0; ks < 2; ++ks) {
                const uint64_t da = smem_desc(a_row + 2 * ks * slab_bytes, slab_bytes, 128);
                const uint64_t db = smem_desc(w_base + tap * 2048 + 2 * ks * 512, 512, 128);
                umma_bf16(d, da, db, kIdesc, accumulate);
                accumulate = 1;
              }
            }
        umma_commit(&slab_empty[st]);
        umma_commit(&acc_full[acc]);
        issued_mma = j + 1;
      }
    }
  } else {
    // epilogue warps 2..5: the residual / mask rows of a tile are loaded before
    // its accumulator is awaited, so their latency overlaps the UMMAs
    const int q = warp & 3;
    const int r = q * 32 + lane;
    const int n = g.n;
    int j = 0;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++j) {
      const int acc = j & 1;
      const int f = tile / g.tpf, t = tile % g.tpf;
      const int p = g.P2 + t * kTile + r;  // frame-local padded row
      const int jj = (p / g.P1) % g.P1, kk = p % g.P1;
      const bool interior = p < (n + 1) * g.P2 && jj >= 1 && jj <= n && kk >= 1 && kk <= n;
      const long long row = g.G + f * g.V + p;
      uint4 ad[4], mk[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const long long off = (c * g.plane + row) * 8;
        ad[c] = (interior && a.add) ? __ldg(reinterpret_cast<const uint4*>(a.add + off)) : make_uint4(0, 0, 0, 0);
        mk[c] = (interior && a.mask) ? __ldg(reinterpret_cast<const uint4*>(a.mask + off)) : make_uint4(0, 0, 0, 0);
      }
      bool ok = mbar_wait(&acc_full[acc], (j >> 1) & 1, abort_flag);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      if (!ok) {
        atomicOr(a.err, kErrTimeout);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      uint32_t v[32];
      tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + acc * kC, v);
      tmem_wait_ld();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[acc]);
      if (!interior) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float o[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          o[e] = __uint_as_float(v[c * 8 + e]) + s.bias[c * 8 + e];
          if (a.relu) o[e] = fmaxf(o[e], 0.0f);
        }
        if (a.add) {
          float ad8[8];
          unpack8(ad[c], ad8);
#pragma unroll
          for (int e = 0; e < 8; ++e) o[e] += ad8[e];
        }
        if (a.mask) {
          float mk8[8];
          unpack8(mk[c], mk8);
#pragma unroll
          for (int e = 0; e < 8; ++e) o[e] = mk8[e] > 0.0f ? o[e] : 0.0f;
        }
        *reinterpret_cast<uint4*>(a.out + (c * g.plane + row) * 8) = pack8(o);
      }
    }
  }

  // drain: no copy or UMMA may still target this CTA's shared or tensor memory
  if (warp == 0 && lane == 0 && issued_loads > 0 && *abort_flag) {
    for (int j = (issued_loads > kStages ? issued_loads - kStages : 0); j < issued_loads; ++j)
      mbar_wait(&slab_full[j % kStages], (j / kStages) & 1, nullptr);
  }
  if (warp == 1 && lane == 0 && issued_mma > 0 && *abort_flag) {
    const int j = issued_mma - 1;
    mbar_wait(&acc_full[j & 1], (j >> 1) & 1, nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// One CTA of 128 threads: D (128 x 32) = A (128 x 32) B^T (B: 32 x 32) on the
// tensor cores, two K = 16 steps. mode 0: both operands K-major as in the
// convolution (core matrices of 8 rows x 8 K-elements; M groups 128 B apart, K
// groups 2048 / 512 B apart). mode 1: both MN-major as in the weight gradient
// (core matrices of 8 K-rows x 8 M-elements; MN groups 512 B apart, K groups
// 128 B apart), descriptors built with `mn_swap`. The allocation is 64 KB and
// every address either assignment of the two descriptor offsets could form
// stays below 10 KB.
__global__ void __launch_bounds__(128, 1)
    selftest_mma_kernel(const float* A, const float* B, float* D, int mode, int mn_swap, int* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __nv_bfloat16* sa = reinterpret_cast<__nv_bfloat16*>(sm);
  __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(sm + 8192);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 49152);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + 49152 + 16);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  for (int i = tid; i < 128 * 32; i += 128) {
    const int row = i / 32, k = i % 32;
    const int off = mode == 0 ? (k / 8) * 128 * 8 + row * 8 + (k % 8)
                              : ((row / 8) * 512 + (k / 8) * 128 + (k % 8) * 16) / 2 + (row % 8);
    sa[off] = __float2bfloat16_rn(A[i]);
  }
  for (int i = tid; i < 32 * 32; i += 128) {
    const int nn = i / 32, k = i % 32;
    const int off = mode == 0 ? (k / 8) * 32 * 8 + nn * 8 + (k % 8)
                              : ((nn / 8) * 512 + (k / 8) * 128 + (k % 8) * 16) / 2 + (nn % 8);
    sb[off] = __float2bfloat16_rn(B[i]);
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(slot, 32);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  if (tid == 0) {
    for (int ks = 0; ks < 2; ++ks) {
      uint64_t da, db;
      if (mode == 0) {
        da = smem_desc(smem_u32(sa) + 2 * ks * 2048, 2048, 128);
        db = smem_desc(smem_u32(sb) + 2 * ks * 512, 512, 128);
      } else {
        da = smem_desc_mn(smem_u32(sa) + ks * 256, 512, 128, mn_swap);
        db = smem_desc_mn(smem_u32(sb) + ks * 256, 512, 128, mn_swap);
      }
      umma_bf16(tmem, da, db, idesc_bf16_f32(128, 32, mode, mode), ks > 0);
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
    tmem_dealloc(tmem, 32);
  }
}

}  // namespace

cudaError_t launch_conv(const ConvArgs& a, int num_sms, cudaStream_t st) {
  const size_t smem = conv_smem_bytes(a.g, kStages);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(conv3_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(conv_smem_bytes(make_geom(64, 1), kStages)));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int total = a.batch * a.g.tpf;
  const int grid = total < num_sms ? total : num_sms;
  if (grid <= 0) return cudaSuccess;
  conv3_umma_kernel<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t selftest_mma(const float* a, const float* b, float* d, int mode, int mn_swap) {
  int* err = nullptr;
  cudaError_t e = cudaFuncSetAttribute(selftest_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
  if (e != cudaSuccess) return e;
  if ((e = cudaMalloc(&err, sizeof(int))) != cudaSuccess) return e;
  cudaMemset(err, 0, sizeof(int));
  selftest_mma_kernel<<<1, 128, 65536>>>(a, b, d, mode, mn_swap, err);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(err);
  if (e == cudaSuccess && h) return cudaErrorTimeout;
  return e;
}

}  // namespace sur
