// Weight and bias gradient of the 3x3x3 convolution on the tensor cores:
//   dW[a][b][c][o][q] = sum over rows u of gy[u][o] x[u + (a-1) P2 + (b-1) P1 + (c-1)][q]
//   db[o]             = sum_u gy[u][o]
// (u over every row of the padded layout; gy is zero outside the interior).
//
// GEMM view, K = rows of a sweep v: for each of the 3 taps c, one UMMA chain
// D_c[m][n] += sum_v A[m][v] B_c[v][n] with
//   M = 128: four row-shifted views of gy, A[(o8g, j, o8)][v] = gy[v + j P1][8 o8g + o8];
//   N = 96: the x rows of the three planes a, B_c[v][(a, q)] = x[v + (a-1) P2 + P1 + (c-1)][q].
// View j meets tap b = 2 - j (j = 3 is discarded), so one chain yields 9 taps:
// 3 chains of 128 x 96 x 16 UMMAs per 16 rows cover all 27. (A UMMA of M = 128
// costs the same issue time for any N up to 128, so N = 96 instead of 32
// triples the useful work per instruction.) Both operands are MN-major (K =
// consecutive 16-byte rows, M/N = the 8 channels inside a row), so the
// channel-planar activation layout is used as is: per stage, 4 bulk copies of
// 4 P1 rows of gy and 12 copies of K + 2 rows of x (planes a x channel groups,
// equally spaced, which is the N stride of B).
//
// Persistent warp-specialised CTA (192 threads, one per SM): warp 0 producer
// (4-stage ring), warp 1 TMEM owner (288 of 512 columns: three 128 x 96 FP32
// accumulators) and UMMA issuer, warps 2-5 sum db from the staged gy rows and,
// at the end, write the CTA's partial dW / db (reduced across CTAs by a second
// kernel).
#include <cuda_bf16.h>

#include "sur_kernels.h"
#include "sur_ptx.cuh"

namespace sur {
namespace {

constexpr int kWStages = 4;
constexpr int kWThreads = 192;
constexpr uint32_t kWTmemCols = 512;

struct WgradArgs {
  const __nv_bfloat16* x;
  const __nv_bfloat16* gy;
  float* partial;  // [gridDim.x][27 * 1024 + 32]
  SurGeom g;
  long long v_first;  // first row of the sweep
  int n_stages;       // stages of kst rows
  int kst;            // rows per stage: multiple of 16, <= 128, <= 2 P1
  int mn_swap;
  int* err;
};

__host__ __device__ inline int g_rows(const SurGeom& g) { return 4 * g.P1; }

__global__ void __launch_bounds__(kWThreads, 1) wgrad_umma_kernel(WgradArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const SurGeom g = a.g;
  const int kst = a.kst;
  const uint32_t gplane = static_cast<uint32_t>(g_rows(g)) * 16;  // one channel group of gy rows
  const uint32_t xplane = static_cast<uint32_t>(kst + 2) * 16;     // one channel group of one x slab
  const uint32_t stage_bytes = 4 * gplane + 12 * xplane;
  uint8_t* stages = smem;
  float* dbred = reinterpret_cast<float*>(smem + kWStages * stage_bytes);      // [4][32]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kWStages * stage_bytes + 512);
  uint64_t* full = bars;
  uint64_t* empty = bars + kWStages;
  uint64_t* acc_full = bars + 2 * kWStages;
  uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2 * kWStages + 1);
  int* abort_flag_w = reinterpret_cast<int*>(slot + 1);
  volatile int* decision = reinterpret_cast<volatile int*>(slot + 2);
  volatile int* abort_flag = abort_flag_w;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kWStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 2);  // the UMMA commit and the db readers
    }
    mbar_init(acc_full, 1);
    *abort_flag_w = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(slot, kWTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  int issued_loads = 0;
  bool mma_issued = false;

  if (warp == 0) {
    if (lane == 0) {
      int j = 0;
      for (int s = blockIdx.x; s < a.n_stages; s += gridDim.x, ++j) {
        const int st = j % kWStages;
        if (j >= kWStages && !mbar_wait(&empty[st], ((j / kWStages) - 1) & 1, abort_flag)) {
          atomicOr(a.err, kErrTimeout);
          *abort_flag_w = 1;
          break;
        }
        mbar_arrive_expect_tx(&full[st], stage_bytes);
        const long long v0 = a.v_first + static_cast<long long>(s) * kst;
        uint8_t* dst = stages + static_cast<size_t>(st) * stage_bytes;
#pragma unroll 1
        for (int c = 0; c < 4; ++c)
          bulk_g2s(dst + c * gplane, a.gy + (c * g.plane + v0) * 8, gplane, &full[st]);
#pragma unroll 1
        for (int dz = 0; dz < 3; ++dz) {
          const long long r = v0 + static_cast<long long>(dz - 1) * g.P2 + g.P1 - 1;
#pragma unroll 1
          for (int c = 0; c < 4; ++c)
            bulk_g2s(dst + 4 * gplane + (dz * 4 + c) * xplane, a.x + (c * g.plane + r) * 8, xplane, &full[st]);
        }
        issued_loads = j + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16_f32(kTile, 3 * kC, 1, 1);
      int j = 0;
      for (int s = blockIdx.x; s < a.n_stages; s += gridDim.x, ++j) {
        const int st = j % kWStages;
        if (!mbar_wait(&full[st], (j / kWStages) & 1, abort_flag)) {
          atomicOr(a.err, kErrTimeout);
          *abort_flag_w = 1;
          break;
        }
        tc_fence_after();
        const uint32_t base = smem_u32(stages + static_cast<size_t>(st) * stage_bytes);
        // K step ks moves both operands 256 bytes on, i.e. 16 in the
        // descriptors' start-address field (address / 16, 14 bits: shared
        // addresses stay below 2^18): the descriptors are built once per stage
        const uint64_t da0 = smem_desc_mn(base, g.P1 * 16, 128, a.mn_swap);
        uint64_t db0[3];
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) db0[dx] = smem_desc_mn(base + 4 * gplane + dx * 16, xplane, 128, a.mn_swap);
#pragma unroll 1
        for (int ks = 0; ks < kst / 16; ++ks) {
          const uint64_t dk = static_cast<uint64_t>(ks * 16);
          const uint32_t acc = (j > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) umma_bf16(tmem + dx * 3 * kC, da0 + dk, db0[dx] + dk, idesc, acc);
        }
        umma_commit(&empty[st]);
        mma_issued = true;
      }
      if (mma_issued) umma_commit(acc_full);
    }
  } else {
    // db from the staged gy rows, then the accumulators. Every decision to
    // leave the loop is taken by one thread between named barriers, so the
    // four warps always meet the same barriers.
    const int t = threadIdx.x - 64;  // 0..127
    const int cg = t / 32;           // channel group of o summed by this warp
    float db8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int j = 0;
    for (int s = blockIdx.x; s < a.n_stages; s += gridDim.x, ++j) {
      const int st = j % kWStages;
      if (!mbar_wait(&full[st], (j / kWStages) & 1, abort_flag)) {
        atomicOr(a.err, kErrTimeout);
        *abort_flag_w = 1;
      }
      named_bar(1, 128);
      if (t == 0) *decision = *abort_flag;
      named_bar(1, 128);
      if (*decision) break;
      const uint4* gp = reinterpret_cast<const uint4*>(stages + static_cast<size_t>(st) * stage_bytes + cg * gplane);
      for (int r = lane; r < kst; r += 32) {
        const uint4 u = gp[r];
        const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 f = __bfloat1622float2(h2[e]);
          db8[2 * e] += f.x;
          db8[2 * e + 1] += f.y;
        }
      }
      named_bar(1, 128);
      if (t == 0) mbar_arrive(&empty[st]);
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) db8[e] += __shfl_xor_sync(0xffffffffu, db8[e], off);
    }
    if (lane == 0)
#pragma unroll
      for (int e = 0; e < 8; ++e) dbred[cg * 8 + e] = db8[e];
    named_bar(1, 128);
    if (t == 0) *decision = (j > 0 && !*abort_flag) ? 1 : 0;
    named_bar(1, 128);
    float* out = a.partial + static_cast<long long>(blockIdx.x) * (27 * 1024 + 32);
    if (t < 32) out[27 * 1024 + t] = dbred[t];
    if (*decision) {
      bool ok = mbar_wait(acc_full, 0, abort_flag);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
      if (ok) {
        tc_fence_after();
        const int q = warp & 3;  // TMEM lane quarter of this warp
        const int jv = lane / 8, oo = q * 8 + lane % 8;
#pragma unroll 1
        for (int dx = 0; dx < 3; ++dx) {
#pragma unroll 1
          for (int dz = 0; dz < 3; ++dz) {
            uint32_t v[32];
            tmem_ld32(tmem + (static_cast<uint32_t>(q * 32) << 16) + (dx * 3 + dz) * kC, v);
            tmem_wait_ld();
            if (jv < 3) {
              const int dy = 2 - jv;
              const int tap = dz * 9 + dy * 3 + dx;
              float4* dst = reinterpret_cast<float4*>(out + tap * 1024 + oo * 32);
#pragma unroll
              for (int i = 0; i < 8; ++i)
                dst[i] = make_float4(__uint_as_float(v[4 * i]), __uint_as_float(v[4 * i + 1]),
                                     __uint_as_float(v[4 * i + 2]), __uint_as_float(v[4 * i + 3]));
            }
          }
        }
        tc_fence_before();
      } else {
        atomicOr(a.err, kErrTimeout);
        *abort_flag_w = 1;
      }
    }
  }

  // drain in-flight copies and UMMAs before the CTA's memory is released
  if (warp == 0 && lane == 0 && issued_loads > 0 && *abort_flag) {
    for (int j = (issued_loads > kWStages ? issued_loads - kWStages : 0); j < issued_loads; ++j)
      mbar_wait(&full[j % kWStages], (j / kWStages) & 1, nullptr);
  }
  if (warp == 1 && lane == 0 && mma_issued && *abort_flag) mbar_wait(acc_full, 0, nullptr);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kWTmemCols);
  }
}

__global__ void reduce_wgrad_kernel(const float* __restrict__ partial, int n_part, int len, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  float s = 0.f;
  for (int c = 0; c < n_part; ++c) s += partial[static_cast<long long>(c) * len + i];
  out[i] = s;
}

}  // namespace

int wgrad_stage_rows(const SurGeom& g) {
  int k = 16 * ((2 * g.P1) / 16);
  return k > 128 ? 128 : k;
}

size_t wgrad_smem_bytes(const SurGeom& g) {
  const int kst = wgrad_stage_rows(g);
  const size_t stage = 16 * (4 * static_cast<size_t>(g_rows(g)) + 12 * static_cast<size_t>(kst + 2));
  return kWStages * stage + 512 + 8 * (2 * kWStages + 1) + 16;  // stages, db scratch, barriers, slot + flags
}

cudaError_t launch_wgrad_umma(const SurGeom& g, int batch, const __nv_bfloat16* x, const __nv_bfloat16* gy,
                              float* partial, int max_ctas, float* grad_wb, int mn_swap, int* err,
                              cudaStream_t st) {
  const int kst = wgrad_stage_rows(g);
  if (kst < 16) return cudaErrorInvalidValue;
  const long long v_first = g.G + g.P2 - 2ll * g.P1;
  const long long v_end = g.G + static_cast<long long>(batch - 1) * g.V + static_cast<long long>(g.n + 1) * g.P2;
  const int n_stages = static_cast<int>((v_end - v_first + kst - 1) / kst);
  const int grid = n_stages < max_ctas ? n_stages : max_ctas;
  const size_t smem = wgrad_smem_bytes(g);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(wgrad_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(wgrad_smem_bytes(make_geom(64, 1))));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  WgradArgs a{x, gy, partial, g, v_first, n_stages, kst, mn_swap, err};
  wgrad_umma_kernel<<<grid, kWThreads, smem, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int len = 27 * 1024 + 32;  // weights then bias of one layer (adjacent in the flat vector)
  reduce_wgrad_kernel<<<(len + 255) / 256, 256, 0, st>>>(partial, grid, len, grad_wb);
  return cudaGetLastError();
}

}  // namespace sur
