// Support kernels: counting sort of particles into grid cells, permutations
// between the library's particle order and the caller's, tool kinematics and
// its adjoint, losses and loss seeds.
#include <climits>
#include <mutex>
#include <set>

#include "common.cuh"
#include "kernels.h"
#include "perm.h"
#include "share.h"

namespace mpm {

constexpr int fX = 0, fF = 15;
static inline int blocks_for(long long n, int t) { return int((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// counting sort by (scene, Morton order of the cell of the stencil origin).
// The Morton order keeps every 4^3 grid block contiguous (its cells are the
// code's lowest 6 bits) and orders the particles of a block by cell, so that
// a CTA's consecutive particles occupy few, densely filled cells: the scatter
// tile then has fewer (cell, node) accumulations and fewer nodes to flush.
// ---------------------------------------------------------------------------
// with_class: water particles before every other material (their keys offset
// by S x MB), so that the non-water particles occupy the index range [Nl, N).
__global__ void sort_key_kernel(Params P, const float* __restrict__ st, const uint32_t* __restrict__ tag,
                                uint32_t* __restrict__ key, uint32_t* __restrict__ rank,
                                uint32_t* __restrict__ bins, int with_class) {
  const int N = P.N;
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int b[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float bf = base_floor(grid_coord(st[(fX + d) * N + p], P));
    bf = fminf(fmaxf(bf, 0.0f), float(P.n - 3));  // NaN -> 0
    b[d] = int(bf);
  }
  uint32_t tg = tag[p];
  uint32_t k = uint32_t(tag_scene(tg)) * uint32_t(P.MB) +
               morton3(uint32_t(b[0]), uint32_t(b[1]), uint32_t(b[2]));
  if (with_class && P.mat[tag_mat(tg)].kind != kLiquid) k += uint32_t(P.S) * uint32_t(P.MB);
  key[p] = k;
  rank[p] = atomicAdd(&bins[k], 1u);
}

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ inline uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums, uint32_t& total) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = warp_sums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_sums[lane] = s;
  }
  __syncthreads();
  uint32_t pre = (wid > 0 ? warp_sums[wid - 1] : 0u) + x - v;
  total = warp_sums[31];
  __syncthreads();
  return pre;
}

// exclusive scan of each tile in place; tile totals to sums
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(uint32_t* __restrict__ a, long long n,
                                                                  uint32_t* __restrict__ sums) {
  __shared__ uint32_t ws[32];
  long long base = (long long)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  uint32_t v[kScanPer], s = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    v[i] = (base + i < n) ? a[base + i] : 0u;
    s += v[i];
  }
  uint32_t total;
  uint32_t pre = block_exclusive_scan(s, ws, total);
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    if (base + i < n) a[base + i] = pre;
    pre += v[i];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// single CTA: exclusive scan of the tile totals (any count, looped)
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(uint32_t* __restrict__ sums, int n) {
  __shared__ uint32_t ws[32];
  uint32_t carry = 0;
  for (int off = 0; off < n; off += kScanThreads) {
    int i = off + threadIdx.x;
    uint32_t v = i < n ? sums[i] : 0u;
    uint32_t total;
    uint32_t pre = block_exclusive_scan(v, ws, total);
    if (i < n) sums[i] = pre + carry;
    carry += total;
  }
}

__global__ void scan_add_kernel(uint32_t* __restrict__ a, long long n, const uint32_t* __restrict__ sums) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += sums[i / kScanTile];
}

__global__ void sort_scatter_kernel(int N, const float* __restrict__ st_in,
                                    const uint32_t* __restrict__ tag_in, const int* __restrict__ pid_in,
                                    float* __restrict__ st_out, uint32_t* __restrict__ tag_out,
                                    int* __restrict__ pid_out, const uint32_t* __restrict__ key,
                                    const uint32_t* __restrict__ rank, const uint32_t* __restrict__ offs,
                                    Params P) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  uint32_t d = offs[key[p]] + rank[p];
  uint32_t tg = tag_in[p];
  bool liquid = is_liquid(P.mat[tag_mat(tg)].kind);
  const int nf = liquid ? fF + 1 : kStateFields;  // a liquid carries only J = F[0]
  for (int f = 0; f < nf; ++f) st_out[(long long)f * N + d] = st_in[(long long)f * N + p];
  tag_out[d] = tg;
  pid_out[d] = pid_in[p];
}

static void bin_particles(const Params& P, const float* st, const uint32_t* tag, SortBuffers sb, int with_class,
                          cudaStream_t s) {
  const int N = P.N;
  const long long nb = with_class ? 2LL * sb.n_bins : sb.n_bins;
  cudaMemsetAsync(sb.bins, 0, sizeof(uint32_t) * (size_t)nb, s);
  if (N > 0) sort_key_kernel<<<blocks_for(N, 256), 256, 0, s>>>(P, st, tag, sb.key, sb.rank, sb.bins, with_class);
  int tiles = blocks_for(nb, kScanTile);
  scan_tiles_kernel<<<tiles, kScanThreads, 0, s>>>(sb.bins, nb, sb.tile_sums);
  scan_sums_kernel<<<1, kScanThreads, 0, s>>>(sb.tile_sums, tiles);
  scan_add_kernel<<<blocks_for(nb, 256), 256, 0, s>>>(sb.bins, nb, sb.tile_sums);
}

void launch_bin(const Params& P, const float* st, const uint32_t* tag, SortBuffers sb, cudaStream_t s) {
  bin_particles(P, st, tag, sb, 0, s);
}

// count of water particles (the material of each tag) into *out
__global__ void count_water_kernel(Params P, const uint32_t* __restrict__ tag, int* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const bool w = p < P.N && P.mat[tag_mat(tag[p])].kind == kLiquid;
  const unsigned b = __ballot_sync(0xffffffffu, w);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(out, __popc(b));
}

void launch_count_water(const Params& P, const uint32_t* tag, int* out, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(int), s);
  if (P.N > 0) count_water_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, tag, out);
}

void launch_sort(const Params& P, const float* st_in, const uint32_t* tag_in, const int* pid_in,
                 float* st_out, uint32_t* tag_out, int* pid_out, SortBuffers sb, cudaStream_t s) {
  const int N = P.N;
  bin_particles(P, st_in, tag_in, sb, 1, s);
  if (N > 0)
    sort_scatter_kernel<<<blocks_for(N, 256), 256, 0, s>>>(N, st_in, tag_in, pid_in, st_out, tag_out,
                                                          pid_out, sb.key, sb.rank, sb.bins, P);
}

// ---------------------------------------------------------------------------
// caller order <-> library order
// ---------------------------------------------------------------------------
// to_caller = 1: dst[pid[p] * fields + c] = src[c * stride_src + p]
// to_caller = 0: dst[c * stride_dst + p] = src[pid[p] * fields + c]
__global__ void gather_rows_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                   const int* __restrict__ pid, int N, int fields, int ss, int sd,
                                   int to_caller) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  long long q = pid ? pid[p] : p;
  if (to_caller) {
    for (int c = 0; c < fields; ++c) dst[q * fields + c] = src[(long long)c * ss + p];
  } else {
    for (int c = 0; c < fields; ++c) dst[(long long)c * sd + p] = src[q * fields + c];
  }
}

__global__ void inverse_perm_kernel(const int* __restrict__ pid, int* __restrict__ inv, int N) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) inv[pid[p]] = p;
}

// dst[f][p'] = src[f][inv_from[pid_to[p']]]: writes coalesced, reads gathered
// (the two orders differ by one re-sort, so the reads stay mostly local)
__global__ void permute_state_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                     const int* __restrict__ inv_from, const int* __restrict__ pid_to, int N,
                                     int fields) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const long long p = inv_from[pid_to[q]];
  for (int f = 0; f < fields; ++f) dst[(long long)f * N + q] = src[(long long)f * N + p];
}

void launch_permute_state(const float* src, float* dst, const int* pid_from, const int* pid_to, int* inv, int N,
                          int fields, cudaStream_t s) {
  if (N == 0) return;
  inverse_perm_kernel<<<blocks_for(N, 256), 256, 0, s>>>(pid_from, inv, N);
  permute_state_kernel<<<blocks_for(N, 256), 256, 0, s>>>(src, dst, inv, pid_to, N, fields);
}

void launch_gather_rows(const float* src, float* dst, const int* pid, int N, int fields,
                        int field_stride_src, int field_stride_dst, int to_caller, cudaStream_t s) {
  if (N == 0) return;
  gather_rows_kernel<<<blocks_for(N, 256), 256, 0, s>>>(src, dst, pid, N, fields, field_stride_src,
                                                       field_stride_dst, to_caller);
}

__global__ void init_state_kernel(float* __restrict__ st, int N) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  for (int k = 0; k < 9; ++k) {
    st[(long long)(6 + k) * N + p] = 0.0f;                       // C = 0
    st[(long long)(15 + k) * N + p] = (k % 4 == 0) ? 1.0f : 0.0f;  // F = I
  }
}

void launch_init_state(float* st, int N, cudaStream_t s) {
  if (N == 0) return;
  init_state_kernel<<<blocks_for(N, 256), 256, 0, s>>>(st, N);
}

// C = 0, F = I and the material of particles [lo, lo + cnt) of the initial state
__global__ void init_particles_kernel(float* __restrict__ X0, uint32_t* __restrict__ tag0,
                                      const uint8_t* __restrict__ mat, int lo, int cnt, int N,
                                      int n_mat, int* __restrict__ err) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= cnt) return;
  long long i = (long long)lo + p;
  for (int k = 0; k < 9; ++k) {
    X0[(long long)(6 + k) * N + i] = 0.0f;
    X0[(long long)(15 + k) * N + i] = (k % 4 == 0) ? 1.0f : 0.0f;
  }
  uint32_t m = mat[p];
  if (m >= (uint32_t)n_mat) {
    atomicOr(err, kErrArg);
    m = 0;
  }
  tag0[i] = (tag0[i] & 0xffffff00u) | m;
}

void launch_init_particles(float* X0, uint32_t* tag0, const uint8_t* mat, int lo, int cnt, int N,
                           int n_mat, int* err, cudaStream_t s) {
  if (cnt == 0) return;
  init_particles_kernel<<<blocks_for(cnt, 256), 256, 0, s>>>(X0, tag0, mat, lo, cnt, N, n_mat, err);
}

__global__ void iota_kernel(int* __restrict__ a, int N) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < N) a[p] = p;
}

int sm_count() {
  constexpr int kMaxDev = 64;
  static int cached[kMaxDev] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return 1;
  }
  if (cached[dev] <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 1;
    }
    cached[dev] = n;  // a plain int store: concurrent first calls write the same value
  }
  return cached[dev];
}

void max_shared_carveout(const void* kernel) {
  static std::mutex lock;
  static std::set<const void*> done;
  std::lock_guard<std::mutex> g(lock);
  if (done.count(kernel)) return;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    cudaGetLastError();
  done.insert(kernel);
}

void launch_iota(int* a, int N, cudaStream_t s) {
  if (N == 0) return;
  iota_kernel<<<blocks_for(N, 256), 256, 0, s>>>(a, N);
}

// adj_field[c * N + p] += seed[pid[p] * ncomp + c], c < ncomp, for particles of
// the caller range [lo, lo + count).
__global__ void add_seed_kernel(float* __restrict__ adj, const float* __restrict__ seed,
                                const int* __restrict__ pid, int lo, int count, int N, int ncomp) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int q = pid[p] - lo;
  if (q < 0 || q >= count) return;
  for (int c = 0; c < ncomp; ++c) adj[(long long)c * N + p] += seed[(long long)q * ncomp + c];
}

__global__ void add_fields_kernel(float* __restrict__ dst, float* __restrict__ src, long long n, int clear_src) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    dst[i] += src[i];
    if (clear_src) src[i] = 0.0f;
  }
}

void launch_add_fields(float* dst, float* src, long long n, int clear_src, cudaStream_t s) {
  if (n <= 0) return;
  long long blocks = (n + 255) / 256;
  const int cap = sm_count() * 8;
  add_fields_kernel<<<int(blocks < cap ? blocks : cap), 256, 0, s>>>(dst, src, n, clear_src);
}

void launch_add_seed(float* adj_field, const float* seed, const int* pid, const uint32_t*, int,
                     int lo, int count, int N, cudaStream_t s, int ncomp) {
  if (N == 0) return;
  add_seed_kernel<<<blocks_for(N, 256), 256, 0, s>>>(adj_field, seed, pid, lo, count, N, ncomp);
}

// ---------------------------------------------------------------------------
// tool kinematics (Sec. 4.2: the action is the tool's linear and angular
// velocity; App. B.1: held for a fixed number of substeps). One thread per
// scene integrates the pose in FP64:
//   p_{n+1} = p_n + dt pdot_n,  q_{n+1} = normalize(dq(omega_n dt) q_n),
//   dq(w) = (cos(|w|/2), sin(|w|/2) w/|w|).
// Pose record per step: p (3), q (4), pdot (3), omega (3).
// ---------------------------------------------------------------------------
__device__ inline void qmul(const double* a, const double* b, double* o) {
  o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// dq(omega dt) and, if J != null, d dq / d omega (4x3, row-major)
__device__ inline void dq_of(const double* om, double dt, double* dq, double* J) {
  double w2 = om[0] * om[0] + om[1] * om[1] + om[2] * om[2];
  double w = sqrt(w2);
  double th = 0.5 * dt * w;  // half angle
  double h = 0.5 * dt;
  // sinc(th) = sin(th)/th and (th cos th - sin th)/th^3, via series near 0
  double sinc, g;
  if (th < 1e-4) {
    double t2 = th * th;
    sinc = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
    g = -1.0 / 3.0 + t2 / 30.0;
  } else {
    sinc = sin(th) / th;
    g = (th * cos(th) - sin(th)) / (th * th * th);
  }
  dq[0] = cos(th);
  for (int i = 0; i < 3; ++i) dq[1 + i] = h * sinc * om[i];
  if (J) {
    // d cos(th)/d om = -sin(th) h om / w = -h^2 sinc om
    for (int k = 0; k < 3; ++k) J[k] = -h * h * sinc * om[k];
    // d (h sinc om_i)/d om_k = h (sinc delta_ik + om_i dsinc/dth h om_k / w)
    //                        = h sinc delta_ik + h^3 g om_i om_k
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) J[3 * (1 + i) + k] = h * sinc * (i == k ? 1.0 : 0.0) + h * h * h * g * om[i] * om[k];
  }
}

__device__ inline void qnormalize(double* q) {
  const double r = 1.0 / sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int i = 0; i < 4; ++i) q[i] *= r;
}

// One warp per scene. Lane a handles action a (in chunks of 32 actions): its
// rotation increment, the action's whole rotation D_a and translation; a
// prefix product / sum across the lanes gives the pose at the action's first
// step, from which the lane integrates the action's steps one by one (the
// same per-step update as a serial walk, in FP64).
__global__ void tool_forward_kernel(int S, const float* __restrict__ pose0,
                                    const float* __restrict__ actions, int n_actions, int spa,
                                    int n_steps, int max_steps, double dt, float* __restrict__ poses) {
  const int sc = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (sc >= S) return;  // whole warps
  double p[3], q[4];
  for (int i = 0; i < 3; ++i) p[i] = pose0[sc * 7 + i];
  for (int i = 0; i < 4; ++i) q[i] = pose0[sc * 7 + 3 + i];
  qnormalize(q);
  for (int a0 = 0; a0 < n_actions; a0 += 32) {
    const int a = a0 + lane;
    const int lo = a * spa;
    const int hi = (a == n_actions - 1) ? n_steps : min((a + 1) * spa, n_steps);
    const int len = (a < n_actions && lo < n_steps) ? hi - lo : 0;
    double pd[3] = {0.0, 0.0, 0.0}, om[3] = {0.0, 0.0, 0.0}, dq[4] = {1.0, 0.0, 0.0, 0.0};
    if (len > 0) {
      const float* act = actions + ((long long)sc * n_actions + a) * 6;
      for (int i = 0; i < 3; ++i) {
        pd[i] = act[i];
        om[i] = act[3 + i];
      }
      dq_of(om, dt, dq, nullptr);
    }
    // the action's rotation and translation over its steps
    double D[4] = {1.0, 0.0, 0.0, 0.0}, tr[3] = {0.0, 0.0, 0.0};
    for (int m = 0; m < len; ++m) {
      double t4[4];
      qmul(dq, D, t4);
      qnormalize(t4);
      for (int i = 0; i < 4; ++i) D[i] = t4[i];
      for (int i = 0; i < 3; ++i) tr[i] += dt * pd[i];
    }
    // inclusive scans across lanes: rotations compose with later ones on the left
    for (int off = 1; off < 32; off <<= 1) {
      double oD[4], ot[3];
      for (int i = 0; i < 4; ++i) oD[i] = __shfl_up_sync(0xffffffffu, D[i], off);
      for (int i = 0; i < 3; ++i) ot[i] = __shfl_up_sync(0xffffffffu, tr[i], off);
      if (lane >= off) {
        double t4[4];
        qmul(D, oD, t4);
        qnormalize(t4);
        for (int i = 0; i < 4; ++i) D[i] = t4[i];
        for (int i = 0; i < 3; ++i) tr[i] += ot[i];
      }
    }
    double E[4], et[3];
    for (int i = 0; i < 4; ++i) E[i] = __shfl_up_sync(0xffffffffu, D[i], 1);
    for (int i = 0; i < 3; ++i) et[i] = __shfl_up_sync(0xffffffffu, tr[i], 1);
    if (lane == 0) {
      E[0] = 1.0;
      E[1] = E[2] = E[3] = 0.0;
      et[0] = et[1] = et[2] = 0.0;
    }
    double qc[4], pc[3];
    qmul(E, q, qc);
    qnormalize(qc);
    for (int i = 0; i < 3; ++i) pc[i] = p[i] + et[i];
    for (int m = 0; m < len; ++m) {
      float* rec = poses + ((long long)sc * max_steps + lo + m) * kToolFields;
      for (int i = 0; i < 3; ++i) rec[i] = float(pc[i]);
      for (int i = 0; i < 4; ++i) rec[3 + i] = float(qc[i]);
      for (int i = 0; i < 3; ++i) {
        rec[7 + i] = float(pd[i]);
        rec[10 + i] = float(om[i]);
      }
      for (int i = 0; i < 3; ++i) pc[i] += dt * pd[i];
      double t4[4];
      qmul(dq, qc, t4);
      qnormalize(t4);
      for (int i = 0; i < 4; ++i) qc[i] = t4[i];
    }
    // carry the pose after this chunk of actions
    double DL[4], tL[3];
    for (int i = 0; i < 4; ++i) DL[i] = __shfl_sync(0xffffffffu, D[i], 31);
    for (int i = 0; i < 3; ++i) tL[i] = __shfl_sync(0xffffffffu, tr[i], 31);
    double t4[4];
    qmul(DL, q, t4);
    qnormalize(t4);
    for (int i = 0; i < 4; ++i) q[i] = t4[i];
    for (int i = 0; i < 3; ++i) p[i] += tL[i];
  }
}

void launch_tool_forward(const Params& P, const float* pose0, const float* actions, int n_actions,
                         int spa, int n_steps, int max_steps, float* poses, cudaStream_t s) {
  tool_forward_kernel<<<blocks_for((long long)P.S * 32, 128), 128, 0, s>>>(P.S, pose0, actions, n_actions, spa,
                                                                         n_steps, max_steps, (double)P.dt, poses);
}

__device__ inline void qmulf(const float* a, const float* b, float* o) {
  o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// d R(q) / d q contracted with gR: returns dL/dq (4)
__device__ inline void rot_q_adjoint(const float* q, const float* gR, float* gq) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  const float* G = gR;
  // R = [[1-2(yy+zz), 2(xy-wz), 2(xz+wy)], [2(xy+wz), 1-2(xx+zz), 2(yz-wx)], [2(xz-wy), 2(yz+wx), 1-2(xx+yy)]]
  gq[0] = 2.0f * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
  gq[1] = 2.0f * (y * G[1] + z * G[2] + y * G[3] - 2.0f * x * G[4] - w * G[5] + z * G[6] + w * G[7] - 2.0f * x * G[8]);
  gq[2] = 2.0f * (-2.0f * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] + z * G[7] - 2.0f * y * G[8]);
  gq[3] = 2.0f * (-2.0f * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2.0f * z * G[4] + y * G[5] + x * G[6] + y * G[7]);
}

// Reverse sweep of the kinematics: per-step tool gradients (p, R, pdot, omega)
// -> action gradients (accumulated into action_grad, [S][n_actions][6]). One
// warp per scene: the lanes evaluate every action's rotation increment and its
// Jacobian (FP64) and stage the pose and gradient rows of 128 steps at a time
// in shared memory; lane 0 walks the steps backwards in FP32 (the adjoint
// recurrence of the orientation is serial).
constexpr int kToolChunk = 128;

size_t tool_backward_smem(int n_actions) {
  return (static_cast<size_t>(n_actions) * (16 + 6) + static_cast<size_t>(kToolChunk) * (kToolFields + kToolGradFields)) *
         sizeof(float);
}

__global__ void tool_backward_kernel(int S, const float* __restrict__ pose0,
                                     const float* __restrict__ actions, int n_actions, int spa,
                                     int n_steps, int max_steps, float dt,
                                     const float* __restrict__ poses,
                                     const float* __restrict__ tool_grad,
                                     float* __restrict__ action_grad) {
  extern __shared__ float tsm[];
  float* sdq = tsm;                                  // [n_actions][16]: dq (4), d dq / d omega (12)
  float* sag = sdq + (size_t)n_actions * 16;         // [n_actions][6] action gradients
  float* srec = sag + (size_t)n_actions * 6;         // [kToolChunk][13]
  float* stg = srec + (size_t)kToolChunk * kToolFields;  // [kToolChunk][18]
  const int sc = blockIdx.x, lane = threadIdx.x;
  if (sc >= S) return;
  for (int a = lane; a < n_actions; a += 32) {
    const float* act = actions + ((long long)sc * n_actions + a) * 6;
    double om[3] = {act[3], act[4], act[5]}, dqd[4], Jd[12];
    dq_of(om, (double)dt, dqd, Jd);
    for (int i = 0; i < 4; ++i) sdq[a * 16 + i] = float(dqd[i]);
    for (int i = 0; i < 12; ++i) sdq[a * 16 + 4 + i] = float(Jd[i]);
    for (int i = 0; i < 6; ++i) sag[a * 6 + i] = 0.0f;
  }
  float Pb[3] = {0, 0, 0}, Qb[4] = {0, 0, 0, 0};
  for (int n1 = n_steps; n1 > 0; n1 -= kToolChunk) {
    const int n0 = max(0, n1 - kToolChunk);
    __syncwarp();
    for (int i = lane; i < (n1 - n0) * kToolFields; i += 32)
      srec[i] = poses[((long long)sc * max_steps + n0) * kToolFields + i];
    for (int i = lane; i < (n1 - n0) * kToolGradFields; i += 32)
      stg[i] = tool_grad[((long long)sc * max_steps + n0) * kToolGradFields + i];
    __syncwarp();
    if (lane == 0) {
      for (int n = n1 - 1; n >= n0; --n) {
        const float* rec = srec + (n - n0) * kToolFields;
        const float* tg = stg + (n - n0) * kToolGradFields;
        const int a = min(n / spa, n_actions - 1);
        const float* dq = sdq + a * 16;
        const float* Jdq = dq + 4;
        // the stored pose (a unit quaternion to FP32 precision) is re-normalised
        float q[4];
        const float qr = rsqrtf(rec[3] * rec[3] + rec[4] * rec[4] + rec[5] * rec[5] + rec[6] * rec[6]);
        for (int i = 0; i < 4; ++i) q[i] = rec[3 + i] * qr;
        // p_{n+1} = p_n + dt pdot_n
        float pdb[3], pb[3];
        for (int i = 0; i < 3; ++i) {
          pdb[i] = tg[12 + i] + dt * Pb[i];
          pb[i] = tg[i] + Pb[i];
        }
        // q_{n+1} = qq / |qq|, qq = dq q
        float qq[4];
        qmulf(dq, q, qq);
        const float inq = rsqrtf(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
        const float qh[4] = {qq[0] * inq, qq[1] * inq, qq[2] * inq, qq[3] * inq};
        const float dotq = qh[0] * Qb[0] + qh[1] * Qb[1] + qh[2] * Qb[2] + qh[3] * Qb[3];
        float qqb[4];
        for (int i = 0; i < 4; ++i) qqb[i] = (Qb[i] - qh[i] * dotq) * inq;
        // qq = L(dq) q: qb = L(dq)^T qqb; dqb = Rm(q)^T qqb with qq = Rm(q) dq
        float qb[4], dqb[4];
        qb[0] = dq[0] * qqb[0] + dq[1] * qqb[1] + dq[2] * qqb[2] + dq[3] * qqb[3];
        qb[1] = -dq[1] * qqb[0] + dq[0] * qqb[1] + dq[3] * qqb[2] - dq[2] * qqb[3];
        qb[2] = -dq[2] * qqb[0] - dq[3] * qqb[1] + dq[0] * qqb[2] + dq[1] * qqb[3];
        qb[3] = -dq[3] * qqb[0] + dq[2] * qqb[1] - dq[1] * qqb[2] + dq[0] * qqb[3];
        dqb[0] = q[0] * qqb[0] + q[1] * qqb[1] + q[2] * qqb[2] + q[3] * qqb[3];
        dqb[1] = -q[1] * qqb[0] + q[0] * qqb[1] - q[3] * qqb[2] + q[2] * qqb[3];
        dqb[2] = -q[2] * qqb[0] + q[3] * qqb[1] + q[0] * qqb[2] - q[1] * qqb[3];
        dqb[3] = -q[3] * qqb[0] - q[2] * qqb[1] + q[1] * qqb[2] + q[0] * qqb[3];
        float gq[4];
        rot_q_adjoint(q, tg + 3, gq);
        for (int i = 0; i < 4; ++i) qb[i] += gq[i];
        float* ag = sag + a * 6;
        for (int k = 0; k < 3; ++k) {
          float omb = tg[15 + k];
          for (int i = 0; i < 4; ++i) omb += Jdq[3 * i + k] * dqb[i];
          ag[k] += pdb[k];
          ag[3 + k] += omb;
        }
        for (int i = 0; i < 3; ++i) Pb[i] = pb[i];
        for (int i = 0; i < 4; ++i) Qb[i] = qb[i];
      }
    }
  }
  __syncwarp();
  for (int i = lane; i < n_actions * 6; i += 32) action_grad[(long long)sc * n_actions * 6 + i] += sag[i];
}

void launch_tool_backward(const Params& P, const float* pose0, const float* actions, int n_actions,
                          int spa, int n_steps, int max_steps, const float* poses,
                          const float* tool_grad, float* action_grad, cudaStream_t s) {
  const size_t smem = tool_backward_smem(n_actions);
  if (smem > 48 * 1024) cudaFuncSetAttribute(tool_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
  tool_backward_kernel<<<P.S, 32, smem, s>>>(P.S, pose0, actions, n_actions, spa, n_steps, max_steps, P.dt, poses,
                                            tool_grad, action_grad);
}

// ---------------------------------------------------------------------------
// losses (App. C)
// ---------------------------------------------------------------------------
__device__ inline void block_add_double(double v, double* out) {
  __shared__ double ws[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && s != 0.0) atomicAdd(out, s);
  }
}

// L_s = w sum |x - t|^2 over particles of scene `scene` (-1: all, per-scene
// totals into loss[scene]); adj_x += 2 w (x - t).
__global__ void position_loss_kernel(Params P, const float* __restrict__ st, const uint32_t* __restrict__ tag,
                                     int scene, float tx, float ty, float tz, float w,
                                     float* __restrict__ adj, double* __restrict__ loss) {
  const int N = P.N;
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  int sc = -1;
  if (p < N) {
    sc = tag_scene(tag[p]);
    if (scene < 0 || sc == scene) {
      float d0 = st[p] - tx, d1 = st[N + p] - ty, d2 = st[2 * N + p] - tz;
      l = (double)w * ((double)d0 * d0 + (double)d1 * d1 + (double)d2 * d2);
      adj[p] += 2.0f * w * d0;
      adj[N + p] += 2.0f * w * d1;
      adj[2 * N + p] += 2.0f * w * d2;
    }
  }
  // one atomic per warp when its particles share the loss entry (particles are
  // sorted by scene, so only warps at a scene boundary add lane by lane)
  const int t = (p < N && (scene < 0 || sc == scene)) ? (scene < 0 ? sc : 0) : -1;
  const int tmax = __reduce_max_sync(0xffffffffu, t);
  const int tmin = __reduce_min_sync(0xffffffffu, t >= 0 ? t : INT_MAX);
  if (tmax < 0) return;
  if (tmin == tmax) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss + tmax, l);
  } else if (l != 0.0) {
    atomicAdd(loss + t, l);
  }
}

void launch_position_loss(const Params& P, const float* st, const uint32_t* tag, int scene,
                          float tx, float ty, float tz, float w, float* adj, double* loss,
                          cudaStream_t s) {
  if (P.N == 0) return;
  position_loss_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, st, tag, scene, tx, ty, tz, w, adj, loss);
}

// P2G mass of the particles of one scene into a dense float grid
__global__ void mass_scatter_kernel(Params P, const float* __restrict__ st, const uint32_t* __restrict__ tag,
                                    int scene, float* __restrict__ mg) {
  const int N = P.N;
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  uint32_t tg = tag[p];
  if (tag_scene(tg) != scene) return;
  float x[3] = {st[p], st[N + p], st[2 * N + p]};
  Stencil sc;
  make_stencil(x, P, sc);
  float m = P.mat[tag_mat(tg)].mass;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) {
        long long idx = ((long long)(sc.base[0] + a) * P.n + sc.base[1] + b) * P.n + sc.base[2] + c;
        atomicAdd(mg + idx, m * sc.w[0][a] * sc.w[1][b] * sc.w[2][c]);
      }
}

void launch_mass_scatter(const Params& P, const float* st, const uint32_t* tag, int scene,
                         float* mgrid, cudaStream_t s) {
  if (P.N == 0) return;
  mass_scatter_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, st, tag, scene, mgrid);
}

// L = sum (m - m*)^2 / M^2 + sum m d* / M; dL/dm per node
__global__ void mass_loss_nodes_kernel(long long n3, const float* __restrict__ mg, const float* __restrict__ tm,
                                       const float* __restrict__ td, float inv_M, float* __restrict__ dLdm,
                                       double* __restrict__ loss) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < n3) {
    double m = mg[i], d = m - (double)tm[i];
    l = d * d * (double)inv_M * inv_M + m * (double)td[i] * inv_M;
    dLdm[i] = float(2.0 * d * inv_M * inv_M + (double)td[i] * inv_M);
  }
  block_add_double(l, loss);
}

void launch_mass_loss_nodes(long long n3, const float* mgrid, const float* tm, const float* td,
                            float inv_M, float* dLdm, double* loss, cudaStream_t s) {
  mass_loss_nodes_kernel<<<blocks_for(n3, 256), 256, 0, s>>>(n3, mgrid, tm, td, inv_M, dLdm, loss);
}

// adj_x += sum_o dL/dm_i m_p grad W_o
__global__ void mass_loss_grad_kernel(Params P, const float* __restrict__ st, const uint32_t* __restrict__ tag,
                                      int scene, const float* __restrict__ g, float* __restrict__ adj) {
  const int N = P.N;
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  uint32_t tg = tag[p];
  if (tag_scene(tg) != scene) return;
  float x[3] = {st[p], st[N + p], st[2 * N + p]};
  Stencil sc;
  make_stencil(x, P, sc);
  float m = P.mat[tag_mat(tg)].mass;
  float gx = 0.f, gy = 0.f, gz = 0.f;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) {
        long long idx = ((long long)(sc.base[0] + a) * P.n + sc.base[1] + b) * P.n + sc.base[2] + c;
        float gm = g[idx] * m * P.inv_dx;
        gx += gm * sc.dw[0][a] * sc.w[1][b] * sc.w[2][c];
        gy += gm * sc.w[0][a] * sc.dw[1][b] * sc.w[2][c];
        gz += gm * sc.w[0][a] * sc.w[1][b] * sc.dw[2][c];
      }
  adj[p] += gx;
  adj[N + p] += gy;
  adj[2 * N + p] += gz;
}

void launch_mass_loss_grad(const Params& P, const float* st, const uint32_t* tag, int scene,
                           const float* dLdm, float* adj, cudaStream_t s) {
  if (P.N == 0) return;
  mass_loss_grad_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, st, tag, scene, dLdm, adj);
}

}  // namespace mpm
