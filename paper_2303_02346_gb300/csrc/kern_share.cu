// Neighbour sums over the particles of a scene (paper Sec. 5.1, "Gradient
// Sharing within Fluid Bodies"): the gradient of particle a is replaced by a
// weighted sum of the gradients of its neighbours, and, as the paper's
// practical approximation, an attraction loss pulls particles towards
// neighbours that had a lower loss:
//   c_j = exp(-ell_j / tau),  k(r) = (1 - r^2)^3 for r < 1, else 0,
//   shared g'_a = sum_j c_j k(d_aj / h) g_j            (j = a included),
//   L_att       = sum_a sum_{j != a} c_j phi(d_aj),    phi(d) = d k(d / h),
//   dL_att/dx_a = sum_{j != a} (c_j + c_a) phi'(d_aj) (x_a - x_j) / d_aj,
//   phi'(d)     = k(r) - 6 r^2 (1 - r^2)^2,  r = d / h.
// (The paper gives the form of the sums; the kernel w = c_j k(d / h) is this
// library's reading.) Neighbours within h <= dx of particle a have stencil
// origins at most one cell away from a's, so the 27 cells around a's cell in
// the Morton bins of the particle sort hold all of them. One thread per
// particle in bin order: the threads of a warp visit nearly the same cells,
// so the candidate loads hit L1.
#include "common.cuh"
#include "kernels.h"
#include "share.h"

namespace mpm {

static inline int blocks_for(long long n, int t) { return int((n + t - 1) / t); }

__global__ void nbr_pack_kernel(int N, const float* __restrict__ st, const int* __restrict__ pid,
                                const uint32_t* __restrict__ key, const uint32_t* __restrict__ rank,
                                const uint32_t* __restrict__ bins, const float* __restrict__ ell,
                                const float* __restrict__ g, int lo, int cnt, float inv_tau,
                                float4* __restrict__ pk, float4* __restrict__ pg, int* __restrict__ sidx) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  const uint32_t slot = bins[key[p]] + rank[p];
  const int q = pid[p] - lo;
  const bool in = q >= 0 && q < cnt;
  const float c = in ? expf(-ell[q] * inv_tau) : -1.0f;
  pk[slot] = make_float4(st[p], st[N + p], st[2 * N + p], c);
  sidx[slot] = p;
  if (g) pg[slot] = in ? make_float4(g[3 * q], g[3 * q + 1], g[3 * q + 2], 0.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Visits the candidate neighbours of the particle at slot s (all particles of
// the 27 cells around its stencil-origin cell, itself included): f(j, xj).
template <class F>
__device__ inline void for_candidates(const Params& P, int scene, const float4& xa, const uint32_t* __restrict__ bins,
                                      int n_bins, const float4* __restrict__ pk, F f) {
  int b[3];
  const float xs[3] = {xa.x, xa.y, xa.z};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float bf = base_floor(grid_coord(xs[d], P));
    b[d] = int(fminf(fmaxf(bf, 0.0f), float(P.n - 3)));
  }
  const uint32_t kbase = uint32_t(scene) * uint32_t(P.MB);
  for (int ox = -1; ox <= 1; ++ox) {
    const int cx = b[0] + ox;
    if (cx < 0 || cx > P.n - 3) continue;
    for (int oy = -1; oy <= 1; ++oy) {
      const int cy = b[1] + oy;
      if (cy < 0 || cy > P.n - 3) continue;
      for (int oz = -1; oz <= 1; ++oz) {
        const int cz = b[2] + oz;
        if (cz < 0 || cz > P.n - 3) continue;
        const uint32_t k = kbase + morton3(uint32_t(cx), uint32_t(cy), uint32_t(cz));
        const int j0 = int(bins[k]);
        const int j1 = (int(k) + 1 < n_bins) ? int(bins[k + 1]) : P.N;
        for (int j = j0; j < j1; ++j) f(j, pk[j]);
      }
    }
  }
}

__global__ void __launch_bounds__(256)
attraction_kernel(Params P, const uint32_t* __restrict__ tag, const uint32_t* __restrict__ bins, int n_bins,
                  const float4* __restrict__ pk, const int* __restrict__ sidx, float h, float weight,
                  float* __restrict__ adj, double* __restrict__ loss) {
  const int N = P.N;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  float L = 0.0f;
  if (s < N) {
    const float4 xa = pk[s];
    if (xa.w >= 0.0f) {
      const int a = sidx[s];
      const float inv_h = 1.0f / h, h2 = h * h;
      float gr[3] = {0.f, 0.f, 0.f};
      for_candidates(P, tag_scene(tag[a]), xa, bins, n_bins, pk, [&](int j, const float4& xj) {
        if (j == s || xj.w < 0.0f) return;
        const float d0 = xa.x - xj.x, d1 = xa.y - xj.y, d2 = xa.z - xj.z;
        const float dd = d0 * d0 + d1 * d1 + d2 * d2;
        if (!(dd > 0.0f && dd < h2)) return;
        const float rd = rsqrtf(dd);  // 1 / d
        const float d = dd * rd;
        const float r2 = dd * inv_h * inv_h, om = 1.0f - r2;
        const float k = om * om * om;
        L += xj.w * d * k;
        const float coef = (xj.w + xa.w) * (k - 6.0f * r2 * om * om) * rd;
        gr[0] += coef * d0;
        gr[1] += coef * d1;
        gr[2] += coef * d2;
      });
#pragma unroll
      for (int d = 0; d < 3; ++d) adj[(long long)d * N + a] += weight * gr[d];
    }
  }
  // block sum of the loss, one FP64 atomic per CTA
  __shared__ float part[8];
  float w = warp_sum(L);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) t += part[i];
    if (t != 0.0f) atomicAdd(loss, double(weight) * double(t));
  }
}

__global__ void __launch_bounds__(256)
share_kernel(Params P, const uint32_t* __restrict__ tag, const int* __restrict__ pid,
             const uint32_t* __restrict__ bins, int n_bins, const float4* __restrict__ pk,
             const float4* __restrict__ pg, const int* __restrict__ sidx, float h, int lo, float* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.N) return;
  const float4 xa = pk[s];
  if (xa.w < 0.0f) return;
  const int a = sidx[s];
  const float inv_h2 = 1.0f / (h * h);
  float acc[3] = {0.f, 0.f, 0.f};
  for_candidates(P, tag_scene(tag[a]), xa, bins, n_bins, pk, [&](int j, const float4& xj) {
    if (xj.w < 0.0f) return;
    const float d0 = xa.x - xj.x, d1 = xa.y - xj.y, d2 = xa.z - xj.z;
    const float r2 = (d0 * d0 + d1 * d1 + d2 * d2) * inv_h2;
    if (!(r2 < 1.0f)) return;
    const float om = 1.0f - r2;
    const float w = xj.w * om * om * om;
    const float4 g = pg[j];
    acc[0] += w * g.x;
    acc[1] += w * g.y;
    acc[2] += w * g.z;
  });
  const int q = pid[a] - lo;
#pragma unroll
  for (int d = 0; d < 3; ++d) out[3 * q + d] = acc[d];
}

void launch_nbr_pack(const Params& P, const float* st, const int* pid, const SortBuffers& sb, const float* ell,
                     const float* g, int lo, int cnt, float tau, NbrBuffers nb, cudaStream_t s) {
  if (P.N == 0) return;
  nbr_pack_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P.N, st, pid, sb.key, sb.rank, sb.bins, ell, g, lo, cnt,
                                                       1.0f / tau, nb.pk, nb.pg, nb.sidx);
}

void launch_attraction(const Params& P, const uint32_t* tag, const SortBuffers& sb, NbrBuffers nb, float radius,
                       float weight, float* adj, double* loss, cudaStream_t s) {
  if (P.N == 0) return;
  attraction_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, tag, sb.bins, sb.n_bins, nb.pk, nb.sidx, radius, weight,
                                                         adj, loss);
}

void launch_share(const Params& P, const uint32_t* tag, const int* pid, const SortBuffers& sb, NbrBuffers nb,
                  float radius, int lo, float* out, cudaStream_t s) {
  if (P.N == 0) return;
  share_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, tag, pid, sb.bins, sb.n_bins, nb.pk, nb.pg, nb.sidx, radius,
                                                    lo, out);
}

}  // namespace mpm
