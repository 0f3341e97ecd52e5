// Grid-based gas solver (paper Sec. 3.2 "Gas", after Stam 1999) and its
// adjoint (App. A: the projection's gradient is written by hand). The step
// and its readings are stated in include/mpm_gas.h.
//
// Every kernel is a stencil over the n^3 cells, one thread per cell, fields
// in SoA FP32 (k fastest, so a warp reads 32 consecutive cells of a row):
//   forward   advect (buoyancy folded into the back-trace and the samples),
//             divergence (+ FP64 block sums for the mean), K damped Jacobi
//             sweeps, gradient subtraction;
//   adjoint   transposed gradient, the same K sweeps, FP64 sums for the mean,
//             transposed divergence with the solid mask, transposed
//             advection (scatter of the trilinear weights by atomics plus the
//             back-trace's derivative), buoyancy.
// The per-step launch sequences are captured once per step index as CUDA
// graphs and replayed.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "mpm_gas.h"

namespace {

constexpr float kOmega = 2.0f / 3.0f;  // Jacobi weight
constexpr int kThreads = 256;
// Launch shape of the cell kernels: a CTA covers 32 cells along k (one warp)
// times 8 rows along j of one i-plane, so no thread divides its linear index.
constexpr int kBx = 32, kBy = 8;

struct Geo {
  int n;
  long long n3;
  float dx, dt_dx, beta_dt, inv2dx;
};

__device__ __forceinline__ long long cid(int n, int i, int j, int k) { return ((long long)i * n + j) * n + k; }

// this thread's cell (i, j, k) and linear index; false outside the grid
__device__ __forceinline__ bool my_cell(int n, int& i, int& j, int& k, long long& c) {
  k = blockIdx.x * kBx + threadIdx.x;
  j = blockIdx.y * kBy + threadIdx.y;
  i = blockIdx.z;
  c = ((long long)i * n + j) * n + k;
  return k < n && j < n;
}

// Neighbour bits of a cell, precomputed once from the solid mask: bit 2a is
// "the +e_a neighbour is a fluid cell", bit 2a + 1 the same for -e_a (a = x,
// y, z); kSolidBit marks a solid cell. Cells outside the grid count as solid.
enum : uint8_t { kSolidBit = 64 };

// trilinear stencil of an index-space point: base corner, fractions, and
// whether the coordinate was clamped (its derivative is then zero)
struct Tri {
  int i0[3];
  float t[3];
  bool cl[3];
};

__device__ __forceinline__ Tri tri_of(const float* X, int n) {
  Tri r;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float hi = float(n - 1);
    r.cl[a] = !(X[a] > 0.0f && X[a] < hi);
    const float x = fminf(fmaxf(X[a], 0.0f), hi);
    int b = int(floorf(x));
    b = min(b, n - 2);
    r.i0[a] = b;
    r.t[a] = x - float(b);
  }
  return r;
}

__device__ __forceinline__ float corner_w(const Tri& T, int a, int b, int c) {
  return (a ? T.t[0] : 1.0f - T.t[0]) * (b ? T.t[1] : 1.0f - T.t[1]) * (c ? T.t[2] : 1.0f - T.t[2]);
}

// d w / d t_axis of corner (a, b, c)
__device__ __forceinline__ float corner_dw(const Tri& T, int axis, int a, int b, int c) {
  const float wa = axis == 0 ? (a ? 1.0f : -1.0f) : (a ? T.t[0] : 1.0f - T.t[0]);
  const float wb = axis == 1 ? (b ? 1.0f : -1.0f) : (b ? T.t[1] : 1.0f - T.t[1]);
  const float wc = axis == 2 ? (c ? 1.0f : -1.0f) : (c ? T.t[2] : 1.0f - T.t[2]);
  return wa * wb * wc;
}

// CTA sum (thread 0's return value), every thread must call it
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double part[kThreads / 32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) part[tid >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (tid == 0)
    for (int w = 0; w < kThreads / 32; ++w) t += part[w];
  return t;
}

__global__ void __launch_bounds__(kThreads)
neighbours_kernel(int n, const uint8_t* __restrict__ solid, uint8_t* __restrict__ nbr) {
  int i, j, k;
  long long c;
  if (!my_cell(n, i, j, k, c)) return;
  auto fl = [&](int a, int b, int e) {
    return a >= 0 && b >= 0 && e >= 0 && a < n && b < n && e < n && solid[cid(n, a, b, e)] == 0;
  };
  uint8_t m = solid[c] ? kSolidBit : 0;
  if (fl(i + 1, j, k)) m |= 1;
  if (fl(i - 1, j, k)) m |= 2;
  if (fl(i, j + 1, k)) m |= 4;
  if (fl(i, j - 1, k)) m |= 8;
  if (fl(i, j, k + 1)) m |= 16;
  if (fl(i, j, k - 1)) m |= 32;
  nbr[c] = m;
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
// The fields an advection samples, packed per cell: (u_x, u_y + dt beta d,
// u_z, d), i.e. the buoyancy-updated velocity and the density, so that a
// trilinear corner is one 16-byte load (and, in the adjoint, one vector
// atomic).
__global__ void __launch_bounds__(kThreads)
pack_kernel(Geo g, const float* __restrict__ u, const float* __restrict__ d, float4* __restrict__ pk) {
  int i, j, k;
  long long c;
  if (!my_cell(g.n, i, j, k, c)) return;
  const long long n3 = g.n3;
  const float dc = d[c];
  pk[c] = make_float4(u[c], u[n3 + c] + g.beta_dt * dc, u[2 * n3 + c], dc);
}

__global__ void __launch_bounds__(kThreads)
advect_kernel(Geo g, const float4* __restrict__ pk, const uint8_t* __restrict__ nbr, float* __restrict__ un,
              float* __restrict__ dn) {
  int i, j, k;
  long long c;
  if (!my_cell(g.n, i, j, k, c)) return;
  const long long n3 = g.n3;
  if (nbr[c] & kSolidBit) {
    un[c] = un[n3 + c] = un[2 * n3 + c] = dn[c] = 0.0f;
    return;
  }
  const float4 ub = pk[c];
  const float X[3] = {i - g.dt_dx * ub.x, j - g.dt_dx * ub.y, k - g.dt_dx * ub.z};
  const Tri T = tri_of(X, g.n);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float4 q = pk[cid(g.n, T.i0[0] + a, T.i0[1] + b, T.i0[2] + e)];
        const float w = corner_w(T, a, b, e);
        v.x += w * q.x;
        v.y += w * q.y;
        v.z += w * q.z;
        v.w += w * q.w;
      }
  un[c] = v.x;
  un[n3 + c] = v.y;
  un[2 * n3 + c] = v.z;
  dn[c] = v.w;
}

// b = divergence of un on fluid cells (solid neighbours hold zero velocity);
// FP64 sum of b into *sum
__global__ void __launch_bounds__(kThreads)
divergence_kernel(Geo g, const float* __restrict__ un, const uint8_t* __restrict__ nbr, float* __restrict__ b,
                  double* __restrict__ sum) {
  int i, j, k;
  long long c;
  const bool in = my_cell(g.n, i, j, k, c);
  float v = 0.0f;
  if (in) {
    const uint8_t m = nbr[c];
    if (!(m & kSolidBit)) {
      const long long n1 = g.n, n2 = (long long)g.n * g.n, n3 = g.n3;
      float s = 0.0f;
      if (m & 1) s += un[c + n2];
      if (m & 2) s -= un[c - n2];
      if (m & 4) s += un[n3 + c + n1];
      if (m & 8) s -= un[n3 + c - n1];
      if (m & 16) s += un[2 * n3 + c + 1];
      if (m & 32) s -= un[2 * n3 + c - 1];
      v = s * g.inv2dx;
    }
    b[c] = v;
  }
  const double t = block_sum(double(v));
  if (threadIdx.x == 0 && threadIdx.y == 0 && t != 0.0) atomicAdd(sum, t);
}

// FP64 sum over the fluid cells of x into *sum
__global__ void __launch_bounds__(kThreads)
fluid_sum_kernel(Geo g, const float* __restrict__ x, const uint8_t* __restrict__ nbr, double* __restrict__ sum) {
  int i, j, k;
  long long c;
  const bool in = my_cell(g.n, i, j, k, c);
  const float v = (in && !(nbr[c] & kSolidBit)) ? x[c] : 0.0f;
  const double t = block_sum(double(v));
  if (threadIdx.x == 0 && threadIdx.y == 0 && t != 0.0) atomicAdd(sum, t);
}

// mean = sum / n_fluid as one float, for the sweeps to read
__global__ void mean_kernel(const double* __restrict__ sum, double inv_nfluid, float* __restrict__ mean) {
  *mean = float(*sum * inv_nfluid);
}

// One damped Jacobi sweep on the zero-flux Laplacian of the fluid cells:
// p_out = p_in / 3 + (2/3) (sum_fluid-nbr p_in - dx^2 (rhs - mean)) / n_fluid-nbr,
// mean read from *mean when given; first: p_in = 0.
__global__ void __launch_bounds__(kThreads)
jacobi_kernel(Geo g, const float* __restrict__ p_in, float* __restrict__ p_out, const float* __restrict__ rhs,
              const uint8_t* __restrict__ nbr, const float* __restrict__ mean_p, int first) {
  int i, j, k;
  long long c;
  if (!my_cell(g.n, i, j, k, c)) return;
  const int n = g.n;
  const long long n1 = n, n2 = (long long)n * n;
  // neighbour loads issued before the neighbour bits arrive (in-grid
  // addresses; a neighbour outside the grid reads the cell itself), then
  // weighted by the bits
  float q[6], pc = 0.0f, r = 0.0f;
  if (!first) {
    q[0] = p_in[i + 1 < n ? c + n2 : c];
    q[1] = p_in[i > 0 ? c - n2 : c];
    q[2] = p_in[j + 1 < n ? c + n1 : c];
    q[3] = p_in[j > 0 ? c - n1 : c];
    q[4] = p_in[k + 1 < n ? c + 1 : c];
    q[5] = p_in[k > 0 ? c - 1 : c];
    pc = p_in[c];
  }
  r = rhs[c];
  const uint8_t m = nbr[c];
  if (m & kSolidBit) {
    p_out[c] = 0.0f;
    return;
  }
  float s = 0.0f;
  if (!first) {
#pragma unroll
    for (int t = 0; t < 6; ++t) s += (m & (1 << t)) ? q[t] : 0.0f;
  }
  const int nf = __popc(m & 63);
  const float mean = mean_p ? *mean_p : 0.0f;
  // 1 / n_fluid-nbr for n = 0..6 (no fluid neighbour: no update)
  const float inv_nf = nf == 0 ? 0.0f : nf == 1 ? 1.0f : nf == 2 ? 0.5f : nf == 3 ? (1.0f / 3.0f) : nf == 4 ? 0.25f
                     : nf == 5 ? 0.2f : (1.0f / 6.0f);
  const float upd = (s - g.dx * g.dx * (r - mean)) * inv_nf;
  p_out[c] = (1.0f - kOmega) * pc + kOmega * upd;
}

// The same sweep for n a multiple of 4: each thread updates 4 consecutive
// cells along k with 16-byte loads of p, the right-hand side and the
// neighbour bits (8 loads and one store for 4 cells instead of 9 and one per
// cell). A CTA covers 128 cells along k times 8 rows along j.
__device__ __forceinline__ float f4(const float4& v, int t) { return t == 0 ? v.x : t == 1 ? v.y : t == 2 ? v.z : v.w; }

__global__ void __launch_bounds__(kThreads)
jacobi4_kernel(Geo g, const float* __restrict__ p_in, float* __restrict__ p_out, const float* __restrict__ rhs,
               const uint8_t* __restrict__ nbr, const float* __restrict__ mean_p, int first) {
  const int n = g.n;
  const int k0 = (blockIdx.x * kBx + threadIdx.x) * 4;
  const int j = blockIdx.y * kBy + threadIdx.y;
  const int i = blockIdx.z;
  if (k0 >= n || j >= n) return;
  const int n1 = n, n2 = n * n;
  const int c = (i * n + j) * n + k0;
  float4 P = make_float4(0.f, 0.f, 0.f, 0.f), Q[4];
  float pl = 0.0f, pr = 0.0f;
  if (!first) {
    P = *reinterpret_cast<const float4*>(p_in + c);
    Q[0] = *reinterpret_cast<const float4*>(p_in + (i + 1 < n ? c + n2 : c));
    Q[1] = *reinterpret_cast<const float4*>(p_in + (i > 0 ? c - n2 : c));
    Q[2] = *reinterpret_cast<const float4*>(p_in + (j + 1 < n ? c + n1 : c));
    Q[3] = *reinterpret_cast<const float4*>(p_in + (j > 0 ? c - n1 : c));
    pl = k0 > 0 ? p_in[c - 1] : 0.0f;
    pr = k0 + 4 < n ? p_in[c + 4] : 0.0f;
  }
  const float4 R = *reinterpret_cast<const float4*>(rhs + c);
  const uint32_t M4 = *reinterpret_cast<const uint32_t*>(nbr + c);
  const float mean = mean_p ? *mean_p : 0.0f;
  const float h2 = g.dx * g.dx;
  float out[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const uint32_t m = (M4 >> (8 * t)) & 0xffu;
    if (m & kSolidBit) {
      out[t] = 0.0f;
      continue;
    }
    float s = 0.0f, pc = 0.0f;
    if (!first) {
      const float zp = t < 3 ? f4(P, t + 1) : pr;
      const float zm = t > 0 ? f4(P, t - 1) : pl;
      s = ((m & 1) ? f4(Q[0], t) : 0.0f) + ((m & 2) ? f4(Q[1], t) : 0.0f) + ((m & 4) ? f4(Q[2], t) : 0.0f) +
          ((m & 8) ? f4(Q[3], t) : 0.0f) + ((m & 16) ? zp : 0.0f) + ((m & 32) ? zm : 0.0f);
      pc = f4(P, t);
    }
    const int nf = __popc(m & 63u);
    const float inv_nf = nf == 0 ? 0.0f : nf == 1 ? 1.0f : nf == 2 ? 0.5f : nf == 3 ? (1.0f / 3.0f) : nf == 4 ? 0.25f
                       : nf == 5 ? 0.2f : (1.0f / 6.0f);
    out[t] = (1.0f - kOmega) * pc + kOmega * (s - h2 * (f4(R, t) - mean)) * inv_nf;
  }
  *reinterpret_cast<float4*>(p_out + c) = make_float4(out[0], out[1], out[2], out[3]);
}

// un -= central-difference gradient of p (p mirrored across solid faces)
__global__ void __launch_bounds__(kThreads)
gradient_kernel(Geo g, const float* __restrict__ p, const uint8_t* __restrict__ nbr, float* __restrict__ un) {
  int i, j, k;
  long long c;
  if (!my_cell(g.n, i, j, k, c)) return;
  const uint8_t m = nbr[c];
  if (m & kSolidBit) return;
  const long long n1 = g.n, n2 = (long long)g.n * g.n, n3 = g.n3;
  const float pc = p[c];
  const long long st[3] = {n2, n1, 1};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float pp = (m & (1 << (2 * a))) ? p[c + st[a]] : pc;
    const float pm = (m & (2 << (2 * a))) ? p[c - st[a]] : pc;
    un[a * n3 + c] -= (pp - pm) * g.inv2dx;
  }
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
// t = G^T v on fluid cells (v = adjoint of the projected velocity): cell c - e
// (fluid, its + neighbour is c) contributes +v(c - e), cell c + e contributes
// -v(c + e), and c mirrors its missing neighbours onto itself.
__global__ void __launch_bounds__(kThreads)
gradient_t_kernel(Geo g, const float* __restrict__ v, const uint8_t* __restrict__ nbr, float* __restrict__ t) {
  int i, j, k;
  long long c;
  if (!my_cell(g.n, i, j, k, c)) return;
  const uint8_t m = nbr[c];
  if (m & kSolidBit) {
    t[c] = 0.0f;
    return;
  }
  const long long n1 = g.n, n2 = (long long)g.n * g.n, n3 = g.n3;
  const long long st[3] = {n2, n1, 1};
  float s = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float* va = v + a * n3;
    const bool fh = m & (1 << (2 * a)), fl = m & (2 << (2 * a));
    if (fl) s += va[c - st[a]];
    if (fh) s -= va[c + st[a]];
    if (!fh) s += va[c];
    if (!fl) s -= va[c];
  }
  t[c] = s * g.inv2dx;
}

// ubar = v - D^T (m - mean) on fluid cells, 0 on solid cells (the advection's
// solid mask); m = the swept adjoint, *mean_p its mean over the fluid cells.
__global__ void __launch_bounds__(kThreads)
divergence_t_kernel(Geo g, const float* __restrict__ v, const float* __restrict__ mm, const uint8_t* __restrict__ nbr,
                    const float* __restrict__ mean_p, float* __restrict__ ubar) {
  int i, j, k;
  long long c;
  if (!my_cell(g.n, i, j, k, c)) return;
  const long long n1 = g.n, n2 = (long long)g.n * g.n, n3 = g.n3;
  const uint8_t m = nbr[c];
  if (m & kSolidBit) {
    ubar[c] = ubar[n3 + c] = ubar[2 * n3 + c] = 0.0f;
    return;
  }
  const float mean = *mean_p;
  const long long st[3] = {n2, n1, 1};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // b(i) = (u(i + e) - u(i - e)) / 2dx on fluid i: u(c) enters b(c - e) with +, b(c + e) with -
    float s = 0.0f;
    if (m & (2 << (2 * a))) s += mm[c - st[a]] - mean;
    if (m & (1 << (2 * a))) s -= mm[c + st[a]] - mean;
    ubar[a * n3 + c] = v[a * n3 + c] - s * g.inv2dx;
  }
}

// Transposed advection: scatter (ubar_adv, dbar_adv) of every fluid cell onto
// the trilinear corners (one vector atomic per corner) and add the
// back-trace's derivative to the cell's own velocity adjoint. acc (float4
// per cell) is zero on entry and receives the adjoint of the packed fields
// (buoyancy-updated velocity, density).
__global__ void __launch_bounds__(kThreads)
advect_t_kernel(Geo g, const float4* __restrict__ pk, const uint8_t* __restrict__ nbr,
                const float* __restrict__ ubar, const float* __restrict__ dbar, float4* __restrict__ acc) {
  int i, j, k;
  long long c;
  if (!my_cell(g.n, i, j, k, c)) return;
  if (nbr[c] & kSolidBit) return;
  const long long n3 = g.n3;
  const float4 ub = pk[c];
  const float X[3] = {i - g.dt_dx * ub.x, j - g.dt_dx * ub.y, k - g.dt_dx * ub.z};
  const Tri T = tri_of(X, g.n);
  const float4 A = make_float4(ubar[c], ubar[n3 + c], ubar[2 * n3 + c], dbar[c]);
  const bool any = A.x != 0.0f || A.y != 0.0f || A.z != 0.0f || A.w != 0.0f;
  if (!any) return;
  float gX[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const long long q = cid(g.n, T.i0[0] + a, T.i0[1] + b, T.i0[2] + e);
        const float w = corner_w(T, a, b, e);
        atomicAdd(acc + q, make_float4(w * A.x, w * A.y, w * A.z, w * A.w));
        const float4 v = pk[q];
        const float s = A.x * v.x + A.y * v.y + A.z * v.z + A.w * v.w;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) gX[ax] += corner_dw(T, ax, a, b, e) * s;
      }
  const float4 own = make_float4(T.cl[0] ? 0.0f : -g.dt_dx * gX[0], T.cl[1] ? 0.0f : -g.dt_dx * gX[1],
                                 T.cl[2] ? 0.0f : -g.dt_dx * gX[2], 0.0f);
  atomicAdd(acc + c, own);
}

// adjoint of the step's input: ubar_n = acc.xyz, dbar_n = acc.w + beta dt acc.y,
// zero on solid cells (the state there is identically zero)
__global__ void __launch_bounds__(kThreads)
finish_t_kernel(Geo g, const float4* __restrict__ acc, const uint8_t* __restrict__ nbr, float* __restrict__ ubar,
                float* __restrict__ dbar) {
  int i, j, k;
  long long c;
  if (!my_cell(g.n, i, j, k, c)) return;
  const long long n3 = g.n3;
  const bool s = nbr[c] & kSolidBit;
  const float4 a = acc[c];
  ubar[c] = s ? 0.0f : a.x;
  ubar[n3 + c] = s ? 0.0f : a.y;
  ubar[2 * n3 + c] = s ? 0.0f : a.z;
  dbar[c] = s ? 0.0f : a.w + g.beta_dt * a.y;
}

// zero `fields` consecutive n^3 fields of x on solid cells
__global__ void __launch_bounds__(kThreads)
mask_kernel(Geo g, const uint8_t* __restrict__ nbr, float* __restrict__ x, int fields) {
  int i, j, k;
  long long c;
  if (!my_cell(g.n, i, j, k, c) || !(nbr[c] & kSolidBit)) return;
  for (int f = 0; f < fields; ++f) x[f * g.n3 + c] = 0.0f;
}

__global__ void add_kernel(long long m, const float* __restrict__ a, float* __restrict__ b) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < m) b[c] += a[c];
}

}  // namespace

// ---------------------------------------------------------------------------
// handle and C-ABI
// ---------------------------------------------------------------------------
struct mpm_gas {
  gas_config cfg{};
  Geo g{};
  cudaStream_t stream = nullptr, cstream = nullptr;
  int nfluid = 0;
  uint8_t* solid = nullptr;
  uint8_t* nbr = nullptr;  // neighbour bits of every cell
  float* states = nullptr;  // (max_steps + 1) x 4 n^3: u (3), d
  float *un = nullptr, *b = nullptr, *p0 = nullptr, *p1 = nullptr;
  float *adj = nullptr, *adj2 = nullptr, *acc = nullptr;  // 4 n^3 each
  float* pack = nullptr;  // 4 n^3: packed fields (float4 per cell) of the step being advected
  double* sum = nullptr;
  float* mean = nullptr;
  int step = 0;
  bool started = false, seeds = false;
  long long launches = 0;
  std::vector<cudaGraphExec_t> fwd, bwd;
  std::vector<long long> fwd_launches, bwd_launches;
  std::string last_error;
};

namespace {

sim_status gfail(gas_h h, sim_status s, const std::string& m) {
  if (h) h->last_error = m;
  return s;
}

sim_status gcuda(gas_h h, cudaError_t e, const char* where) {
  return gfail(h, SIM_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

inline int nblocks(long long m) { return int((m + kThreads - 1) / kThreads); }
inline dim3 cell_grid(int n) { return dim3((n + kBx - 1) / kBx, (n + kBy - 1) / kBy, n); }
const dim3 kCellBlock(kBx, kBy);

// one Jacobi sweep, 4 cells a thread when n allows 16-byte rows
void sweep(const Geo& g, const float* p_in, float* p_out, const float* rhs, const uint8_t* nbr, const float* mean,
           int first, cudaStream_t st) {
  if (g.n % 4 == 0) {
    const dim3 gr((g.n / 4 + kBx - 1) / kBx, (g.n + kBy - 1) / kBy, g.n);
    jacobi4_kernel<<<gr, kCellBlock, 0, st>>>(g, p_in, p_out, rhs, nbr, mean, first);
  } else {
    jacobi_kernel<<<cell_grid(g.n), kCellBlock, 0, st>>>(g, p_in, p_out, rhs, nbr, mean, first);
  }
}

float* state_ptr(gas_h h, int s) { return h->states + (size_t)s * 4 * h->g.n3; }

// Launches of one forward step s -> s + 1 on stream st; returns the launch count.
long long enqueue_forward(gas_h h, int s, cudaStream_t st) {
  const Geo& g = h->g;
  const long long n3 = g.n3;
  const dim3 gr = cell_grid(g.n);
  const float* in = state_ptr(h, s);
  float* out = state_ptr(h, s + 1);
  const double inv_nf = h->nfluid > 0 ? 1.0 / h->nfluid : 0.0;
  float4* pk = reinterpret_cast<float4*>(h->pack);
  pack_kernel<<<gr, kCellBlock, 0, st>>>(g, in, in + 3 * n3, pk);
  advect_kernel<<<gr, kCellBlock, 0, st>>>(g, pk, h->nbr, h->un, out + 3 * n3);
  cudaMemsetAsync(h->sum, 0, sizeof(double), st);
  divergence_kernel<<<gr, kCellBlock, 0, st>>>(g, h->un, h->nbr, h->b, h->sum);
  mean_kernel<<<1, 1, 0, st>>>(h->sum, inv_nf, h->mean);
  float* pa = h->p0;
  float* pb = h->p1;
  for (int it = 0; it < h->cfg.jacobi_iters; ++it) {
    sweep(g, pa, pb, h->b, h->nbr, h->mean, it == 0, st);
    float* t = pa;
    pa = pb;
    pb = t;
  }
  gradient_kernel<<<gr, kCellBlock, 0, st>>>(g, pa, h->nbr, h->un);
  cudaMemcpyAsync(out, h->un, sizeof(float) * 3 * n3, cudaMemcpyDeviceToDevice, st);
  return 5 + h->cfg.jacobi_iters;
}

// Launches of the adjoint of step s (adj holds the adjoint of state s + 1,
// and receives the adjoint of state s).
long long enqueue_backward(gas_h h, int s, cudaStream_t st) {
  const Geo& g = h->g;
  const long long n3 = g.n3;
  const dim3 gr = cell_grid(g.n);
  const float* in = state_ptr(h, s);
  const double inv_nf = h->nfluid > 0 ? 1.0 / h->nfluid : 0.0;
  float* v = h->adj;  // u (3 n^3), d (n^3)
  // projection: ubar_pre = v - D^T M J G^T v
  gradient_t_kernel<<<gr, kCellBlock, 0, st>>>(g, v, h->nbr, h->b);
  float* pa = h->p0;
  float* pb = h->p1;
  for (int it = 0; it < h->cfg.jacobi_iters; ++it) {
    sweep(g, pa, pb, h->b, h->nbr, nullptr, it == 0, st);
    float* t = pa;
    pa = pb;
    pb = t;
  }
  cudaMemsetAsync(h->sum, 0, sizeof(double), st);
  fluid_sum_kernel<<<gr, kCellBlock, 0, st>>>(g, pa, h->nbr, h->sum);
  mean_kernel<<<1, 1, 0, st>>>(h->sum, inv_nf, h->mean);
  divergence_t_kernel<<<gr, kCellBlock, 0, st>>>(g, v, pa, h->nbr, h->mean, h->adj2);
  // the density output is not projected; its adjoint passes the solid mask
  cudaMemcpyAsync(h->adj2 + 3 * n3, v + 3 * n3, sizeof(float) * n3, cudaMemcpyDeviceToDevice, st);
  mask_kernel<<<gr, kCellBlock, 0, st>>>(g, h->nbr, h->adj2 + 3 * n3, 1);
  // advection and buoyancy, from the packed fields of step s
  float4* pk = reinterpret_cast<float4*>(h->pack);
  pack_kernel<<<gr, kCellBlock, 0, st>>>(g, in, in + 3 * n3, pk);
  float4* acc = reinterpret_cast<float4*>(h->acc);
  cudaMemsetAsync(acc, 0, sizeof(float4) * n3, st);
  advect_t_kernel<<<gr, kCellBlock, 0, st>>>(g, pk, h->nbr, h->adj2, h->adj2 + 3 * n3, acc);
  finish_t_kernel<<<gr, kCellBlock, 0, st>>>(g, acc, h->nbr, h->adj, h->adj + 3 * n3);
  return 8 + h->cfg.jacobi_iters;
}

sim_status run_graph(gas_h h, std::vector<cudaGraphExec_t>& cache, std::vector<long long>& counts, int s,
                     long long (*enq)(gas_h, int, cudaStream_t)) {
  if (!cache[s]) {
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(h->cstream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return gcuda(h, e, "gas graph capture");
    counts[s] = enq(h, s, h->cstream);
    e = cudaStreamEndCapture(h->cstream, &graph);
    if (e != cudaSuccess) return gcuda(h, e, "gas graph capture");
    e = cudaGraphInstantiate(&cache[s], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return gcuda(h, e, "gas graph instantiate");
  }
  cudaError_t e = cudaGraphLaunch(cache[s], h->stream);
  if (e != cudaSuccess) return gcuda(h, e, "gas graph launch");
  h->launches += counts[s];
  return SIM_OK;
}

sim_status sync(gas_h h, const char* where) {
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? SIM_OK : gcuda(h, e, where);
}

cudaError_t copy_in(gas_h h, void* dst, const void* src, size_t bytes, int on_device) {
  return cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
}

cudaError_t copy_out(gas_h h, void* dst, const void* src, size_t bytes, int on_device) {
  return cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
}

}  // namespace

extern "C" {

sim_status gas_create(const gas_config* cfg, const uint8_t* solid, gas_h* out) {
  if (!cfg || !solid || !out) return SIM_E_ARG;
  *out = nullptr;
  if (cfg->n < 8 || cfg->n > 512 || !(cfg->dt > 0.0f) || cfg->jacobi_iters < 1 || cfg->max_steps < 1) return SIM_E_ARG;
  gas_h h = new mpm_gas();
  h->cfg = *cfg;
  const int n = cfg->n;
  Geo& g = h->g;
  g.n = n;
  g.n3 = (long long)n * n * n;
  g.dx = 1.0f / n;
  g.dt_dx = cfg->dt * n;
  g.beta_dt = cfg->dt * cfg->buoyancy;
  g.inv2dx = 0.5f * n;
  h->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  const size_t n3 = (size_t)g.n3;
  for (size_t c = 0; c < n3; ++c) h->nfluid += solid[c] ? 0 : 1;
  bool ok = cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaMalloc(&h->solid, n3) == cudaSuccess;
  ok = ok && cudaMalloc(&h->nbr, n3) == cudaSuccess;
  ok = ok && cudaMalloc(&h->states, sizeof(float) * 4 * n3 * (size_t)(cfg->max_steps + 1)) == cudaSuccess;
  float** bufs[8] = {&h->un, &h->b, &h->p0, &h->p1, &h->adj, &h->adj2, &h->acc, &h->pack};
  const size_t sizes[8] = {3 * n3, n3, n3, n3, 4 * n3, 4 * n3, 4 * n3, 4 * n3};
  for (int q = 0; q < 8 && ok; ++q) ok = cudaMalloc(bufs[q], sizeof(float) * sizes[q]) == cudaSuccess;
  ok = ok && cudaMalloc(&h->sum, sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->mean, sizeof(float)) == cudaSuccess;
  ok = ok && cudaMemcpy(h->solid, solid, n3, cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok) {
    neighbours_kernel<<<cell_grid(n), kCellBlock>>>(n, h->solid, h->nbr);
    ok = cudaDeviceSynchronize() == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    gas_destroy(h);
    return SIM_E_OOM;
  }
  h->fwd.assign(cfg->max_steps, nullptr);
  h->bwd.assign(cfg->max_steps, nullptr);
  h->fwd_launches.assign(cfg->max_steps, 0);
  h->bwd_launches.assign(cfg->max_steps, 0);
  *out = h;
  return SIM_OK;
}

sim_status gas_destroy(gas_h h) {
  if (!h) return SIM_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto e : h->fwd)
    if (e) cudaGraphExecDestroy(e);
  for (auto e : h->bwd)
    if (e) cudaGraphExecDestroy(e);
  void* ptrs[13] = {h->solid, h->nbr, h->states, h->un, h->b, h->p0, h->p1, h->adj, h->adj2, h->acc, h->sum,
                    h->mean, h->pack};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->cstream) cudaStreamDestroy(h->cstream);
  delete h;
  return SIM_OK;
}

sim_status gas_set_state(gas_h h, const float* u, const float* d, int on_device) {
  if (!h) return SIM_E_ARG;
  if (!u || !d) return gfail(h, SIM_E_ARG, "gas_set_state: null u or d");
  const long long n3 = h->g.n3;
  float* s0 = state_ptr(h, 0);
  cudaError_t e = copy_in(h, s0, u, sizeof(float) * 3 * n3, on_device);
  if (e == cudaSuccess) e = copy_in(h, s0 + 3 * n3, d, sizeof(float) * n3, on_device);
  if (e != cudaSuccess) return gcuda(h, e, "gas_set_state");
  mask_kernel<<<cell_grid(h->g.n), kCellBlock, 0, h->stream>>>(h->g, h->nbr, s0, 4);
  cudaMemsetAsync(h->adj, 0, sizeof(float) * 4 * n3, h->stream);
  h->launches += 1;
  h->step = 0;
  h->started = true;
  h->seeds = false;
  return sync(h, "gas_set_state");
}

sim_status gas_step(gas_h h, int n_steps) {
  if (!h) return SIM_E_ARG;
  if (!h->started) return gfail(h, SIM_E_STATE, "gas_step: no state set");
  if (n_steps < 0 || h->step + n_steps > h->cfg.max_steps) return gfail(h, SIM_E_ARG, "gas_step: beyond max_steps");
  for (int q = 0; q < n_steps; ++q) {
    sim_status st = run_graph(h, h->fwd, h->fwd_launches, h->step, enqueue_forward);
    if (st != SIM_OK) return st;
    ++h->step;
  }
  return sync(h, "gas_step");
}

sim_status gas_get_state(gas_h h, float* u, float* d, int on_device) {
  if (!h) return SIM_E_ARG;
  if (!h->started) return gfail(h, SIM_E_STATE, "gas_get_state: no state set");
  const long long n3 = h->g.n3;
  const float* s = state_ptr(h, h->step);
  cudaError_t e = cudaSuccess;
  if (u) e = copy_out(h, u, s, sizeof(float) * 3 * n3, on_device);
  if (e == cudaSuccess && d) e = copy_out(h, d, s + 3 * n3, sizeof(float) * n3, on_device);
  if (e != cudaSuccess) return gcuda(h, e, "gas_get_state");
  return sync(h, "gas_get_state");
}

sim_status gas_add_grad(gas_h h, const float* dLdu, const float* dLdd, int on_device) {
  if (!h) return SIM_E_ARG;
  if (!h->started) return gfail(h, SIM_E_STATE, "gas_add_grad: no state set");
  const long long n3 = h->g.n3;
  const float* src[2] = {dLdu, dLdd};
  const long long cnt[2] = {3 * n3, n3};
  const long long off[2] = {0, 3 * n3};
  for (int q = 0; q < 2; ++q) {
    if (!src[q]) continue;
    cudaError_t e = copy_in(h, h->acc, src[q], sizeof(float) * cnt[q], on_device);
    if (e != cudaSuccess) return gcuda(h, e, "gas_add_grad");
    add_kernel<<<nblocks(cnt[q]), kThreads, 0, h->stream>>>(cnt[q], h->acc, h->adj + off[q]);
    h->launches += 1;
  }
  h->seeds = true;
  return sync(h, "gas_add_grad");
}

sim_status gas_backward(gas_h h, float* dLdu0, float* dLdd0, int on_device) {
  if (!h) return SIM_E_ARG;
  if (!h->started || h->step == 0) return gfail(h, SIM_E_STATE, "gas_backward: no step taken");
  for (int s = h->step - 1; s >= 0; --s) {
    sim_status st = run_graph(h, h->bwd, h->bwd_launches, s, enqueue_backward);
    if (st != SIM_OK) return st;
  }
  const long long n3 = h->g.n3;
  cudaError_t e = cudaSuccess;
  if (dLdu0) e = copy_out(h, dLdu0, h->adj, sizeof(float) * 3 * n3, on_device);
  if (e == cudaSuccess && dLdd0) e = copy_out(h, dLdd0, h->adj + 3 * n3, sizeof(float) * n3, on_device);
  if (e != cudaSuccess) return gcuda(h, e, "gas_backward");
  cudaMemsetAsync(h->adj, 0, sizeof(float) * 4 * n3, h->stream);
  h->seeds = false;
  return sync(h, "gas_backward");
}

long long gas_kernel_launches(gas_h h) { return h ? h->launches : 0; }

const char* gas_last_error(gas_h h) { return h ? h->last_error.c_str() : "null gas handle"; }

}  // extern "C"
