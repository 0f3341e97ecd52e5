// Shared device-side definitions of the MPM library: step parameters, particle
// state layout, small vector helpers and atomics.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpm {

constexpr int kMaxMat = 8;
constexpr int kBlockEdge = 4;        // grid blocks of 4^3 nodes
constexpr int kStateFields = 24;     // x3 v3 C9 F9 (SoA, field f at f * N)
constexpr int kToolFields = 13;      // p3 q4 pdot3 omega3 per scene per step
constexpr int kToolGradFields = 18;  // p3 R9 pdot3 omega3 per scene per step

// error word bits
constexpr int kErrDomain = 1;
constexpr int kErrNaN = 2;
constexpr int kErrTimeout = 4;
constexpr int kErrArg = 8;      // invalid per-particle input (material index)

enum : int { kLiquid = 0, kVonMises = 1, kDruckerPrager = 2, kBoxYield = 3, kViscousLiquid = 4, kRigid = 5 };
// Liquids carry J = det F only (F reset to J^(1/3) I every step); a viscous
// liquid also needs its C to rebuild the step's trial F.
__host__ __device__ inline bool is_liquid(int kind) { return kind == kLiquid || kind == kViscousLiquid; }

struct MatParams {
  int kind;
  float mass;     // rho * V_p
  float vol;      // V_p
  float mu, lam;  // Lame parameters (liquid: mu = 0, lam = K)
  float k_yield;  // von Mises: tau_Y / (2 mu); box yield: theta_c
  float c_dp;     // Drucker-Prager: alpha (3 lam + 2 mu) / (2 mu); box yield: theta_s
  float pad;
};

struct Params {
  int n;          // nodes per axis
  int nb;         // blocks per axis (n / 4 rounded up)
  int S;          // scenes
  int N;          // particles (all scenes)
  long long n3;   // nodes per scene
  int NB;         // blocks per scene
  int MB;         // Morton codes per scene: cells (next power of two of n, cubed)
  float dx, inv_dx, dt;
  float g[3];
  int bound;
  int n_mat;
  // particles are sorted water first: [0, Nl) water, [Nl, N) every other
  // material; only those have F_p and SVD slots (stride Ns = N - Nl)
  int Nl, Ns;
  MatParams mat[kMaxMat];
  int ext;        // 1 if a material is box yield, viscous liquid or rigid (kernels built with those branches)
  int tool;
  float half[3];
  float eps_c, inv_ell, mu_f;
};

// Ask L2 for the line holding *p ahead of its use (no register, no fault on a
// valid address; only ever given addresses of the particle's own fields).
__device__ __forceinline__ void prefetch_l2(const float* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Slot of entry k of a particle p that is not water (F_p, the SVD of the trial
// F) in arrays of Ns entries per field.
__device__ inline long long sslot(const Params& P, int k, int p) { return (long long)k * P.Ns + (p - P.Nl); }

// Particle tag: material in the low 8 bits, scene above.
__host__ __device__ inline int tag_mat(uint32_t t) { return int(t & 0xffu); }
__host__ __device__ inline int tag_scene(uint32_t t) { return int(t >> 8); }

// ---------------------------------------------------------------------------
// quadratic B-spline stencil
// ---------------------------------------------------------------------------
struct Stencil {
  int base[3];
  float f[3];
  float w[3][3];   // w[d][o]
  float dw[3][3];  // dw[d][o] = d w / d f
};

// x / dx and floor(x / dx - 0.5) with each operation rounded on its own (no
// contraction into an FMA), so that every kernel that derives a particle's
// stencil origin gets the same cell.
__device__ inline float grid_coord(float x, const Params& P) { return __fmul_rn(x, P.inv_dx); }
__device__ inline float base_floor(float xs) { return floorf(__fsub_rn(xs, 0.5f)); }

// base = floor(x / dx - 0.5) clamped to [0, n - 3]; returns false if the
// unclamped base left that range or x is not finite.
__device__ inline bool make_stencil(const float x[3], const Params& P, Stencil& s) {
  bool ok = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float xs = grid_coord(x[d], P);
    float bf = base_floor(xs);
    float f;
    if (!(bf >= 0.0f && bf <= float(P.n - 3))) {  // also catches NaN
      // outside the grid: report it and use the nearest valid stencil so that
      // every access stays in bounds and the weights stay a partition of unity
      ok = false;
      bf = fminf(fmaxf(bf, 0.0f), float(P.n - 3));
      f = (xs == xs) ? fminf(fmaxf(xs - bf, 0.5f), 1.5f) : 1.0f;
    } else {
      f = xs - bf;
    }
    int b = int(bf);
    s.base[d] = b;
    s.f[d] = f;
    float a = 1.5f - f, c = f - 1.0f, e = f - 0.5f;
    s.w[d][0] = 0.5f * a * a;
    s.w[d][1] = 0.75f - c * c;
    s.w[d][2] = 0.5f * e * e;
    s.dw[d][0] = -a;
    s.dw[d][1] = -2.0f * c;
    s.dw[d][2] = e;
  }
  return ok;
}

__device__ inline long long node_index(const Params& P, int scene, int i, int j, int k) {
  return (long long)scene * P.n3 + ((long long)i * P.n + j) * P.n + k;
}

// Morton (Z-order) code of a cell coordinate (up to 10 bits per axis): cells
// that are close in space are close in this order.
__host__ __device__ inline uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__host__ __device__ inline uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  return (spread3(x) << 2) | (spread3(y) << 1) | spread3(z);
}

__device__ inline int block_of_base(const Params& P, const int b[3]) {
  return ((b[0] / kBlockEdge) * P.nb + b[1] / kBlockEdge) * P.nb + b[2] / kBlockEdge;
}

// ---------------------------------------------------------------------------
// small matrix helpers (row-major 3x3 in float[9])
// ---------------------------------------------------------------------------
__device__ inline void mat_mul(const float* A, const float* B, float* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      C[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}
// C = A^T B
__device__ inline void mat_tmul(const float* A, const float* B, float* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      C[3 * r + c] = A[r] * B[c] + A[3 + r] * B[3 + c] + A[6 + r] * B[6 + c];
}
// C = A B^T
__device__ inline void mat_mult(const float* A, const float* B, float* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      C[3 * r + c] = A[3 * r] * B[3 * c] + A[3 * r + 1] * B[3 * c + 1] + A[3 * r + 2] * B[3 * c + 2];
}
__device__ inline float det3(const float* A) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}
// cofactor matrix: cof(A) = det(A) A^{-T}
__device__ inline void cof3(const float* A, float* K) {
  K[0] = A[4] * A[8] - A[5] * A[7];
  K[1] = A[5] * A[6] - A[3] * A[8];
  K[2] = A[3] * A[7] - A[4] * A[6];
  K[3] = A[2] * A[7] - A[1] * A[8];
  K[4] = A[0] * A[8] - A[2] * A[6];
  K[5] = A[1] * A[6] - A[0] * A[7];
  K[6] = A[1] * A[5] - A[2] * A[4];
  K[7] = A[2] * A[3] - A[0] * A[5];
  K[8] = A[0] * A[4] - A[1] * A[3];
}

// global float4 vector reduction (sm_90+)
__device__ inline void red_add_v4(float4* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}

__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace mpm
