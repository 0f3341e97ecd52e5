// Particle-represented rigid bodies (paper Sec. 3.2 "Rigid body": the
// object's particles are simulated as an elastic material by MLS-MPM, then an
// object-level transformation is fitted and rigidity enforced). The paper
// gives no formulas; this library's reading, per object after each G2P:
//   c = S1 / M,  A = S2 - c sbar^T,  R = polar factor of A (via its SVD),
//   vbar = S3 / M,  L = sum m (R rbar) x v  (from R S4^T),  w = R K R^T L,
//   x' = c + R rbar,  v' = vbar + w x (R rbar),  C' = [w]_x,  F' = R,
// i.e. the mass-weighted least-squares rigid fit of the positions (shape
// matching, Mueller et al. 2005) and of the velocities (keeping the linear
// momentum and the angular momentum about c). With F a rotation the
// corotated stress vanishes, so a rigid particle's P2G prologue is tau = 0,
// F_p = F. The adjoint pulls the per-particle adjoints back through the
// per-object chain to the adjoints of the four sums, then to x and v (the
// projection's outputs do not depend on C or F).
//
// One thread per particle for the sums (a warp whose particles all belong to
// one object sums in registers first, then one FP64 atomic per value), one
// thread per object for the FP64 solve. Objects are few and small next to the
// MPM kernels, so these kernels are plain and latency-bound.
#include <math.h>

#include "common.cuh"
#include "rigid.h"

namespace mpm {

namespace {

constexpr int fX = 0, fV = 3, fC = 6, fF = 15;
inline int blocks_for(long long n, int t) { return int((n + t - 1) / t); }

__device__ inline int rigid_object(const Params& P, uint32_t tg) {
  const int mat = tag_mat(tg);
  if (mat >= P.n_mat || P.mat[mat].kind != kRigid) return -1;
  return tag_scene(tg) * P.n_mat + mat;
}

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Adds this lane's vals to base[o * stride + q] (o < 0: nothing). Every lane
// of the warp must call it; a warp whose lanes all add to one object sums
// first and issues one atomic per value.
template <int NV>
__device__ inline void add_to_object(double* __restrict__ base, int stride, int o, const double (&vals)[NV]) {
  const int o0 = __shfl_sync(0xffffffffu, o, 0);
  const bool uniform = __all_sync(0xffffffffu, o == o0);
  if (uniform) {
    if (o0 < 0) return;
    const bool lead = (threadIdx.x & 31) == 0;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const double s = warp_sum_d(vals[q]);
      if (lead) atomicAdd(base + (long long)o0 * stride + q, s);
    }
  } else if (o >= 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) atomicAdd(base + (long long)o * stride + q, vals[q]);
  }
}

__device__ inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// SVD A = U diag(sg) V^T of a 3x3 (row-major) by one-sided Jacobi rotations
// of A's columns (Hestenes' method), in FP64; U and V are rotations and
// sg[0] >= sg[1] >= |sg[2]| (sg[2] < 0 when det A < 0). Returns false when A
// has rank < 2 (U, sg, V undefined).
__device__ bool svd3_jacobi(const double* A, double* U, double* sg, double* V) {
  double B[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    B[k] = A[k];
    V[k] = (k % 4 == 0) ? 1.0 : 0.0;
  }
  for (int sweep = 0; sweep < 32; ++sweep) {
    bool rotated = false;
    for (int pair = 0; pair < 3; ++pair) {
      const int i = pair == 2 ? 1 : 0, j = pair == 0 ? 1 : 2;
      double a = 0.0, b = 0.0, g = 0.0;
      for (int r = 0; r < 3; ++r) {
        a += B[3 * r + i] * B[3 * r + i];
        b += B[3 * r + j] * B[3 * r + j];
        g += B[3 * r + i] * B[3 * r + j];
      }
      if (!(fabs(g) > 1e-15 * sqrt(a * b))) continue;
      rotated = true;
      // rotation zeroing the inner product of columns i and j
      const double z = (b - a) / (2.0 * g);
      const double t = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
      const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
      for (int r = 0; r < 3; ++r) {
        const double bi = B[3 * r + i], bj = B[3 * r + j];
        B[3 * r + i] = cs * bi - sn * bj;
        B[3 * r + j] = sn * bi + cs * bj;
        const double vi = V[3 * r + i], vj = V[3 * r + j];
        V[3 * r + i] = cs * vi - sn * vj;
        V[3 * r + j] = sn * vi + cs * vj;
      }
    }
    if (!rotated) break;
  }
  double nrm[3];
  for (int k = 0; k < 3; ++k)
    nrm[k] = sqrt(B[k] * B[k] + B[3 + k] * B[3 + k] + B[6 + k] * B[6 + k]);
  // columns by decreasing norm; a swap negates one column of B and V so that
  // A V = B still holds and det V stays +1
  const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int q = 0; q < 3; ++q) {
    const int i = pairs[q][0], j = pairs[q][1];
    if (nrm[j] > nrm[i]) {
      for (int r = 0; r < 3; ++r) {
        double t = B[3 * r + i];
        B[3 * r + i] = B[3 * r + j];
        B[3 * r + j] = -t;
        t = V[3 * r + i];
        V[3 * r + i] = V[3 * r + j];
        V[3 * r + j] = -t;
      }
      const double t = nrm[i];
      nrm[i] = nrm[j];
      nrm[j] = t;
    }
  }
  if (!(nrm[0] > 0.0) || !(nrm[1] > 1e-12 * nrm[0])) return false;
  double u0[3], u1[3], u2[3];
  for (int r = 0; r < 3; ++r) {
    u0[r] = B[3 * r] / nrm[0];
    u1[r] = B[3 * r + 1] / nrm[1];
  }
  cross3(u0, u1, u2);
  sg[0] = nrm[0];
  sg[1] = nrm[1];
  sg[2] = u2[0] * B[2] + u2[1] * B[5] + u2[2] * B[8];
  for (int r = 0; r < 3; ++r) {
    U[3 * r] = u0[r];
    U[3 * r + 1] = u1[r];
    U[3 * r + 2] = u2[r];
  }
  return true;
}

// ---------------------------------------------------------------------------
// rest shape
// ---------------------------------------------------------------------------
// sums[o][0] = M, sums[o][1..3] = sum m X
__global__ void rest_mass_kernel(Params P, const float* __restrict__ X0, const uint32_t* __restrict__ tag0, int lo,
                                 int cnt, double* __restrict__ sums) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = P.N;
  int o = -1;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (i < cnt) {
    const int p = lo + i;
    const uint32_t tg = tag0[p];
    o = rigid_object(P, tg);
    if (o >= 0) {
      const double m = P.mat[tag_mat(tg)].mass;
      v[0] = m;
      for (int d = 0; d < 3; ++d) v[1 + d] = m * double(X0[(fX + d) * N + p]);
    }
  }
  add_to_object(sums, kRigidSums, o, v);
}

// rest offsets rbar = X - X_c (stored as floats); sums[o][4..6] = sum m rbar,
// sums[o][7..15] = sum m rbar rbar^T of the stored offsets
__global__ void rest_offsets_kernel(Params P, const float* __restrict__ X0, const uint32_t* __restrict__ tag0,
                                    int lo, int cnt, double* __restrict__ sums, float* __restrict__ rest) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = P.N;
  int o = -1;
  double v[12];
  for (int q = 0; q < 12; ++q) v[q] = 0.0;
  if (i < cnt) {
    const int p = lo + i;
    const uint32_t tg = tag0[p];
    o = rigid_object(P, tg);
    if (o >= 0) {
      const double m = P.mat[tag_mat(tg)].mass;
      const double* S = sums + (long long)o * kRigidSums;
      double r[3];
      for (int d = 0; d < 3; ++d) {
        const float rf = float(double(X0[(fX + d) * N + p]) - S[1 + d] / S[0]);
        rest[d * N + p] = rf;
        r[d] = rf;
      }
      for (int d = 0; d < 3; ++d) v[d] = m * r[d];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) v[3 + 3 * a + b] = m * r[a] * r[b];
    }
  }
  double* base = sums + 4;
  add_to_object(base, kRigidSums, o, v);
}

// constants of the objects [o_lo, o_lo + o_cnt): M, sbar, K = I0^{-1} with
// I0 = tr(J) 1 - J, J = sum m rbar rbar^T; clears the sums
__global__ void rest_finish_kernel(Params P, int o_lo, int o_cnt, double* __restrict__ sums,
                                   double* __restrict__ cst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= o_cnt) return;
  const int o = o_lo + i;
  const int m = o % P.n_mat;
  double* S = sums + (long long)o * kRigidSums;
  double* k = cst + (long long)o * kRigidConst;
  for (int q = 0; q < kRigidConst; ++q) k[q] = 0.0;
  if (P.mat[m].kind == kRigid && S[0] > 0.0) {
    k[0] = S[0];
    for (int d = 0; d < 3; ++d) k[1 + d] = S[4 + d];
    const double* J = S + 7;
    const double tr = J[0] + J[4] + J[8];
    double I[9];
    for (int q = 0; q < 9; ++q) I[q] = ((q % 4 == 0) ? tr : 0.0) - J[q];
    const double c0 = I[4] * I[8] - I[5] * I[7], c1 = I[5] * I[6] - I[3] * I[8], c2 = I[3] * I[7] - I[4] * I[6];
    const double det = I[0] * c0 + I[1] * c1 + I[2] * c2;
    const double s = tr / 3.0;
    if (det > 1e-12 * s * s * s) {
      // adjugate / det (I0 is symmetric)
      double* K = k + 4;
      K[0] = c0 / det;
      K[3] = c1 / det;
      K[6] = c2 / det;
      K[1] = (I[2] * I[7] - I[1] * I[8]) / det;
      K[4] = (I[0] * I[8] - I[2] * I[6]) / det;
      K[7] = (I[1] * I[6] - I[0] * I[7]) / det;
      K[2] = (I[1] * I[5] - I[2] * I[4]) / det;
      K[5] = (I[2] * I[3] - I[0] * I[5]) / det;
      K[8] = (I[0] * I[4] - I[1] * I[3]) / det;
    }
  }
  for (int q = 0; q < kRigidSums; ++q) S[q] = 0.0;
}

// ---------------------------------------------------------------------------
// forward projection
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) rigid_sums_kernel(Params P, const float* __restrict__ st,
                                                         const uint32_t* __restrict__ tag,
                                                         const int* __restrict__ pid,
                                                         const float* __restrict__ rest,
                                                         double* __restrict__ sums) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = P.N;
  int o = -1;
  double v[kRigidSums];
#pragma unroll
  for (int q = 0; q < kRigidSums; ++q) v[q] = 0.0;
  if (p < N) {
    const uint32_t tg = tag[p];
    o = rigid_object(P, tg);
    if (o >= 0) {
      const double m = P.mat[tag_mat(tg)].mass;
      const int c = pid[p];
      double rb[3], x[3], u[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        rb[d] = rest[d * N + c];
        x[d] = st[(fX + d) * N + p];
        u[d] = st[(fV + d) * N + p];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        v[i] = m * x[i];
        v[12 + i] = m * u[i];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          v[3 + 3 * i + j] = m * x[i] * rb[j];
          v[15 + 3 * i + j] = m * u[i] * rb[j];
        }
      }
    }
  }
  add_to_object(sums, kRigidSums, o, v);
}

__global__ void rigid_solve_kernel(Params P, double* __restrict__ sums, const double* __restrict__ cst,
                                   double* __restrict__ rec) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= P.S * P.n_mat) return;
  double* S = sums + (long long)o * kRigidSums;
  const double* k = cst + (long long)o * kRigidConst;
  double* r = rec + (long long)o * kRigidRecord;
  double c[3] = {0.0, 0.0, 0.0}, vb[3] = {0.0, 0.0, 0.0}, w[3] = {0.0, 0.0, 0.0}, L[3] = {0.0, 0.0, 0.0};
  double R[9], U[9], V[9], sg[3] = {1.0, 1.0, 1.0}, S4[9];
  for (int q = 0; q < 9; ++q) {
    R[q] = U[q] = V[q] = (q % 4 == 0) ? 1.0 : 0.0;
    S4[q] = 0.0;
  }
  const double M = k[0];
  if (P.mat[o % P.n_mat].kind == kRigid && M > 0.0) {
    double A[9];
    for (int i = 0; i < 3; ++i) {
      c[i] = S[i] / M;
      vb[i] = S[12 + i] / M;
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A[3 * i + j] = S[3 + 3 * i + j] - c[i] * k[1 + j];
    if (svd3_jacobi(A, U, sg, V)) {
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[3 * i + j] = U[3 * i] * V[3 * j] + U[3 * i + 1] * V[3 * j + 1] + U[3 * i + 2] * V[3 * j + 2];
    } else {
      for (int q = 0; q < 9; ++q) U[q] = V[q] = (q % 4 == 0) ? 1.0 : 0.0;
      sg[0] = sg[1] = sg[2] = 1.0;
    }
    for (int q = 0; q < 9; ++q) S4[q] = S[15 + q];
    // L_i = eps_ijk (R S4^T)_jk
    double Mm[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Mm[3 * i + j] = R[3 * i] * S4[3 * j] + R[3 * i + 1] * S4[3 * j + 1] + R[3 * i + 2] * S4[3 * j + 2];
    L[0] = Mm[5] - Mm[7];
    L[1] = Mm[6] - Mm[2];
    L[2] = Mm[1] - Mm[3];
    // w = R K R^T L
    const double* K = k + 4;
    double t[3], u[3];
    for (int i = 0; i < 3; ++i) t[i] = R[i] * L[0] + R[3 + i] * L[1] + R[6 + i] * L[2];
    for (int i = 0; i < 3; ++i) u[i] = K[3 * i] * t[0] + K[3 * i + 1] * t[1] + K[3 * i + 2] * t[2];
    for (int i = 0; i < 3; ++i) w[i] = R[3 * i] * u[0] + R[3 * i + 1] * u[1] + R[3 * i + 2] * u[2];
  }
  for (int i = 0; i < 3; ++i) {
    r[i] = c[i];
    r[12 + i] = vb[i];
    r[15 + i] = w[i];
    r[18 + i] = L[i];
    r[30 + i] = sg[i];
  }
  for (int q = 0; q < 9; ++q) {
    r[3 + q] = R[q];
    r[21 + q] = U[q];
    r[33 + q] = V[q];
    r[42 + q] = S4[q];
  }
  for (int q = 0; q < kRigidSums; ++q) S[q] = 0.0;
}

__global__ void __launch_bounds__(256) rigid_apply_kernel(Params P, float* __restrict__ st,
                                                          const uint32_t* __restrict__ tag,
                                                          const int* __restrict__ pid,
                                                          const float* __restrict__ rest,
                                                          const double* __restrict__ rec) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = P.N;
  if (p >= N) return;
  const int o = rigid_object(P, tag[p]);
  if (o < 0) return;
  const double* r = rec + (long long)o * kRigidRecord;
  const int c = pid[p];
  double rb[3], arm[3];
  for (int d = 0; d < 3; ++d) rb[d] = rest[d * N + c];
  for (int i = 0; i < 3; ++i) arm[i] = r[3 + 3 * i] * rb[0] + r[4 + 3 * i] * rb[1] + r[5 + 3 * i] * rb[2];
  const double* w = r + 15;
  double wr[3];
  cross3(w, arm, wr);
  for (int d = 0; d < 3; ++d) {
    st[(fX + d) * N + p] = float(r[d] + arm[d]);
    st[(fV + d) * N + p] = float(r[12 + d] + wr[d]);
  }
  const float Cw[9] = {0.0f, float(-w[2]), float(w[1]), float(w[2]), 0.0f, float(-w[0]),
                       float(-w[1]), float(w[0]), 0.0f};
  for (int q = 0; q < 9; ++q) {
    st[(fC + q) * N + p] = Cw[q];
    st[(fF + q) * N + p] = float(r[3 + q]);
  }
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) rigid_adj_sums_kernel(Params P, const float* __restrict__ adj,
                                                             const uint32_t* __restrict__ tag,
                                                             const int* __restrict__ pid,
                                                             const float* __restrict__ rest,
                                                             const double* __restrict__ rec,
                                                             double* __restrict__ gsums) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = P.N;
  int o = -1;
  double v[kRigidGrad];
#pragma unroll
  for (int q = 0; q < kRigidGrad; ++q) v[q] = 0.0;
  if (p < N) {
    o = rigid_object(P, tag[p]);
    if (o >= 0) {
      const double* r = rec + (long long)o * kRigidRecord;
      const int c = pid[p];
      double rb[3], arm[3], dx[3], dv[3], dC[9];
      for (int d = 0; d < 3; ++d) {
        rb[d] = rest[d * N + c];
        dx[d] = adj[(fX + d) * N + p];
        dv[d] = adj[(fV + d) * N + p];
      }
      for (int q = 0; q < 9; ++q) dC[q] = adj[(fC + q) * N + p];
      for (int i = 0; i < 3; ++i) arm[i] = r[3 + 3 * i] * rb[0] + r[4 + 3 * i] * rb[1] + r[5 + 3 * i] * rb[2];
      // v' = vbar + w x arm: arm gets dv x w, w gets arm x dv; C' = [w]_x
      double dvw[3], adv[3];
      cross3(dv, r + 15, dvw);
      cross3(arm, dv, adv);
      for (int i = 0; i < 3; ++i) {
        v[i] = dx[i];
        v[12 + i] = dv[i];
        const double gx = dx[i] + dvw[i];
        for (int j = 0; j < 3; ++j) v[3 + 3 * i + j] = gx * rb[j] + double(adj[(fF + 3 * i + j) * N + p]);
      }
      v[15] = adv[0] + dC[7] - dC[5];
      v[16] = adv[1] + dC[2] - dC[6];
      v[17] = adv[2] + dC[3] - dC[1];
    }
  }
  add_to_object(gsums, kRigidGrad, o, v);
}

__global__ void rigid_adj_solve_kernel(Params P, double* __restrict__ gsums, const double* __restrict__ cst,
                                       const double* __restrict__ rec, double* __restrict__ gout) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= P.S * P.n_mat) return;
  double* g = gsums + (long long)o * kRigidGrad;
  const double* k = cst + (long long)o * kRigidConst;
  const double* r = rec + (long long)o * kRigidRecord;
  double* out = gout + (long long)o * kRigidSums;
  double d[kRigidSums];
  for (int q = 0; q < kRigidSums; ++q) d[q] = 0.0;
  const double M = k[0];
  if (P.mat[o % P.n_mat].kind == kRigid && M > 0.0) {
    const double *R = r + 3, *L = r + 18, *U = r + 21, *sg = r + 30, *V = r + 33, *S4 = r + 42, *K = k + 4;
    const double* gw = g + 15;
    double gR[9];
    for (int q = 0; q < 9; ++q) gR[q] = g[3 + q];
    // w = R K R^T L: Lbar = R K R^T wbar, Rbar += wbar (K R^T L)^T + L (K R^T wbar)^T
    double t[3], kg[3], kl[3], dL[3];
    for (int i = 0; i < 3; ++i) t[i] = R[i] * gw[0] + R[3 + i] * gw[1] + R[6 + i] * gw[2];
    for (int i = 0; i < 3; ++i) kg[i] = K[3 * i] * t[0] + K[3 * i + 1] * t[1] + K[3 * i + 2] * t[2];
    for (int i = 0; i < 3; ++i) dL[i] = R[3 * i] * kg[0] + R[3 * i + 1] * kg[1] + R[3 * i + 2] * kg[2];
    for (int i = 0; i < 3; ++i) t[i] = R[i] * L[0] + R[3 + i] * L[1] + R[6 + i] * L[2];
    for (int i = 0; i < 3; ++i) kl[i] = K[3 * i] * t[0] + K[3 * i + 1] * t[1] + K[3 * i + 2] * t[2];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) gR[3 * i + j] += gw[i] * kl[j] + L[i] * kg[j];
    // L = eps (R S4^T): (R S4^T)bar = -[Lbar]_x, so Rbar -= [Lbar]_x S4 and
    // S4bar = [Lbar]_x R
    const double X[9] = {0.0, -dL[2], dL[1], dL[2], 0.0, -dL[0], -dL[1], dL[0], 0.0};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        gR[3 * i + j] -= X[3 * i] * S4[j] + X[3 * i + 1] * S4[3 + j] + X[3 * i + 2] * S4[6 + j];
        d[15 + 3 * i + j] = X[3 * i] * R[j] + X[3 * i + 1] * R[3 + j] + X[3 * i + 2] * R[6 + j];
      }
    // polar factor R = U V^T of A = U diag(sg) V^T:
    // Abar = U Y V^T, Y_ij = (B_ij - B_ji) / (sg_i + sg_j), B = U^T Rbar V
    double T[9], B[9], Y[9], Z[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) T[3 * i + j] = gR[3 * i] * V[j] + gR[3 * i + 1] * V[3 + j] + gR[3 * i + 2] * V[6 + j];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) B[3 * i + j] = U[i] * T[j] + U[3 + i] * T[3 + j] + U[6 + i] * T[6 + j];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const double den = sg[i] + sg[j];
        Y[3 * i + j] = (i != j && fabs(den) > 1e-300) ? (B[3 * i + j] - B[3 * j + i]) / den : 0.0;
      }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Z[3 * i + j] = U[3 * i] * Y[j] + U[3 * i + 1] * Y[3 + j] + U[3 * i + 2] * Y[6 + j];
    double dA[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) dA[3 * i + j] = Z[3 * i] * V[3 * j] + Z[3 * i + 1] * V[3 * j + 1] + Z[3 * i + 2] * V[3 * j + 2];
    // A = S2 - c sbar^T, c = S1 / M, vbar = S3 / M
    for (int i = 0; i < 3; ++i) {
      const double dc = g[i] - (dA[3 * i] * k[1] + dA[3 * i + 1] * k[2] + dA[3 * i + 2] * k[3]);
      d[i] = dc / M;
      d[12 + i] = g[12 + i] / M;
    }
    for (int q = 0; q < 9; ++q) d[3 + q] = dA[q];
  }
  for (int q = 0; q < kRigidSums; ++q) out[q] = d[q];
  for (int q = 0; q < kRigidGrad; ++q) g[q] = 0.0;
}

__global__ void __launch_bounds__(256) rigid_adj_apply_kernel(Params P, float* __restrict__ adj,
                                                              const uint32_t* __restrict__ tag,
                                                              const int* __restrict__ pid,
                                                              const float* __restrict__ rest,
                                                              const double* __restrict__ gout) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = P.N;
  if (p >= N) return;
  const uint32_t tg = tag[p];
  const int o = rigid_object(P, tg);
  if (o < 0) return;
  const double m = P.mat[tag_mat(tg)].mass;
  const double* d = gout + (long long)o * kRigidSums;
  const int c = pid[p];
  double rb[3];
  for (int j = 0; j < 3; ++j) rb[j] = rest[j * N + c];
  for (int i = 0; i < 3; ++i) {
    adj[(fX + i) * N + p] = float(m * (d[i] + d[3 + 3 * i] * rb[0] + d[4 + 3 * i] * rb[1] + d[5 + 3 * i] * rb[2]));
    adj[(fV + i) * N + p] =
        float(m * (d[12 + i] + d[15 + 3 * i] * rb[0] + d[16 + 3 * i] * rb[1] + d[17 + 3 * i] * rb[2]));
  }
  for (int q = 0; q < 9; ++q) {
    adj[(fC + q) * N + p] = 0.0f;
    adj[(fF + q) * N + p] = 0.0f;
  }
}

}  // namespace

void launch_rigid_rest(const Params& P, const float* X0, const uint32_t* tag0, int scene, int lo, int cnt,
                       RigidBuffers rb, cudaStream_t s) {
  if (cnt <= 0) return;
  rest_mass_kernel<<<blocks_for(cnt, 256), 256, 0, s>>>(P, X0, tag0, lo, cnt, rb.sums);
  rest_offsets_kernel<<<blocks_for(cnt, 256), 256, 0, s>>>(P, X0, tag0, lo, cnt, rb.sums, rb.rest);
  // scene < 0: every scene's objects
  const int o_lo = scene < 0 ? 0 : scene * P.n_mat;
  const int o_cnt = scene < 0 ? rb.n_obj : P.n_mat;
  rest_finish_kernel<<<blocks_for(o_cnt, 64), 64, 0, s>>>(P, o_lo, o_cnt, rb.sums, rb.cst);
}

void launch_rigid_project(const Params& P, float* st, const uint32_t* tag, const int* pid, RigidBuffers rb,
                          double* rec, cudaStream_t s) {
  if (P.N == 0) return;
  rigid_sums_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, st, tag, pid, rb.rest, rb.sums);
  rigid_solve_kernel<<<blocks_for(rb.n_obj, 64), 64, 0, s>>>(P, rb.sums, rb.cst, rec);
  rigid_apply_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, st, tag, pid, rb.rest, rec);
}

void launch_rigid_adjoint(const Params& P, float* adj, const uint32_t* tag, const int* pid, RigidBuffers rb,
                          const double* rec, cudaStream_t s) {
  if (P.N == 0) return;
  rigid_adj_sums_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, adj, tag, pid, rb.rest, rec, rb.gsums);
  rigid_adj_solve_kernel<<<blocks_for(rb.n_obj, 64), 64, 0, s>>>(P, rb.gsums, rb.cst, rec, rb.gout);
  rigid_adj_apply_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, adj, tag, pid, rb.rest, rb.gout);
}

}  // namespace mpm
