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
// One thread per particle for the sums (FP32 products; a warp whose particles
// all belong to one object sums them over the warp, then one FP64 atomic per
// value into one of the object's replica lines), one block per object for the
// solve (its threads sum the replica lines, then one thread solves with the
// library's FP32 3x3 SVD of A scaled to unit norm), FP32 per-particle updates. FP64 arithmetic is kept
// to the atomics and the once-per-object centroid: on this GPU the FP64 pipes
// run at a small fraction of the FP32 rate. The rest shape (computed once per
// sim_set_particles) is summed in FP64.
#include <math.h>

#include "common.cuh"
#include "constitutive.cuh"
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

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline double* acc_line(double* acc, int o, int rep) {
  return acc + ((long long)o * kRigidReplicas + rep) * kRigidLine;
}

// Adds this lane's vals to slots [q0, q0 + NV) of object o's accumulators
// (o < 0: nothing). Every lane of the warp must call it. A warp whose lanes
// all add to one object sums over the warp first (in T) and issues one FP64
// atomic per value; the warp's index picks the replica line.
template <typename T, int NV>
__device__ inline void add_to_object(double* __restrict__ acc, int q0, int o, const T (&vals)[NV]) {
  const int o0 = __shfl_sync(0xffffffffu, o, 0);
  const bool uniform = __all_sync(0xffffffffu, o == o0);
  const int rep = int((blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) & (kRigidReplicas - 1));
  if (uniform) {
    if (o0 < 0) return;
    const bool lead = (threadIdx.x & 31) == 0;
    double* line = acc_line(acc, o0, rep) + q0;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const T s = warp_sum(vals[q]);
      if (lead) atomicAdd(line + q, double(s));
    }
  } else if (o >= 0) {
    double* line = acc_line(acc, o, rep) + q0;
#pragma unroll
    for (int q = 0; q < NV; ++q) atomicAdd(line + q, double(vals[q]));
  }
}

// Block of kRigidReplicas threads per object: thread q < nv sums slot q0 + q
// over the replica lines of object o into out[q] (shared) and clears them.
// Ends with a barrier.
__device__ inline void reduce_object(double* __restrict__ acc, int o, int q0, int nv, double* out) {
  const int q = threadIdx.x;
  if (q < nv) {
    double s = 0.0;
#pragma unroll 8
    for (int rep = 0; rep < kRigidReplicas; ++rep) {
      double* a = acc_line(acc, o, rep) + q0 + q;
      s += *a;
      *a = 0.0;
    }
    out[q] = s;
  }
  __syncthreads();
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
  add_to_object(sums, 0, o, v);
}

// totals of slots 0..3 (M, sum m X) of the objects [o_lo, o_lo + o_cnt), one
// block each, written back to replica line 0
__global__ void rest_center_kernel(Params P, int o_lo, double* __restrict__ sums) {
  __shared__ double t[4];
  const int o = o_lo + blockIdx.x;
  reduce_object(sums, o, 0, 4, t);
  if (threadIdx.x < 4) acc_line(sums, o, 0)[threadIdx.x] = t[threadIdx.x];
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
      const double* S = acc_line(sums, o, 0);
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
  add_to_object(sums, 4, o, v);
}

// constants of the objects [o_lo, o_lo + o_cnt), one block each: M, sbar,
// K = I0^{-1} with I0 = tr(J) 1 - J, J = sum m rbar rbar^T; clears the sums
__global__ void rest_finish_kernel(Params P, int o_lo, double* __restrict__ sums, float* __restrict__ cst) {
  __shared__ double S[16];
  const int o = o_lo + blockIdx.x;
  const int m = o % P.n_mat;
  reduce_object(sums, o, 4, 12, S + 4);
  if (threadIdx.x != 0) return;
  double* l0 = acc_line(sums, o, 0);
  S[0] = l0[0];
  for (int q = 0; q < 4; ++q) l0[q] = 0.0;
  double k[kRigidConst];
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
  for (int q = 0; q < kRigidConst; ++q) cst[(long long)o * kRigidConst + q] = float(k[q]);
}

// ---------------------------------------------------------------------------
// forward projection (FP32 per particle: the FP64 pipes of this GPU are a
// small fraction of its FP32 rate; the per-object sums stay FP64 across warps)
// ---------------------------------------------------------------------------
__device__ inline void cross3f(const float* a, const float* b, float* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

__global__ void __launch_bounds__(256) rigid_sums_kernel(Params P, const float* __restrict__ st,
                                                         const uint32_t* __restrict__ tag,
                                                         const int* __restrict__ pid,
                                                         const float* __restrict__ rest,
                                                         double* __restrict__ sums) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = P.N;
  int o = -1;
  float v[kRigidSums];
#pragma unroll
  for (int q = 0; q < kRigidSums; ++q) v[q] = 0.0f;
  if (p < N) {
    const uint32_t tg = tag[p];
    o = rigid_object(P, tg);
    if (o >= 0) {
      const float m = P.mat[tag_mat(tg)].mass;
      const int c = pid[p];
      float rb[3], x[3], u[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        rb[d] = rest[d * N + c];
        x[d] = st[(fX + d) * N + p];
        u[d] = st[(fV + d) * N + p];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float mx = m * x[i], mu = m * u[i];
        v[i] = mx;
        v[12 + i] = mu;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          v[3 + 3 * i + j] = mx * rb[j];
          v[15 + 3 * i + j] = mu * rb[j];
        }
      }
    }
  }
  add_to_object(sums, 0, o, v);
}

__global__ void rigid_solve_kernel(Params P, double* __restrict__ sums, const float* __restrict__ cst,
                                   float* __restrict__ rec) {
  __shared__ double S[kRigidSums];
  const int o = blockIdx.x;
  reduce_object(sums, o, 0, kRigidSums, S);
  if (threadIdx.x != 0) return;
  const float* k = cst + (long long)o * kRigidConst;
  float* r = rec + (long long)o * kRigidRecord;
  float c[3] = {0.f, 0.f, 0.f}, vb[3] = {0.f, 0.f, 0.f}, w[3] = {0.f, 0.f, 0.f}, L[3] = {0.f, 0.f, 0.f};
  float R[9], U[9], V[9], sg[3] = {1.f, 1.f, 1.f}, S4[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    R[q] = U[q] = V[q] = (q % 4 == 0) ? 1.0f : 0.0f;
    S4[q] = 0.0f;
  }
  const float M = k[0];
  if (P.mat[o % P.n_mat].kind == kRigid && M > 0.0f) {
    // centroid and A = S2 - c sbar^T from the FP64 sums
    double cd[3];
    for (int i = 0; i < 3; ++i) {
      cd[i] = S[i] / double(M);
      c[i] = float(cd[i]);
      vb[i] = float(S[12 + i] / double(M));
    }
    float A[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A[3 * i + j] = float(S[3 + 3 * i + j] - cd[i] * double(k[1 + j]));
    // polar factor R = U V^T from the SVD of A scaled to unit norm (the
    // factor does not depend on the scale; sigma is scaled back)
    float a2 = 0.0f;
    for (int q = 0; q < 9; ++q) a2 += A[q] * A[q];
    if (a2 > 0.0f) {
      const float inv = rsqrtf(a2), sc = a2 * inv;
      float An[9];
      for (int q = 0; q < 9; ++q) An[q] = A[q] * inv;
      svd3(An, U, sg, V);
      for (int i = 0; i < 3; ++i) sg[i] *= sc;
      mat_mult(U, V, R);
    }
    for (int q = 0; q < 9; ++q) S4[q] = float(S[15 + q]);
    // L_i = eps_ijk (R S4^T)_jk
    float Mm[9];
    mat_mult(R, S4, Mm);
    L[0] = Mm[5] - Mm[7];
    L[1] = Mm[6] - Mm[2];
    L[2] = Mm[1] - Mm[3];
    // w = R K R^T L
    const float* K = k + 4;
    float t[3], u[3];
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
}

__global__ void __launch_bounds__(256) rigid_apply_kernel(Params P, float* __restrict__ st,
                                                          const uint32_t* __restrict__ tag,
                                                          const int* __restrict__ pid,
                                                          const float* __restrict__ rest,
                                                          const float* __restrict__ rec) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = P.N;
  if (p >= N) return;
  const int o = rigid_object(P, tag[p]);
  if (o < 0) return;
  const float* r = rec + (long long)o * kRigidRecord;
  const int c = pid[p];
  float rb[3], arm[3];
  for (int d = 0; d < 3; ++d) rb[d] = rest[d * N + c];
  for (int i = 0; i < 3; ++i) arm[i] = r[3 + 3 * i] * rb[0] + r[4 + 3 * i] * rb[1] + r[5 + 3 * i] * rb[2];
  const float* w = r + 15;
  float wr[3];
  cross3f(w, arm, wr);
  for (int d = 0; d < 3; ++d) {
    st[(fX + d) * N + p] = r[d] + arm[d];
    st[(fV + d) * N + p] = r[12 + d] + wr[d];
  }
  const float Cw[9] = {0.0f, -w[2], w[1], w[2], 0.0f, -w[0], -w[1], w[0], 0.0f};
  for (int q = 0; q < 9; ++q) {
    st[(fC + q) * N + p] = Cw[q];
    st[(fF + q) * N + p] = r[3 + q];
  }
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) rigid_adj_sums_kernel(Params P, const float* __restrict__ adj,
                                                             const uint32_t* __restrict__ tag,
                                                             const int* __restrict__ pid,
                                                             const float* __restrict__ rest,
                                                             const float* __restrict__ rec,
                                                             double* __restrict__ gsums) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = P.N;
  int o = -1;
  float v[kRigidGrad];
#pragma unroll
  for (int q = 0; q < kRigidGrad; ++q) v[q] = 0.0f;
  if (p < N) {
    o = rigid_object(P, tag[p]);
    if (o >= 0) {
      const float* r = rec + (long long)o * kRigidRecord;
      const int c = pid[p];
      float rb[3], arm[3], dx[3], dv[3], dC[9];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        rb[d] = rest[d * N + c];
        dx[d] = adj[(fX + d) * N + p];
        dv[d] = adj[(fV + d) * N + p];
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) dC[q] = adj[(fC + q) * N + p];
#pragma unroll
      for (int i = 0; i < 3; ++i) arm[i] = r[3 + 3 * i] * rb[0] + r[4 + 3 * i] * rb[1] + r[5 + 3 * i] * rb[2];
      // v' = vbar + w x arm: arm gets dv x w, w gets arm x dv; C' = [w]_x
      float dvw[3], adv[3];
      cross3f(dv, r + 15, dvw);
      cross3f(arm, dv, adv);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        v[i] = dx[i];
        v[12 + i] = dv[i];
        const float gx = dx[i] + dvw[i];
#pragma unroll
        for (int j = 0; j < 3; ++j) v[3 + 3 * i + j] = gx * rb[j] + adj[(fF + 3 * i + j) * N + p];
      }
      v[15] = adv[0] + dC[7] - dC[5];
      v[16] = adv[1] + dC[2] - dC[6];
      v[17] = adv[2] + dC[3] - dC[1];
    }
  }
  add_to_object(gsums, 0, o, v);
}

__global__ void rigid_adj_solve_kernel(Params P, double* __restrict__ gsums, const float* __restrict__ cst,
                                       const float* __restrict__ rec, float* __restrict__ gout) {
  __shared__ double g[kRigidGrad];
  const int o = blockIdx.x;
  reduce_object(gsums, o, 0, kRigidGrad, g);
  if (threadIdx.x != 0) return;
  const float* k = cst + (long long)o * kRigidConst;
  const float* r = rec + (long long)o * kRigidRecord;
  float* out = gout + (long long)o * kRigidSums;
  float d[kRigidSums];
  for (int q = 0; q < kRigidSums; ++q) d[q] = 0.0f;
  const float M = k[0];
  if (P.mat[o % P.n_mat].kind == kRigid && M > 0.0f) {
    const float *R = r + 3, *L = r + 18, *U = r + 21, *sg = r + 30, *V = r + 33, *S4 = r + 42, *K = k + 4;
    float gw[3], gR[9];
    for (int i = 0; i < 3; ++i) gw[i] = float(g[15 + i]);
    for (int q = 0; q < 9; ++q) gR[q] = float(g[3 + q]);
    // w = R K R^T L: Lbar = R K R^T wbar, Rbar += wbar (K R^T L)^T + L (K R^T wbar)^T
    float t[3], kg[3], kl[3], dL[3];
    for (int i = 0; i < 3; ++i) t[i] = R[i] * gw[0] + R[3 + i] * gw[1] + R[6 + i] * gw[2];
    for (int i = 0; i < 3; ++i) kg[i] = K[3 * i] * t[0] + K[3 * i + 1] * t[1] + K[3 * i + 2] * t[2];
    for (int i = 0; i < 3; ++i) dL[i] = R[3 * i] * kg[0] + R[3 * i + 1] * kg[1] + R[3 * i + 2] * kg[2];
    for (int i = 0; i < 3; ++i) t[i] = R[i] * L[0] + R[3 + i] * L[1] + R[6 + i] * L[2];
    for (int i = 0; i < 3; ++i) kl[i] = K[3 * i] * t[0] + K[3 * i + 1] * t[1] + K[3 * i + 2] * t[2];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) gR[3 * i + j] += gw[i] * kl[j] + L[i] * kg[j];
    // L = eps (R S4^T): (R S4^T)bar = -[Lbar]_x, so Rbar -= [Lbar]_x S4 and
    // S4bar = [Lbar]_x R
    const float X[9] = {0.0f, -dL[2], dL[1], dL[2], 0.0f, -dL[0], -dL[1], dL[0], 0.0f};
    float XS[9], XR[9];
    mat_mul(X, S4, XS);
    mat_mul(X, R, XR);
    for (int q = 0; q < 9; ++q) {
      gR[q] -= XS[q];
      d[15 + q] = XR[q];
    }
    // polar factor R = U V^T of A = U diag(sg) V^T:
    // Abar = U Y V^T, Y_ij = (B_ij - B_ji) / (sg_i + sg_j), B = U^T Rbar V
    float T[9], B[9], Y[9], Z[9], dA[9];
    mat_mul(gR, V, T);
    mat_tmul(U, T, B);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const float den = sg[i] + sg[j];
        Y[3 * i + j] = (i != j && fabsf(den) > 1e-30f) ? (B[3 * i + j] - B[3 * j + i]) / den : 0.0f;
      }
    mat_mul(U, Y, Z);
    mat_mult(Z, V, dA);
    // A = S2 - c sbar^T, c = S1 / M, vbar = S3 / M
    for (int i = 0; i < 3; ++i) {
      const float dc = float(g[i]) - (dA[3 * i] * k[1] + dA[3 * i + 1] * k[2] + dA[3 * i + 2] * k[3]);
      d[i] = dc / M;
      d[12 + i] = float(g[12 + i]) / M;
    }
    for (int q = 0; q < 9; ++q) d[3 + q] = dA[q];
  }
  for (int q = 0; q < kRigidSums; ++q) out[q] = d[q];
}

__global__ void __launch_bounds__(256) rigid_adj_apply_kernel(Params P, float* __restrict__ adj,
                                                              const uint32_t* __restrict__ tag,
                                                              const int* __restrict__ pid,
                                                              const float* __restrict__ rest,
                                                              const float* __restrict__ gout) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = P.N;
  if (p >= N) return;
  const uint32_t tg = tag[p];
  const int o = rigid_object(P, tg);
  if (o < 0) return;
  const float m = P.mat[tag_mat(tg)].mass;
  const float* d = gout + (long long)o * kRigidSums;
  const int c = pid[p];
  float rb[3];
  for (int j = 0; j < 3; ++j) rb[j] = rest[j * N + c];
  for (int i = 0; i < 3; ++i) {
    adj[(fX + i) * N + p] = m * (d[i] + d[3 + 3 * i] * rb[0] + d[4 + 3 * i] * rb[1] + d[5 + 3 * i] * rb[2]);
    adj[(fV + i) * N + p] = m * (d[12 + i] + d[15 + 3 * i] * rb[0] + d[16 + 3 * i] * rb[1] + d[17 + 3 * i] * rb[2]);
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
  // scene < 0: every scene's objects
  const int o_lo = scene < 0 ? 0 : scene * P.n_mat;
  const int o_cnt = scene < 0 ? rb.n_obj : P.n_mat;
  rest_mass_kernel<<<blocks_for(cnt, 256), 256, 0, s>>>(P, X0, tag0, lo, cnt, rb.sums);
  rest_center_kernel<<<o_cnt, kRigidReplicas, 0, s>>>(P, o_lo, rb.sums);
  rest_offsets_kernel<<<blocks_for(cnt, 256), 256, 0, s>>>(P, X0, tag0, lo, cnt, rb.sums, rb.rest);
  rest_finish_kernel<<<o_cnt, kRigidReplicas, 0, s>>>(P, o_lo, rb.sums, rb.cst);
}

void launch_rigid_project(const Params& P, float* st, const uint32_t* tag, const int* pid, RigidBuffers rb,
                          float* rec, cudaStream_t s) {
  if (P.N == 0) return;
  rigid_sums_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, st, tag, pid, rb.rest, rb.sums);
  rigid_solve_kernel<<<rb.n_obj, kRigidReplicas, 0, s>>>(P, rb.sums, rb.cst, rec);
  rigid_apply_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, st, tag, pid, rb.rest, rec);
}

void launch_rigid_adjoint(const Params& P, float* adj, const uint32_t* tag, const int* pid, RigidBuffers rb,
                          const float* rec, cudaStream_t s) {
  if (P.N == 0) return;
  rigid_adj_sums_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, adj, tag, pid, rb.rest, rec, rb.gsums);
  rigid_adj_solve_kernel<<<rb.n_obj, kRigidReplicas, 0, s>>>(P, rb.gsums, rb.cst, rec, rb.gout);
  rigid_adj_apply_kernel<<<blocks_for(P.N, 256), 256, 0, s>>>(P, adj, tag, pid, rb.rest, rb.gout);
}

}  // namespace mpm
