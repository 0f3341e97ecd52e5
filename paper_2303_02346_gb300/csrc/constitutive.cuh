// Constitutive models, return mappings and their adjoints (device code).
//
// Paper Sec. 3.2: corotated stress for solids and liquids, liquid deformation
// gradient reset every step, von Mises plasticity for the elastoplastic
// material; granular sand follows the Drucker-Prager projection of Klar et
// al. 2016 in Hencky strain. Sec. 3.3 / App. A: the SVD gradient is written by
// hand. Here it is the spectral form of the derivative of an isotropic matrix
// function, F = U diag(sigma) V^T:
//   F_p = U diag(s(sigma)) V^T  ->  Z_ii = sum_k M_kk ds_k/dsig_i,
//       Z_ij = a_ij M_ij + b_ij M_ji, a/b = (D^s_ij +/- (s_i+s_j)/(sig_i+sig_j)) / 2,
//   tau = U diag(t(sigma)) U^T ->  Z_ii = sum_k N_kk dt_k/dsig_i,
//       Z_ij = D^t_ij sig_j (N_ij + N_ji) / (sig_i + sig_j),
// with M = U^T Fbar_p V, N = U^T taubar U, Fbar = U Z V^T and D the divided
// differences (g_i - g_j)/(sig_i - sig_j). Every divided difference is
// evaluated in a factorised form (expm1, log1p) that stays accurate in FP32
// when singular values coincide (F = I at rest), so no denominator clamping
// changes the result there.
#pragma once

#include "common.cuh"

namespace mpm {

constexpr float kSigmaFloor = 1e-4f;
enum : int { kElastic = 0, kProject = 1, kApex = 2 };

// ---------------------------------------------------------------------------
// 3x3 SVD: cyclic Jacobi on F^T F (Golub & Van Loan, symmetric Schur
// rotations), columns sorted by decreasing singular value, then Givens QR of
// F V so that U and V are rotations and sigma_3 carries the sign of det F.
// ---------------------------------------------------------------------------
// Rotation in the (p, q) plane that annihilates A[p][q] (r = the third
// index); V accumulates it. With d = a_qq - a_pp and e = 2 a_pq the tangent of
// the angle is t = sgn(d) e / (|d| + sqrt(d^2 + e^2)) (the smaller root of
// t^2 + 2 t d / e - 1 = 0). c = 1 / sqrt(1 + t^2) and s = t c keep the rotation
// orthogonal to rounding whatever the accuracy of t, so t uses the fast
// reciprocal; a_pq = 0 gives t = 0, the identity.
__device__ inline void jacobi_rotate(float* A, float* V, int p, int q, int r) {
  const float apq = A[3 * p + q];
  const float app = A[3 * p + p], aqq = A[3 * q + q];
  const float d = aqq - app, e = 2.0f * apq;
  const float h2 = fmaf(d, d, e * e);
  const float h = h2 * rsqrtf(fmaxf(h2, 1e-37f));
  const float t = __fdividef(copysignf(1.0f, d) * e, fmaxf(fabsf(d) + h, 1e-30f));
  const float c = rsqrtf(fmaf(t, t, 1.0f));
  const float s = t * c;
  A[3 * p + p] = app - t * apq;
  A[3 * q + q] = aqq + t * apq;
  A[3 * p + q] = A[3 * q + p] = 0.0f;
  const float arp = A[3 * r + p], arq = A[3 * r + q];
  A[3 * r + p] = A[3 * p + r] = c * arp - s * arq;
  A[3 * r + q] = A[3 * q + r] = s * arp + c * arq;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float vp = V[3 * i + p], vq = V[3 * i + q];
    V[3 * i + p] = c * vp - s * vq;
    V[3 * i + q] = s * vp + c * vq;
  }
}

__device__ inline void swap_cols_neg(float* V, float* lam, int a, int b) {
  float t = lam[a];
  lam[a] = lam[b];
  lam[b] = t;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float va = V[3 * i + a];
    V[3 * i + a] = V[3 * i + b];
    V[3 * i + b] = -va;  // keep det V = +1
  }
}

// rows i, j of B rotated to zero B[j][col]; U accumulates the transposed rotation
__device__ inline void givens_qr(float* B, float* U, int i, int j, int col) {
  float a = B[3 * i + col], b = B[3 * j + col];
  float r2 = a * a + b * b;
  if (r2 < 1e-38f) return;
  float rinv = rsqrtf(r2);
  float c = a * rinv, s = b * rinv;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float bi = B[3 * i + k], bj = B[3 * j + k];
    B[3 * i + k] = c * bi + s * bj;
    B[3 * j + k] = -s * bi + c * bj;
    float ui = U[3 * k + i], uj = U[3 * k + j];
    U[3 * k + i] = c * ui + s * uj;
    U[3 * k + j] = -s * ui + c * uj;
  }
}

__device__ inline void svd3(const float* F, float* U, float* sig, float* V) {
  float A[9];
  mat_tmul(F, F, A);
#pragma unroll
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0f : 0.0f;
  float scale = A[0] + A[4] + A[8] + 1e-30f;
#pragma unroll 1
  for (int sweep = 0; sweep < 6; ++sweep) {
    // stop once the off-diagonal part is at FP32 rounding level of the trace
    float off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    if (off <= 1e-14f * scale * scale) break;
    jacobi_rotate(A, V, 0, 1, 2);
    jacobi_rotate(A, V, 0, 2, 1);
    jacobi_rotate(A, V, 1, 2, 0);
  }
  float lam[3] = {A[0], A[4], A[8]};
  if (lam[0] < lam[1]) swap_cols_neg(V, lam, 0, 1);
  if (lam[0] < lam[2]) swap_cols_neg(V, lam, 0, 2);
  if (lam[1] < lam[2]) swap_cols_neg(V, lam, 1, 2);
  float B[9];
  mat_mul(F, V, B);
#pragma unroll
  for (int i = 0; i < 9; ++i) U[i] = (i % 4 == 0) ? 1.0f : 0.0f;
  givens_qr(B, U, 0, 1, 0);
  givens_qr(B, U, 0, 2, 0);
  givens_qr(B, U, 1, 2, 1);
  sig[0] = B[0];
  sig[1] = B[4];
  sig[2] = B[8];
}

// U diag(d) W^T
__device__ inline void udwt(const float* U, const float* d, const float* W, float* out) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      out[3 * r + c] = U[3 * r] * d[0] * W[3 * c] + U[3 * r + 1] * d[1] * W[3 * c + 1] +
                       U[3 * r + 2] * d[2] * W[3 * c + 2];
}

// ---------------------------------------------------------------------------
// singular-value maps: sigma -> projected singular values s, stress
// eigenvalues t, branch
// ---------------------------------------------------------------------------
__device__ inline float hencky(float s) { return logf(fmaxf(s, kSigmaFloor)); }

struct SigmaMap {
  float s[3], t[3], ep[3];
  float eps[3];
  float uhat[3];
  float nrm, tr;
  int branch;
};

// kExt: compiled with the box-yield and viscous-liquid branches; kernels of a
// handle without those materials are built with kExt = false.
template <bool kExt = true>
__device__ inline void sigma_map(const MatParams& M, const float* sg, SigmaMap& o) {
  if (kExt && M.kind == kViscousLiquid) {
    // no projection (the liquid's reset happens outside): fixed-corotated stress
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      o.s[i] = sg[i];
      o.eps[i] = o.ep[i] = o.uhat[i] = 0.0f;
    }
    o.nrm = o.tr = 0.0f;
    o.branch = kElastic;
    const float J = sg[0] * sg[1] * sg[2];
    const float pj = M.lam * J * (J - 1.0f);
#pragma unroll
    for (int i = 0; i < 3; ++i) o.t[i] = 2.0f * M.mu * (sg[i] - 1.0f) * sg[i] + pj;
    return;
  }
  if (kExt && M.kind == kBoxYield) {
    // box criterion: singular values clamped to [1 - theta_c, 1 + theta_s],
    // fixed-corotated stress of the clamped values
    const float lo = 1.0f - M.k_yield, hi = 1.0f + M.c_dp;
    bool clamped = false;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      o.s[i] = fminf(fmaxf(sg[i], lo), hi);
      clamped = clamped || o.s[i] != sg[i];
      o.eps[i] = o.ep[i] = o.uhat[i] = 0.0f;
    }
    o.nrm = o.tr = 0.0f;
    o.branch = clamped ? kProject : kElastic;
    const float J = o.s[0] * o.s[1] * o.s[2];
    const float pj = M.lam * J * (J - 1.0f);
#pragma unroll
    for (int i = 0; i < 3; ++i) o.t[i] = 2.0f * M.mu * (o.s[i] - 1.0f) * o.s[i] + pj;
    return;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) o.eps[i] = hencky(sg[i]);
  float tr = o.eps[0] + o.eps[1] + o.eps[2];
  float mean = tr * (1.0f / 3.0f);
  float eh[3] = {o.eps[0] - mean, o.eps[1] - mean, o.eps[2] - mean};
  float nrm = sqrtf(eh[0] * eh[0] + eh[1] * eh[1] + eh[2] * eh[2]);
  o.nrm = nrm;
  o.tr = tr;
  float inv = nrm > 0.0f ? 1.0f / nrm : 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) o.uhat[i] = eh[i] * inv;
  if (M.kind == kVonMises) {
    if (nrm - M.k_yield > 0.0f) {
      o.branch = kProject;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        o.ep[i] = mean + M.k_yield * o.uhat[i];
        o.s[i] = expf(o.ep[i]);
      }
    } else {
      o.branch = kElastic;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        o.ep[i] = o.eps[i];
        o.s[i] = sg[i];
      }
    }
    float J = o.s[0] * o.s[1] * o.s[2];
    float pj = M.lam * J * (J - 1.0f);
#pragma unroll
    for (int i = 0; i < 3; ++i) o.t[i] = 2.0f * M.mu * (o.s[i] - 1.0f) * o.s[i] + pj;
  } else {  // Drucker-Prager
    float dg = nrm + M.c_dp * tr;
    if (dg <= 0.0f) {
      o.branch = kElastic;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        o.ep[i] = o.eps[i];
        o.s[i] = sg[i];
      }
    } else if (tr > 0.0f || nrm == 0.0f) {
      o.branch = kApex;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        o.ep[i] = 0.0f;
        o.s[i] = 1.0f;
      }
    } else {
      o.branch = kProject;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        o.ep[i] = o.eps[i] - dg * o.uhat[i];
        o.s[i] = expf(o.ep[i]);
      }
    }
    float tre = o.ep[0] + o.ep[1] + o.ep[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) o.t[i] = 2.0f * M.mu * o.ep[i] + M.lam * tre;
  }
}

// Forward: projected F_p and Kirchhoff stress tau of a solid particle; if
// usv is given, also its SVD (U, sigma, V: 9 + 3 + 9 floats).
template <bool kExt = true>
__device__ inline void solid_forward(const MatParams& M, const float* F, float* Fp, float* tau,
                                     float* usv = nullptr) {
  float U[9], sg[3], V[9];
  svd3(F, U, sg, V);
  if (usv) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      usv[i] = U[i];
      usv[12 + i] = V[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) usv[9 + i] = sg[i];
  }
  SigmaMap o;
  sigma_map<kExt>(M, sg, o);
  if (o.branch == kElastic) {
#pragma unroll
    for (int i = 0; i < 9; ++i) Fp[i] = F[i];
  } else {
    udwt(U, o.s, V, Fp);
  }
  udwt(U, o.t, U, tau);
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
// (e^a - e^b) / (a - b) = e^b * expm1(a - b) / (a - b)
__device__ inline float exp_dd(float a, float b) {
  float d = a - b;
  float e1 = (d == 0.0f) ? 1.0f : expm1f(d) / d;
  return expf(b) * e1;
}
// (log max(si, floor) - log max(sj, floor)) / (si - sj)
__device__ inline float log_dd(float si, float sj) {
  bool ci = si > kSigmaFloor, cj = sj > kSigmaFloor;
  if (ci && cj) {
    float d = si - sj;
    if (d == 0.0f) return 1.0f / sj;
    float r = d / sj;
    return log1pf(r) / d;
  }
  if (!ci && !cj) return 0.0f;
  return (hencky(si) - hencky(sj)) / (si - sj);
}
__device__ inline float safe_den(float a) {
  return copysignf(fmaxf(fabsf(a), 1e-6f), a);
}

// Kirchhoff stress from a stored SVD of the trial F.
template <bool kExt = true>
__device__ inline void solid_tau_from_svd(const MatParams& M, const float* U, const float* sg,
                                          float* tau) {
  SigmaMap o;
  sigma_map<kExt>(M, sg, o);
  udwt(U, o.t, U, tau);
}

// Fbar = dPhi/dF^T [Fbar_p, taubar] for a solid particle whose trial F has
// the SVD (U, sg, V).
template <bool kExt = true>
__device__ inline void solid_adjoint_svd(const MatParams& M, const float* U, const float* sg,
                                         const float* V, const float* gFp, const float* gtau,
                                         float* Fbar) {
  SigmaMap o;
  sigma_map<kExt>(M, sg, o);
  float c[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) c[k] = sg[k] > kSigmaFloor ? 1.0f / sg[k] : 0.0f;
  float Js[9], Jt[9], Ds[3], Dt[3];  // pairs (0,1), (0,2), (1,2)
  const int PI[3] = {0, 0, 1}, PJ[3] = {1, 2, 2};
  const float mu = M.mu, lam = M.lam;
  if (kExt && M.kind == kBoxYield) {
    // s_i = clamp(sigma_i): ds_i/dsigma_k = chi_i delta_ik (chi = 1 inside the
    // box); t_i = 2 mu (s_i - 1) s_i + lam J (J - 1), J = s_0 s_1 s_2, so
    // dt_i/dsigma_k = delta_ik 2 mu (2 s_i - 1) chi_i + lam (2 J - 1) (J / s_k) chi_k,
    // and t_i - t_j = 2 mu (s_i - s_j)(s_i + s_j - 1).
    const float lo = 1.0f - M.k_yield, hi = 1.0f + M.c_dp;
    float chi[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) chi[i] = (sg[i] >= lo && sg[i] <= hi) ? 1.0f : 0.0f;
    const float J = o.s[0] * o.s[1] * o.s[2];
    const float Pk[3] = {o.s[1] * o.s[2], o.s[0] * o.s[2], o.s[0] * o.s[1]};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        Js[3 * i + k] = (i == k) ? chi[i] : 0.0f;
        Jt[3 * i + k] = ((i == k) ? 2.0f * mu * (2.0f * o.s[i] - 1.0f) * chi[i] : 0.0f) +
                        lam * (2.0f * J - 1.0f) * Pk[k] * chi[k];
      }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int i = PI[q], j = PJ[q];
      float d;
      if (chi[i] > 0.0f && chi[j] > 0.0f) {
        d = 1.0f;  // both inside: s = sigma
      } else if (o.s[i] == o.s[j]) {
        d = 0.0f;  // clamped to the same value
      } else {
        // (s_i - s_j) / (sigma_i - sigma_j) lies in [0, 1]: keep it there under rounding
        d = fminf(fmaxf((o.s[i] - o.s[j]) / (sg[i] - sg[j]), 0.0f), 1.0f);
      }
      Ds[q] = d;
      Dt[q] = 2.0f * mu * (o.s[i] + o.s[j] - 1.0f) * d;
    }
  } else if (M.kind == kVonMises || (kExt && M.kind == kViscousLiquid)) {
    if (o.branch == kElastic) {
      float J = sg[0] * sg[1] * sg[2];
      float Pk[3] = {sg[1] * sg[2], sg[0] * sg[2], sg[0] * sg[1]};
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          Js[3 * i + k] = (i == k) ? 1.0f : 0.0f;
          Jt[3 * i + k] = ((i == k) ? 2.0f * mu * (2.0f * sg[i] - 1.0f) : 0.0f) +
                          lam * (2.0f * J - 1.0f) * Pk[k];
        }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        Ds[q] = 1.0f;
        Dt[q] = 2.0f * mu * (sg[PI[q]] + sg[PJ[q]] - 1.0f);
      }
    } else {
      float kn = M.k_yield / o.nrm;
      float J = o.s[0] * o.s[1] * o.s[2];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          float E = (1.0f / 3.0f) + kn * (((i == k) ? 1.0f : 0.0f) - (1.0f / 3.0f) - o.uhat[i] * o.uhat[k]);
          Js[3 * i + k] = o.s[i] * E * c[k];
        }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          Jt[3 * i + k] = 2.0f * mu * (2.0f * o.s[i] - 1.0f) * Js[3 * i + k] +
                          lam * (2.0f * J - 1.0f) * J * c[k];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        int i = PI[q], j = PJ[q];
        Ds[q] = exp_dd(o.ep[i], o.ep[j]) * kn * log_dd(sg[i], sg[j]);
        Dt[q] = 2.0f * mu * (o.s[i] + o.s[j] - 1.0f) * Ds[q];
      }
    }
  } else {
    if (o.branch == kElastic) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          Js[3 * i + k] = (i == k) ? 1.0f : 0.0f;
          Jt[3 * i + k] = (((i == k) ? 2.0f * mu : 0.0f) + lam) * c[k];
        }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        Ds[q] = 1.0f;
        Dt[q] = 2.0f * mu * log_dd(sg[PI[q]], sg[PJ[q]]);
      }
    } else if (o.branch == kApex) {
#pragma unroll
      for (int i = 0; i < 9; ++i) Js[i] = Jt[i] = 0.0f;
#pragma unroll
      for (int q = 0; q < 3; ++q) Ds[q] = Dt[q] = 0.0f;
    } else {
      float B = -M.c_dp * o.tr / o.nrm;
      float trn = o.tr / o.nrm;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          float E = (1.0f / 3.0f) -
                    M.c_dp * (o.uhat[i] + trn * (((i == k) ? 1.0f : 0.0f) - (1.0f / 3.0f) - o.uhat[i] * o.uhat[k]));
          Js[3 * i + k] = o.s[i] * E * c[k];
          Jt[3 * i + k] = (2.0f * mu * E + lam) * c[k];
        }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        int i = PI[q], j = PJ[q];
        float L = log_dd(sg[i], sg[j]);
        Ds[q] = exp_dd(o.ep[i], o.ep[j]) * B * L;
        Dt[q] = 2.0f * mu * B * L;
      }
    }
  }
  // Z accumulation
  float Z[9];
  float tmp[9], Mx[9], Nx[9];
  // N = U^T taubar U
  mat_tmul(U, gtau, tmp);
  mat_mul(tmp, U, Nx);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float z = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) z += Nx[4 * k] * Jt[3 * k + i];
    Z[4 * i] = z;
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    int i = PI[q], j = PJ[q];
    float den = safe_den(sg[i] + sg[j]);
    float ns = Nx[3 * i + j] + Nx[3 * j + i];
    Z[3 * i + j] = Dt[q] * sg[j] * ns / den;
    Z[3 * j + i] = Dt[q] * sg[i] * ns / den;
  }
  bool proj = o.branch != kElastic;
  if (proj) {
    // M = U^T Fbar_p V
    mat_tmul(U, gFp, tmp);
    mat_mul(tmp, V, Mx);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float z = 0.0f;
#pragma unroll
      for (int k = 0; k < 3; ++k) z += Mx[4 * k] * Js[3 * k + i];
      Z[4 * i] += z;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      int i = PI[q], j = PJ[q];
      float Dp = (o.s[i] + o.s[j]) / safe_den(sg[i] + sg[j]);
      float a = 0.5f * (Ds[q] + Dp), b = 0.5f * (Ds[q] - Dp);
      float mij = Mx[3 * i + j], mji = Mx[3 * j + i];
      Z[3 * i + j] += a * mij + b * mji;
      Z[3 * j + i] += a * mji + b * mij;
    }
  }
  // Fbar = U Z V^T (+ Fbar_p on the elastic branch)
  float UZ[9];
  mat_mul(U, Z, UZ);
  float out[9];
  mat_mult(UZ, V, out);
#pragma unroll
  for (int i = 0; i < 9; ++i) Fbar[i] = out[i] + (proj ? 0.0f : gFp[i]);
}

// Same, computing the SVD of the trial F first.
__device__ inline void solid_adjoint(const MatParams& M, const float* F, const float* gFp,
                                     const float* gtau, float* Fbar) {
  float U[9], sg[3], V[9];
  svd3(F, U, sg, V);
  solid_adjoint_svd(M, U, sg, V, gFp, gtau, Fbar);
}

}  // namespace mpm
