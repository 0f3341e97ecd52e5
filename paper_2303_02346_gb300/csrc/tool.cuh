// Kinematic box tool: SDF, soft Coulomb contact and its adjoint (device code).
//
// Paper Sec. 3.2 "Inter-material coupling": contact between SDF objects and
// particle material is computed on the grid from the SDF normal with Coulomb
// friction (Stomakhin et al. 2013). Sec. 5.1 "Soft Contact Model": contact acts
// within a distance threshold, and the post-contact velocity v_c is blended
// with the original one by alpha = min(exp(-d), 1); here d = phi / l with phi
// the signed distance and l the softness length.
#pragma once

#include "common.cuh"

namespace mpm {

struct ToolState {
  float p[3], q[4], R[9], pd[3], om[3];
};

__device__ inline void quat_rot(const float* q, float* R) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.0f - 2.0f * (y * y + z * z);
  R[1] = 2.0f * (x * y - w * z);
  R[2] = 2.0f * (x * z + w * y);
  R[3] = 2.0f * (x * y + w * z);
  R[4] = 1.0f - 2.0f * (x * x + z * z);
  R[5] = 2.0f * (y * z - w * x);
  R[6] = 2.0f * (x * z - w * y);
  R[7] = 2.0f * (y * z + w * x);
  R[8] = 1.0f - 2.0f * (x * x + y * y);
}

__device__ inline void load_tool(const float* pose, ToolState& t) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    t.p[i] = pose[i];
    t.pd[i] = pose[7 + i];
    t.om[i] = pose[10 + i];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) t.q[i] = pose[3 + i];
  quat_rot(t.q, t.R);
}

// Box SDF in the tool frame: phi and its gradient g (unit) w.r.t. y.
struct SdfEval {
  float r[3], y[3], sgn[3], e[3];
  float phi, g[3], n[3];
  float nrm;   // |max(e, 0)| when outside
  int outside, kmax;
};

__device__ inline void eval_sdf(const Params& P, const ToolState& T, const float* xi, SdfEval& s) {
#pragma unroll
  for (int d = 0; d < 3; ++d) s.r[d] = xi[d] - T.p[d];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    s.y[a] = T.R[a] * s.r[0] + T.R[3 + a] * s.r[1] + T.R[6 + a] * s.r[2];
    s.sgn[a] = s.y[a] >= 0.0f ? 1.0f : -1.0f;
    s.e[a] = fabsf(s.y[a]) - P.half[a];
  }
  s.outside = (s.e[0] > 0.0f) || (s.e[1] > 0.0f) || (s.e[2] > 0.0f);
  if (s.outside) {
    float ep0 = fmaxf(s.e[0], 0.0f), ep1 = fmaxf(s.e[1], 0.0f), ep2 = fmaxf(s.e[2], 0.0f);
    float nrm = sqrtf(ep0 * ep0 + ep1 * ep1 + ep2 * ep2);
    s.nrm = nrm;
    s.phi = nrm;
    float inv = 1.0f / nrm;
    s.g[0] = s.sgn[0] * ep0 * inv;
    s.g[1] = s.sgn[1] * ep1 * inv;
    s.g[2] = s.sgn[2] * ep2 * inv;
    s.kmax = -1;
  } else {
    // axis of the largest e (lowest axis on a tie), without dynamic indexing
    const bool k1 = s.e[1] > s.e[0];
    const float e01 = k1 ? s.e[1] : s.e[0];
    const bool k2 = s.e[2] > e01;
    const int k = k2 ? 2 : (k1 ? 1 : 0);
    s.kmax = k;
    s.phi = k2 ? s.e[2] : e01;
    s.nrm = 0.0f;
    s.g[0] = k == 0 ? s.sgn[0] : 0.0f;
    s.g[1] = k == 1 ? s.sgn[1] : 0.0f;
    s.g[2] = k == 2 ? s.sgn[2] : 0.0f;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d)
    s.n[d] = T.R[3 * d] * s.g[0] + T.R[3 * d + 1] * s.g[1] + T.R[3 * d + 2] * s.g[2];
}

// v: node velocity before contact (in) / after contact (out).
__device__ inline void contact_forward(const Params& P, const ToolState& T, const float* xi, float* v) {
  SdfEval s;
  eval_sdf(P, T, xi, s);
  if (!(s.phi < P.eps_c)) return;
  float vT[3] = {T.pd[0] + T.om[1] * s.r[2] - T.om[2] * s.r[1],
                 T.pd[1] + T.om[2] * s.r[0] - T.om[0] * s.r[2],
                 T.pd[2] + T.om[0] * s.r[1] - T.om[1] * s.r[0]};
  float vr[3] = {v[0] - vT[0], v[1] - vT[1], v[2] - vT[2]};
  float vn = vr[0] * s.n[0] + vr[1] * s.n[1] + vr[2] * s.n[2];
  if (!(vn < 0.0f)) return;
  float t[3] = {vr[0] - vn * s.n[0], vr[1] - vn * s.n[1], vr[2] - vn * s.n[2]};
  float tn = sqrtf(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  float vrn[3];
  if (tn <= -P.mu_f * vn) {
    vrn[0] = vrn[1] = vrn[2] = 0.0f;
  } else {
    float f = 1.0f + P.mu_f * vn / tn;
    vrn[0] = t[0] * f;
    vrn[1] = t[1] * f;
    vrn[2] = t[2] * f;
  }
  float alpha = s.phi > 0.0f ? expf(-s.phi * P.inv_ell) : 1.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) v[d] = alpha * (vrn[d] + vT[d]) + (1.0f - alpha) * v[d];
}

// Adjoint of contact_forward. u: velocity before contact; vbar: dL/d(output).
// Writes ubar = dL/du and adds the tool gradients of this node to
// gp (position), gR (rotation matrix), gpd (linear velocity), gom (angular velocity).
__device__ inline void contact_adjoint(const Params& P, const ToolState& T, const float* xi,
                                       const float* u, const float* vbar, float* ubar,
                                       float* gp, float* gR, float* gpd, float* gom) {
#pragma unroll
  for (int d = 0; d < 3; ++d) ubar[d] = vbar[d];
  SdfEval s;
  eval_sdf(P, T, xi, s);
  if (!(s.phi < P.eps_c)) return;
  const float* r = s.r;
  float vT[3] = {T.pd[0] + T.om[1] * r[2] - T.om[2] * r[1],
                 T.pd[1] + T.om[2] * r[0] - T.om[0] * r[2],
                 T.pd[2] + T.om[0] * r[1] - T.om[1] * r[0]};
  float vr[3] = {u[0] - vT[0], u[1] - vT[1], u[2] - vT[2]};
  float vn = vr[0] * s.n[0] + vr[1] * s.n[1] + vr[2] * s.n[2];
  if (!(vn < 0.0f)) return;
  float t[3] = {vr[0] - vn * s.n[0], vr[1] - vn * s.n[1], vr[2] - vn * s.n[2]};
  float tn = sqrtf(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  bool stick = tn <= -P.mu_f * vn;
  float f = stick ? 0.0f : 1.0f + P.mu_f * vn / tn;
  float vrn[3] = {t[0] * f, t[1] * f, t[2] * f};
  bool pos = s.phi > 0.0f;
  float alpha = pos ? expf(-s.phi * P.inv_ell) : 1.0f;
  // v = alpha (vrn + vT) + (1 - alpha) u
  float vcbar[3], abar = 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ubar[d] = (1.0f - alpha) * vbar[d];
    vcbar[d] = alpha * vbar[d];
    abar += vbar[d] * (vrn[d] + vT[d] - u[d]);
  }
  float phibar = pos ? -abar * alpha * P.inv_ell : 0.0f;
  float vTbar[3] = {vcbar[0], vcbar[1], vcbar[2]};
  float vrbar[3] = {0.0f, 0.0f, 0.0f}, nbar[3] = {0.0f, 0.0f, 0.0f}, vnbar = 0.0f;
  if (!stick) {
    // vrn = t * f, f = 1 + mu vn / tn
    float tbar[3];
    float fbar = vcbar[0] * t[0] + vcbar[1] * t[1] + vcbar[2] * t[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) tbar[d] = f * vcbar[d];
    vnbar += P.mu_f * fbar / tn;
    float tnbar = -P.mu_f * vn * fbar / (tn * tn);
#pragma unroll
    for (int d = 0; d < 3; ++d) tbar[d] += tnbar * t[d] / tn;
    // t = vr - vn n
    float tdotn = tbar[0] * s.n[0] + tbar[1] * s.n[1] + tbar[2] * s.n[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      vrbar[d] += tbar[d];
      nbar[d] -= vn * tbar[d];
    }
    vnbar -= tdotn;
  }
  // vn = vr . n
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    vrbar[d] += vnbar * s.n[d];
    nbar[d] += vnbar * vr[d];
  }
  // vr = u - vT
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ubar[d] += vrbar[d];
    vTbar[d] -= vrbar[d];
  }
  // vT = pd + om x r
  float rbar[3];
  gpd[0] += vTbar[0];
  gpd[1] += vTbar[1];
  gpd[2] += vTbar[2];
  gom[0] += r[1] * vTbar[2] - r[2] * vTbar[1];
  gom[1] += r[2] * vTbar[0] - r[0] * vTbar[2];
  gom[2] += r[0] * vTbar[1] - r[1] * vTbar[0];
  rbar[0] = vTbar[1] * T.om[2] - vTbar[2] * T.om[1];
  rbar[1] = vTbar[2] * T.om[0] - vTbar[0] * T.om[2];
  rbar[2] = vTbar[0] * T.om[1] - vTbar[1] * T.om[0];
  // n = R g: gR += nbar g^T, gbar = R^T nbar
  float gbar[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gbar[a] = T.R[a] * nbar[0] + T.R[3 + a] * nbar[1] + T.R[6 + a] * nbar[2];
#pragma unroll
    for (int b = 0; b < 3; ++b) gR[3 * a + b] += nbar[a] * s.g[b];
  }
  // y: phi(y) has gradient g; g(y) depends on y only outside
  float ybar[3] = {phibar * s.g[0], phibar * s.g[1], phibar * s.g[2]};
  if (s.outside) {
    // g = sgn * ep / |ep|; with ghat = ep / |ep| (the ep > 0 components):
    // d(ep/|ep|) = (I - ghat ghat^T) dep / |ep|, dep_k = sgn_k dy_k (ep_k > 0)
    float gh[3], w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      gh[a] = s.g[a] * s.sgn[a];
      w[a] = s.sgn[a] * gbar[a];  // dL/d(ghat)
    }
    float wd = w[0] * gh[0] + w[1] * gh[1] + w[2] * gh[2];
    float inv = 1.0f / s.nrm;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float epbar = (w[a] - gh[a] * wd) * inv;
      if (s.e[a] > 0.0f) ybar[a] += s.sgn[a] * epbar;
    }
  }
  // y = R^T r: rbar += R ybar; gR += r ybar^T
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    rbar[a] += T.R[3 * a] * ybar[0] + T.R[3 * a + 1] * ybar[1] + T.R[3 * a + 2] * ybar[2];
#pragma unroll
    for (int b = 0; b < 3; ++b) gR[3 * a + b] += r[a] * ybar[b];
  }
  // r = xi - p
  gp[0] -= rbar[0];
  gp[1] -= rbar[1];
  gp[2] -= rbar[2];
}

}  // namespace mpm
