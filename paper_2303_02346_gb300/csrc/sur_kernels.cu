// Surrogate kernels other than the tensor-core convolution and its weight
// gradient: weight layout preparation, grid features and their velocity
// adjoint, the 1x1x1 lift and projection (with loss, gradients and error
// sums), the lift backward, and Adam.
#include <cuda_bf16.h>

#include <algorithm>

#include "sur_kernels.h"

namespace sur {
namespace {

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

__device__ __forceinline__ float rbf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// offsets into the flat parameter vector
__host__ __device__ inline long long conv_w_offset(int layer) {  // layer = 2 * block + (0: w1, 1: w2)
  return 288ll + static_cast<long long>(layer / 2) * 2 * (27 * 1024 + 32) + (layer % 2) * (27 * 1024 + 32);
}

// ---------------------------------------------------------------------------
// weights: FP32 master W[a][b][c][o][q] -> the BF16 UMMA A layout of the
// convolution (sur_conv.cu), [row c*32 + o][pair a*3+b][q]; the
// backward layout holds the mirrored taps with the channel roles swapped,
// W'[2-a][2-b][2-c][q][o] = W[a][b][c][o][q] (the input gradient of conv3 is
// conv3 of the output gradient with these weights). Rows 96..127 of every
// pair stay zero (set once at allocation).
// ---------------------------------------------------------------------------
__global__ void prep_weights_kernel(const float* params, int layers, __nv_bfloat16* wf, __nv_bfloat16* wb) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<long long>(layers) * 27 * 1024) return;
  const int L = static_cast<int>(i / (27 * 1024));
  const int rem = static_cast<int>(i % (27 * 1024));
  const int tap = rem / 1024, o = (rem / 32) % 32, q = rem % 32;
  const int pair = tap / 3, c = tap % 3;
  const int tapm = 26 - tap, pairm = tapm / 3, cm = tapm % 3;
  const __nv_bfloat16 w = __float2bfloat16_rn(params[conv_w_offset(L) + rem]);
  const long long base = static_cast<long long>(L) * kConvWElems;
  wf[base + ((c * 32 + o) * 9 + pair) * 32 + q] = w;
  wb[base + ((cm * 32 + q) * 9 + pairm) * 32 + o] = w;
}

// ---------------------------------------------------------------------------
// grid features: MLS-MPM quadratic B-spline transfer of m, m (v + C dpos) and
// the per-material mass, then normalisation and BF16 rounding.
// ---------------------------------------------------------------------------
struct Stencil {
  int base[3];
  float w[3][3];
  float fx[3];
};

__device__ __forceinline__ bool make_stencil(const float* x, int n, Stencil& s) {
  bool ok = true;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float xs = x[d] * n;
    const int b = static_cast<int>(floorf(xs - 0.5f));
    const float f = xs - b;
    s.base[d] = b;
    s.fx[d] = f;
    s.w[0][d] = 0.5f * (1.5f - f) * (1.5f - f);
    s.w[1][d] = 0.75f - (f - 1.0f) * (f - 1.0f);
    s.w[2][d] = 0.5f * (f - 0.5f) * (f - 0.5f);
    ok = ok && b >= 0 && b <= n - 3;
  }
  return ok;
}

__global__ void features_scatter_kernel(FeatArgs a, const float* __restrict__ x, const float* __restrict__ v,
                                        const float* __restrict__ C, const uint8_t* __restrict__ mat,
                                        float* acc, int* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.N) return;
  float xp[3] = {x[3 * p], x[3 * p + 1], x[3 * p + 2]};
  Stencil s;
  if (!make_stencil(xp, a.n, s)) {
    atomicOr(err, kErrDomain);
    return;
  }
  const int mt = mat[p];
  if (mt >= a.n_mat) {
    atomicOr(err, kErrArg);
    return;
  }
  const float mp = a.mmass[mt];
  float vp[3] = {v[3 * p], v[3 * p + 1], v[3 * p + 2]};
  float Cp[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) Cp[i] = C[9 * p + i];
  const float dx = 1.0f / a.n;
  const int n = a.n;
#pragma unroll
  for (int oi = 0; oi < 3; ++oi)
#pragma unroll
    for (int oj = 0; oj < 3; ++oj)
#pragma unroll
      for (int ok = 0; ok < 3; ++ok) {
        const float W = s.w[oi][0] * s.w[oj][1] * s.w[ok][2];
        const float d0 = (oi - s.fx[0]) * dx, d1 = (oj - s.fx[1]) * dx, d2 = (ok - s.fx[2]) * dx;
        const float wm = W * mp;
        const long long node =
            (static_cast<long long>(s.base[0] + oi) * n + (s.base[1] + oj)) * n + (s.base[2] + ok);
        float* dst = acc + node * 8;
        atomicAdd(dst + 0, wm);
        atomicAdd(dst + 1, wm * (vp[0] + Cp[0] * d0 + Cp[1] * d1 + Cp[2] * d2));
        atomicAdd(dst + 2, wm * (vp[1] + Cp[3] * d0 + Cp[4] * d1 + Cp[5] * d2));
        atomicAdd(dst + 3, wm * (vp[2] + Cp[6] * d0 + Cp[7] * d1 + Cp[8] * d2));
        if (mt < 3) atomicAdd(dst + 4 + mt, wm);
      }
}

__global__ void features_finalize_kernel(FeatArgs a, float* acc, uint16_t* frame) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  const long long n3 = static_cast<long long>(a.n) * a.n * a.n;
  if (i >= n3) return;
  float4* src = reinterpret_cast<float4*>(acc + i * 8);
  const float4 u = src[0], w = src[1];
  float o[8];
  const float m = u.x;
  o[0] = m * a.inv_mref;
  o[1] = u.y * a.inv_mvref;
  o[2] = u.z * a.inv_mvref;
  o[3] = u.w * a.inv_mvref;
  const float inv = m > 0.0f ? 1.0f / m : 0.0f;
  o[4] = w.x * inv;
  o[5] = w.y * inv;
  o[6] = w.z * inv;
  o[7] = 0.0f;
  reinterpret_cast<uint4*>(frame)[i] = pack8(o);
  src[0] = make_float4(0.f, 0.f, 0.f, 0.f);
  src[1] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Adjoint of the mass and momentum channels of the transfer, for a cotangent
// g (FP32 [n^3][8]; channels 4..7 are not differentiated): with s = m_p /
// (m_ref v_ref), d = x_i - x_p and grad W the B-spline weight gradient,
//   dL/dv_p = s sum_i W g_i[1:4]
//   dL/dC_p = s sum_i W g_i[1:4] d^T
//   dL/dx_p = sum_i (s g_i[1:4] . (v_p + C_p d) + g_i[0] m_p / m_ref) grad W - s W C_p^T g_i[1:4]
__global__ void features_vjp_kernel(FeatArgs a, const float* __restrict__ x, const float* __restrict__ v,
                                    const float* __restrict__ C, const uint8_t* __restrict__ mat,
                                    const float* __restrict__ g, float* dLdx, float* dLdv, float* dLdC, int* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.N) return;
  float xp[3] = {x[3 * p], x[3 * p + 1], x[3 * p + 2]};
  Stencil st;
  if (!make_stencil(xp, a.n, st) || mat[p] >= a.n_mat) {
    atomicOr(err, kErrDomain);
    if (dLdx) dLdx[3 * p] = dLdx[3 * p + 1] = dLdx[3 * p + 2] = 0.0f;
    if (dLdv) dLdv[3 * p] = dLdv[3 * p + 1] = dLdv[3 * p + 2] = 0.0f;
    if (dLdC)
      for (int k = 0; k < 9; ++k) dLdC[9 * p + k] = 0.0f;
    return;
  }
  const float mp = a.mmass[mat[p]];
  const float sm = mp * a.inv_mvref, smass = mp * a.inv_mref;
  const float dx = 1.0f / a.n, inv_dx = static_cast<float>(a.n);
  float vp[3] = {0.f, 0.f, 0.f}, Cp[9];
  if (v) {
    vp[0] = v[3 * p];
    vp[1] = v[3 * p + 1];
    vp[2] = v[3 * p + 2];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) Cp[k] = C ? C[9 * p + k] : 0.0f;
  // B-spline weight derivatives w.r.t. f (= x inv_dx - base)
  float dw[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float f = st.fx[d];
    dw[0][d] = -(1.5f - f);
    dw[1][d] = -2.0f * (f - 1.0f);
    dw[2][d] = f - 0.5f;
  }
  const int n = a.n;
  float gv[3] = {0.f, 0.f, 0.f}, gC[9], gx[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 9; ++k) gC[k] = 0.0f;
  for (int oi = 0; oi < 3; ++oi)
    for (int oj = 0; oj < 3; ++oj)
#pragma unroll
      for (int ok = 0; ok < 3; ++ok) {
        const float W = st.w[oi][0] * st.w[oj][1] * st.w[ok][2];
        const float gW[3] = {dw[oi][0] * st.w[oj][1] * st.w[ok][2] * inv_dx,
                             st.w[oi][0] * dw[oj][1] * st.w[ok][2] * inv_dx,
                             st.w[oi][0] * st.w[oj][1] * dw[ok][2] * inv_dx};
        const float d[3] = {(oi - st.fx[0]) * dx, (oj - st.fx[1]) * dx, (ok - st.fx[2]) * dx};
        const long long node =
            (static_cast<long long>(st.base[0] + oi) * n + (st.base[1] + oj)) * n + (st.base[2] + ok);
        const float* gn = g + node * 8;
        const float g0 = gn[0], gm[3] = {gn[1], gn[2], gn[3]};
        float mom[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) mom[r] = vp[r] + Cp[3 * r] * d[0] + Cp[3 * r + 1] * d[1] + Cp[3 * r + 2] * d[2];
        const float coef = sm * (gm[0] * mom[0] + gm[1] * mom[1] + gm[2] * mom[2]) + g0 * smass;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          gx[c] += coef * gW[c] - sm * W * (Cp[c] * gm[0] + Cp[3 + c] * gm[1] + Cp[6 + c] * gm[2]);
          gv[c] += sm * W * gm[c];
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) gC[3 * r + c] += sm * W * gm[r] * d[c];
      }
  if (dLdx)
    for (int c = 0; c < 3; ++c) dLdx[3 * p + c] = gx[c];
  if (dLdv)
    for (int c = 0; c < 3; ++c) dLdv[3 * p + c] = gv[c];
  if (dLdC)
    for (int k = 0; k < 9; ++k) dLdC[9 * p + k] = gC[k];
}

// (i, j, k) of node v = (i n + j) n + k of a frame: 32-bit divisions (a frame
// has n^3 < 2^32 nodes), far cheaper than 64-bit ones in these load-bound loops.
__device__ __forceinline__ void split_node(const SurGeom& g, long long v, int& i, int& j, int& k) {
  const unsigned n = static_cast<unsigned>(g.n), u = static_cast<unsigned>(v);
  const unsigned ij = u / n;
  k = static_cast<int>(u - ij * n);
  i = static_cast<int>(ij / n);
  j = static_cast<int>(ij - static_cast<unsigned>(i) * n);
}

// ---------------------------------------------------------------------------
// lift: h0 = bf16(W_l f + b_l) at every interior row
// ---------------------------------------------------------------------------
__global__ void lift_kernel(SurGeom g, const uint16_t* __restrict__ frames, const int* __restrict__ idx,
                            const float* __restrict__ wl, const float* __restrict__ bl, __nv_bfloat16* h0) {
  __shared__ float sw[32 * 8 + 32];
  for (int i = threadIdx.x; i < 256 + 32; i += blockDim.x) sw[i] = i < 256 ? rbf(wl[i]) : bl[i - 256];
  __syncthreads();
  const int b = blockIdx.y;
  const long long n3 = static_cast<long long>(g.n) * g.n * g.n;
  const long long fr = idx ? idx[b] : b;
  for (long long vtx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; vtx < n3;
       vtx += static_cast<long long>(gridDim.x) * blockDim.x) {
    float f[8];
    unpack8(reinterpret_cast<const uint4*>(frames)[fr * n3 + vtx], f);
    int i, j, k;
    split_node(g, vtx, i, j, k);
    const long long row = pad_row(g, b, i, j, k);
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      float o[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int oc = c * 8 + e;
        float s = sw[256 + oc];
#pragma unroll
        for (int q = 0; q < 8; ++q) s += sw[oc * 8 + q] * f[q];
        o[e] = s;
      }
      *reinterpret_cast<uint4*>(h0 + (c * g.plane + row) * 8) = pack8(o);
    }
  }
}

// ---------------------------------------------------------------------------
// projection: pred = f[1:4] + W_p h + b_p, optionally with the loss, dL/dh
// (BF16), dL/dW_p, dL/db_p and per-frame error sums
// ---------------------------------------------------------------------------
constexpr int kProjThreads = 256;

template <int MODE>
__global__ void __launch_bounds__(kProjThreads) proj_kernel(SurGeom g, int batch,
                                                            const uint16_t* __restrict__ frames,
                                                            const int* __restrict__ idx,
                                                            const int* __restrict__ tgt,
                                                            const __nv_bfloat16* __restrict__ h,
                                                            const float* __restrict__ wp,
                                                            const float* __restrict__ bp, float* pred,
                                                            __nv_bfloat16* g_h, float* g_pred, float* grad_wp,
                                                            double* loss_acc, double* frame_sums) {
  __shared__ float sw[96 + 3];
  __shared__ float red[kProjThreads / 32][101];
  for (int i = threadIdx.x; i < 99; i += blockDim.x) sw[i] = i < 96 ? rbf(wp[i]) : bp[i - 96];
  __syncthreads();
  const int b = blockIdx.y;
  const long long n3 = static_cast<long long>(g.n) * g.n * g.n;
  const long long fr = idx ? idx[b] : b;
  const long long ft = tgt ? tgt[b] : 0;
  const float inv_count = 1.0f / (static_cast<float>(batch) * static_cast<float>(n3) * 3.0f);
  constexpr bool want_grad = MODE & 2, want_sums = MODE & 4, given = MODE & 8;
  float gw[96], gb[3], l2 = 0.f, t2 = 0.f;
  if (want_grad) {
#pragma unroll
    for (int i = 0; i < 96; ++i) gw[i] = 0.f;
    gb[0] = gb[1] = gb[2] = 0.f;
  }
  for (long long vtx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; vtx < n3;
       vtx += static_cast<long long>(gridDim.x) * blockDim.x) {
    int i, j, k;
    split_node(g, vtx, i, j, k);
    const long long row = pad_row(g, b, i, j, k);
    float hv[32];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float t[8];
      unpack8(*reinterpret_cast<const uint4*>(h + (c * g.plane + row) * 8), t);
#pragma unroll
      for (int e = 0; e < 8; ++e) hv[c * 8 + e] = t[e];
    }
    float f[8];
    unpack8(reinterpret_cast<const uint4*>(frames)[fr * n3 + vtx], f);
    float p[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float s = sw[96 + c];
#pragma unroll
      for (int o = 0; o < 32; ++o) s += sw[c * 32 + o] * hv[o];
      p[c] = f[1 + c] + s;
    }
    if (MODE & 1) {
      float* dst = pred + (static_cast<long long>(b) * n3 + vtx) * 3;
      dst[0] = p[0];
      dst[1] = p[1];
      dst[2] = p[2];
    }
    if (given) {
      // cotangent of the prediction supplied by the caller: dL/dh only
      const float* gp = g_pred + (static_cast<long long>(b) * n3 + vtx) * 3;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float o8[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int o = c * 8 + e;
          o8[e] = sw[o] * gp[0] + sw[32 + o] * gp[1] + sw[64 + o] * gp[2];
        }
        *reinterpret_cast<uint4*>(g_h + (c * g.plane + row) * 8) = pack8(o8);
      }
    }
    if (want_grad || want_sums) {
      float tf[8];
      unpack8(reinterpret_cast<const uint4*>(frames)[ft * n3 + vtx], tf);
      float d[3] = {p[0] - tf[1], p[1] - tf[2], p[2] - tf[3]};
      l2 += d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      t2 += tf[1] * tf[1] + tf[2] * tf[2] + tf[3] * tf[3];
      if (want_grad) {
        float gp[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          gp[c] = 2.0f * d[c] * inv_count;
          gb[c] += gp[c];
#pragma unroll
          for (int o = 0; o < 32; ++o) gw[c * 32 + o] += gp[c] * hv[o];
        }
        if (g_pred) {
          float* dst = g_pred + (static_cast<long long>(b) * n3 + vtx) * 3;
          dst[0] = gp[0];
          dst[1] = gp[1];
          dst[2] = gp[2];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float o8[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int o = c * 8 + e;
            o8[e] = sw[o] * gp[0] + sw[32 + o] * gp[1] + sw[64 + o] * gp[2];
          }
          *reinterpret_cast<uint4*>(g_h + (c * g.plane + row) * 8) = pack8(o8);
        }
      }
    }
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (want_grad) {
#pragma unroll 4
    for (int i = 0; i < 96; ++i) {
      const float s = warp_sum(gw[i]);
      if (lane == 0) red[warp][i] = s;
    }
    for (int c = 0; c < 3; ++c) {
      const float s = warp_sum(gb[c]);
      if (lane == 0) red[warp][96 + c] = s;
    }
  }
  const float sl = warp_sum(l2), st = warp_sum(t2);
  if (lane == 0) {
    red[warp][99] = sl;
    red[warp][100] = st;
  }
  __syncthreads();
  if (want_grad && threadIdx.x < 99) {
    float s = 0.f;
    for (int w = 0; w < kProjThreads / 32; ++w) s += red[w][threadIdx.x];
    atomicAdd(grad_wp + threadIdx.x, s);  // w_proj (96) and b_proj (3) are adjacent
  }
  if (threadIdx.x == 128 && (want_grad || want_sums)) {
    double s = 0.0, t = 0.0;
    for (int w = 0; w < kProjThreads / 32; ++w) {
      s += red[w][99];
      t += red[w][100];
    }
    if (want_grad) atomicAdd(loss_acc, s);
    if (want_sums) {
      atomicAdd(frame_sums + 2 * b, s);
      atomicAdd(frame_sums + 2 * b + 1, t);
    }
  }
}

// ---------------------------------------------------------------------------
// lift backward: dW_l, db_l and optionally dL/dframe
// ---------------------------------------------------------------------------
constexpr int kLbThreads = 256;

__global__ void __launch_bounds__(kLbThreads) lift_bwd_kernel(SurGeom g, int batch,
                                                              const uint16_t* __restrict__ frames,
                                                              const int* __restrict__ idx,
                                                              const __nv_bfloat16* __restrict__ gh,
                                                              const float* __restrict__ wl,
                                                              const float* __restrict__ g_pred, float* grad_wl,
                                                              float* grad_bl, float* g_frames) {
  __shared__ float sw[256];
  __shared__ float sg[kLbThreads][33];
  __shared__ float sf[kLbThreads][9];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) sw[i] = rbf(wl[i]);
  const int b = blockIdx.y;
  const long long n3 = static_cast<long long>(g.n) * g.n * g.n;
  const long long fr = idx ? idx[b] : b;
  const int o_me = threadIdx.x / 8, q_me = threadIdx.x % 8;  // (o, q) pair of this thread's dW_l entry
  float accw = 0.f, accb = 0.f;
  const long long step = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long base = blockIdx.x * static_cast<long long>(blockDim.x); base < n3; base += step) {
    const long long vtx = base + threadIdx.x;
    __syncthreads();
    if (vtx < n3) {
      int i, j, k;
      split_node(g, vtx, i, j, k);
      const long long row = pad_row(g, b, i, j, k);
      float gv[32];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float t[8];
        unpack8(*reinterpret_cast<const uint4*>(gh + (c * g.plane + row) * 8), t);
#pragma unroll
        for (int e = 0; e < 8; ++e) gv[c * 8 + e] = t[e];
      }
      float f[8];
      unpack8(reinterpret_cast<const uint4*>(frames)[fr * n3 + vtx], f);
#pragma unroll
      for (int o = 0; o < 32; ++o) sg[threadIdx.x][o] = gv[o];
#pragma unroll
      for (int q = 0; q < 8; ++q) sf[threadIdx.x][q] = f[q];
      if (g_frames) {
        float gf[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float s = 0.f;
#pragma unroll
          for (int o = 0; o < 32; ++o) s += sw[o * 8 + q] * gv[o];
          gf[q] = s;
        }
        const float* gp = g_pred + (static_cast<long long>(b) * n3 + vtx) * 3;
        gf[1] += gp[0];
        gf[2] += gp[1];
        gf[3] += gp[2];
        float4* dst = reinterpret_cast<float4*>(g_frames + (static_cast<long long>(b) * n3 + vtx) * 8);
        dst[0] = make_float4(gf[0], gf[1], gf[2], gf[3]);
        dst[1] = make_float4(gf[4], gf[5], gf[6], gf[7]);
      }
    } else {
#pragma unroll
      for (int o = 0; o < 32; ++o) sg[threadIdx.x][o] = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) sf[threadIdx.x][q] = 0.f;
    }
    __syncthreads();
    for (int r = 0; r < kLbThreads; ++r) accw += sg[r][o_me] * sf[r][q_me];
    if (threadIdx.x < 32)
      for (int r = 0; r < kLbThreads; ++r) accb += sg[r][threadIdx.x];
  }
  atomicAdd(grad_wl + o_me * 8 + q_me, accw);
  if (threadIdx.x < 32) atomicAdd(grad_bl + threadIdx.x, accb);
}

// ---------------------------------------------------------------------------
// Adam (Kingma and Ba 2015) with bias correction
// ---------------------------------------------------------------------------
__global__ void adam_kernel(float* p, const float* __restrict__ gr, float* m, float* v, long long count, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  if (i >= count) return;
  const float gi = gr[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

cudaError_t launch_prep_weights(const float* params, int blocks, __nv_bfloat16* wf, __nv_bfloat16* wb,
                                cudaStream_t st) {
  const long long total = 2ll * blocks * 27 * 1024;
  prep_weights_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(params, 2 * blocks, wf, wb);
  return cudaGetLastError();
}

cudaError_t launch_lift(const SurGeom& g, int batch, const uint16_t* frames, const int* idx, const float* w_lift,
                        const float* b_lift, __nv_bfloat16* h0, cudaStream_t st) {
  const long long n3 = static_cast<long long>(g.n) * g.n * g.n;
  dim3 grid(static_cast<unsigned>(std::min<long long>((n3 + 255) / 256, 256)), batch);
  lift_kernel<<<grid, 256, 0, st>>>(g, frames, idx, w_lift, b_lift, h0);
  return cudaGetLastError();
}

cudaError_t launch_proj(const SurGeom& g, int batch, int mode, const uint16_t* frames, const int* idx,
                        const int* tgt, const __nv_bfloat16* h, const float* w_proj, const float* b_proj,
                        float* pred, __nv_bfloat16* g_h, float* g_pred, float* grad_wp, double* loss_acc,
                        double* frame_sums, cudaStream_t st) {
  const long long n3 = static_cast<long long>(g.n) * g.n * g.n;
  dim3 grid(static_cast<unsigned>(std::min<long long>((n3 + kProjThreads * 8 - 1) / (kProjThreads * 8), 512)),
            batch);
  switch (mode) {
    case 1:
      proj_kernel<1><<<grid, kProjThreads, 0, st>>>(g, batch, frames, idx, tgt, h, w_proj, b_proj, pred, g_h, g_pred,
                                                    grad_wp, loss_acc, frame_sums);
      break;
    case 2:
      proj_kernel<2><<<grid, kProjThreads, 0, st>>>(g, batch, frames, idx, tgt, h, w_proj, b_proj, pred, g_h, g_pred,
                                                    grad_wp, loss_acc, frame_sums);
      break;
    case 4:
      proj_kernel<4><<<grid, kProjThreads, 0, st>>>(g, batch, frames, idx, tgt, h, w_proj, b_proj, pred, g_h, g_pred,
                                                    grad_wp, loss_acc, frame_sums);
      break;
    case 8:
      proj_kernel<8><<<grid, kProjThreads, 0, st>>>(g, batch, frames, idx, tgt, h, w_proj, b_proj, pred, g_h, g_pred,
                                                    grad_wp, loss_acc, frame_sums);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_lift_bwd(const SurGeom& g, int batch, const uint16_t* frames, const int* idx,
                            const __nv_bfloat16* g_h0, const float* w_lift, const float* g_pred, float* grad_wl,
                            float* grad_bl, float* g_frames, cudaStream_t st) {
  const long long n3 = static_cast<long long>(g.n) * g.n * g.n;
  dim3 grid(static_cast<unsigned>(std::min<long long>((n3 + kLbThreads - 1) / kLbThreads, 128)), batch);
  lift_bwd_kernel<<<grid, kLbThreads, 0, st>>>(g, batch, frames, idx, g_h0, w_lift, g_pred, grad_wl, grad_bl,
                                               g_frames);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* grad, float* m, float* v, long long count, float lr, float beta1,
                        float beta2, float eps, int t, cudaStream_t st) {
  const float c1 = 1.0f - powf(beta1, static_cast<float>(t));
  const float c2 = 1.0f - powf(beta2, static_cast<float>(t));
  adam_kernel<<<static_cast<unsigned>((count + 255) / 256), 256, 0, st>>>(p, grad, m, v, count, lr, beta1, beta2,
                                                                          eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_features(const FeatArgs& a, const float* x, const float* v, const float* C, const uint8_t* mat,
                            float* acc, uint16_t* frame, int* err, cudaStream_t st) {
  if (a.N > 0) features_scatter_kernel<<<(a.N + 255) / 256, 256, 0, st>>>(a, x, v, C, mat, acc, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n3 = static_cast<long long>(a.n) * a.n * a.n;
  features_finalize_kernel<<<static_cast<unsigned>((n3 + 255) / 256), 256, 0, st>>>(a, acc, frame);
  return cudaGetLastError();
}

cudaError_t launch_features_vjp(const FeatArgs& a, const float* x, const float* v, const float* C,
                                const uint8_t* mat, const float* g_frame, float* dLdx, float* dLdv, float* dLdC,
                                int* err, cudaStream_t st) {
  if (a.N > 0)
    features_vjp_kernel<<<(a.N + 255) / 256, 256, 0, st>>>(a, x, v, C, mat, g_frame, dLdx, dLdv, dLdC, err);
  return cudaGetLastError();
}

}  // namespace sur
