// Host implementation of the surrogate C-ABI (include/mpm_surrogate.h).
//
// Device memory owned by a handle:
//   params, adam_m, adam_v, grad   FP32 flat vectors (sur_param_count floats)
//   wf, wb                         BF16 conv weights of the 2B layers in the UMMA B
//                                  layout, forward and mirrored-transposed (backward)
//   h[0..B], r[0..B-1]             stored activations (padded channel-planar BF16,
//                                  sur_kernels.h), zero halo
//   gh[2], ga                      activation gradients (same layout)
//   gpred                          dL/dpred (FP32) when the input gradient is wanted
//   partial                        per-CTA partial sums of the conv weight gradient
//   feat_acc                       FP32 accumulation grid of the feature transfer
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "mpm_surrogate.h"
#include "sur_kernels.h"

using namespace sur;

namespace {

struct SurProf {
  const char* name;
  cudaEvent_t a, b;
};

}  // namespace

struct mpm_surrogate {
  sur_config cfg;
  SurGeom g;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int B = 0;
  long long np = 0;
  float *params = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr;
  int t = 0;
  __nv_bfloat16 *wf = nullptr, *wb = nullptr;
  std::vector<__nv_bfloat16*> h, r;
  __nv_bfloat16 *gh[2] = {nullptr, nullptr}, *ga = nullptr;
  float* gpred = nullptr;
  float* partial = nullptr;
  int n_part = 0;
  int mn_swap = 0;  // descriptor offset assignment of MN-major operands (self-test)
  int apack = 0;    // BF16 pair order of an A operand in tensor memory (self-test)
  float* feat_acc = nullptr;
  double* dsum = nullptr;
  int* err = nullptr;
  bool dirty = true;
  std::string last_error;
  bool prof = false;
  std::vector<SurProf> prof_recs;
  long long launches = 0;
  std::vector<void*> allocs;
};

namespace {

sim_status fail(sur_h h, sim_status s, const std::string& msg) {
  if (h) h->last_error = msg;
  return s;
}

sim_status cuda_fail(sur_h h, cudaError_t e, const char* where) {
  return fail(h, SIM_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <class T>
bool dalloc(sur_h h, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  h->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return true;
}

struct Prof {
  sur_h h;
  const char* name;
  cudaEvent_t a = nullptr;
  Prof(sur_h hh, const char* nm) : h(hh), name(nm) {
    if (h->prof) {
      cudaEventCreate(&a);
      cudaEventRecord(a, h->stream);
    }
  }
  ~Prof() {
    if (h->prof) {
      cudaEvent_t b;
      cudaEventCreate(&b);
      cudaEventRecord(b, h->stream);
      h->prof_recs.push_back({name, a, b});
    }
  }
};

bool valid_config(const sur_config* c) {
  return c && c->grid_n >= 8 && c->grid_n <= 64 && c->channels == kC && c->blocks >= 1 && c->blocks <= 8 &&
         c->max_batch >= 1 && c->m_ref > 0.0f && c->v_ref > 0.0f && std::isfinite(c->m_ref) &&
         std::isfinite(c->v_ref) && c->adam_beta1 >= 0.0f && c->adam_beta1 < 1.0f && c->adam_beta2 >= 0.0f &&
         c->adam_beta2 < 1.0f && c->adam_eps > 0.0f;
}

long long count_params(int C, int B) { return C * kCin + C + 2ll * B * (27ll * C * C + C) + 3 * C + 3; }
long long w1_off(int b) { return 288ll + 2ll * b * (27 * 1024 + 32); }
long long w2_off(int b) { return w1_off(b) + 27 * 1024 + 32; }
long long proj_off(int B) { return 288ll + 2ll * B * (27 * 1024 + 32); }

// Hardware check of the UMMA operand layouts the kernels rely on, once per
// process and device: 128 x 32 x 32 products against host sums, K-major
// shared-memory operands, MN-major shared-memory operands (the weight
// gradient) and an A operand in tensor memory (the convolution). For the last
// two, both candidate conventions are tried (every address either one forms
// stays inside the self-test's buffers); the one that reproduces the product
// is used by the kernels.
std::mutex g_selftest_mu;
int g_selftest_state[64] = {0};  // 0 = not run, 1 = pass, -1 = fail
int g_mn_swap[64] = {0};
int g_apack[64] = {0};

bool product_matches(const std::vector<float>& A, const std::vector<float>& Bm, const std::vector<float>& D) {
  for (int m = 0; m < 128; ++m)
    for (int n = 0; n < 32; ++n) {
      double s = 0.0;
      for (int k = 0; k < 32; ++k) s += static_cast<double>(A[m * 32 + k]) * Bm[n * 32 + k];
      if (std::fabs(s - D[m * 32 + n]) > 1e-3 * (1.0 + std::fabs(s))) return false;
    }
  return true;
}

sim_status selftest_run(int mode, int mn_swap, const std::vector<float>& A, const std::vector<float>& Bm,
                        std::vector<float>& D) {
  float *da = nullptr, *db = nullptr, *dd = nullptr;
  cudaError_t e = cudaMalloc(&da, 128 * 32 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&db, 32 * 32 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&dd, 128 * 32 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(da, A.data(), 128 * 32 * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(db, Bm.data(), 32 * 32 * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = selftest_mma(da, db, dd, mode, mn_swap);
  cudaError_t e2 = cudaSuccess;
  if (e == cudaSuccess) e2 = cudaMemcpy(D.data(), dd, 128 * 32 * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(da);
  cudaFree(db);
  cudaFree(dd);
  if (e == cudaErrorTimeout) return SIM_E_TIMEOUT;
  if (e != cudaSuccess || e2 != cudaSuccess) return SIM_E_CUDA;
  return SIM_OK;
}

sim_status run_selftest(sur_h h) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_selftest_mu);
  const bool slot_ok = dev >= 0 && dev < 64;
  if (slot_ok && g_selftest_state[dev] == 1) {
    if (h) {
      h->mn_swap = g_mn_swap[dev];
      h->apack = g_apack[dev];
    }
    return SIM_OK;
  }
  if (slot_ok && g_selftest_state[dev] == -1)
    return fail(h, SIM_E_CUDA, "tensor-core self-test failed earlier on this device");
  std::vector<float> A(128 * 32), Bm(32 * 32), D(128 * 32);
  for (int i = 0; i < 128 * 32; ++i) A[i] = static_cast<float>(((i * 37) % 17) - 8) * 0.125f;
  for (int i = 0; i < 32 * 32; ++i) Bm[i] = static_cast<float>(((i * 11) % 13) - 6) * 0.25f;
  sim_status st = selftest_run(0, 0, A, Bm, D);
  if (st != SIM_OK || !product_matches(A, Bm, D)) {
    if (slot_ok) g_selftest_state[dev] = -1;
    return fail(h, SIM_E_CUDA, "tensor-core self-test failed: K-major UMMA result mismatch");
  }
  int found[3] = {0, -1, -1};
  for (int mode = 1; mode <= 2; ++mode)
    for (int o = 0; o < 2 && found[mode] < 0; ++o) {
      st = selftest_run(mode, o, A, Bm, D);
      if (st == SIM_OK && product_matches(A, Bm, D)) found[mode] = o;
    }
  if (found[1] < 0 || found[2] < 0) {
    if (slot_ok) g_selftest_state[dev] = -1;
    return fail(h, SIM_E_CUDA, found[1] < 0 ? "tensor-core self-test failed: MN-major UMMA result mismatch"
                                            : "tensor-core self-test failed: tensor-memory A operand mismatch");
  }
  if (slot_ok) {
    g_selftest_state[dev] = 1;
    g_mn_swap[dev] = found[1];
    g_apack[dev] = found[2];
  }
  if (h) {
    h->mn_swap = found[1];
    h->apack = found[2];
  }
  return SIM_OK;
}

sim_status check_err(sur_h h, const char* where) {
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, where);
  int v = 0;
  e = cudaMemcpy(&v, h->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, where);
  if (v) {
    cudaMemset(h->err, 0, sizeof(int));
    if (v & kErrTimeout) return fail(h, SIM_E_TIMEOUT, std::string(where) + ": tensor-core pipeline wait timed out");
    if (v & kErrDomain) return fail(h, SIM_E_DOMAIN, std::string(where) + ": particle stencil leaves the grid");
    return fail(h, SIM_E_ARG, std::string(where) + ": material index out of range");
  }
  return SIM_OK;
}

cudaError_t conv(sur_h h, const __nv_bfloat16* in, __nv_bfloat16* out, const __nv_bfloat16* w, const float* bias,
                 const __nv_bfloat16* add, const __nv_bfloat16* mask, int relu, int batch) {
  Prof pr(h, "sur_conv3_umma");
  ConvArgs a{in, out, w, bias, add, mask, relu, h->apack, h->g, batch, h->err};
  h->launches += 1;
  return launch_conv(a, h->num_sms, h->stream);
}

cudaError_t ensure_weights(sur_h h) {
  if (!h->dirty) return cudaSuccess;
  Prof pr(h, "sur_prep_weights");
  h->launches += 1;
  cudaError_t e = launch_prep_weights(h->params, h->B, h->wf, h->wb, h->stream);
  if (e == cudaSuccess) h->dirty = false;
  return e;
}

cudaError_t forward(sur_h h, int batch, const uint16_t* frames, const int* idx) {
  cudaError_t e = ensure_weights(h);
  if (e != cudaSuccess) return e;
  {
    Prof pr(h, "sur_lift");
    h->launches += 1;
    e = launch_lift(h->g, batch, frames, idx, h->params, h->params + 256, h->h[0], h->stream);
  }
  for (int b = 0; e == cudaSuccess && b < h->B; ++b) {
    const size_t L1 = static_cast<size_t>(2 * b) * kConvWElems, L2 = L1 + kConvWElems;
    e = conv(h, h->h[b], h->r[b], h->wf + L1, h->params + w1_off(b) + 27 * 1024, nullptr, nullptr, 1, batch);
    if (e == cudaSuccess)
      e = conv(h, h->r[b], h->h[b + 1], h->wf + L2, h->params + w2_off(b) + 27 * 1024, h->h[b], nullptr, 0,
               batch);
  }
  return e;
}

// Reverse pass of the last forward. With g_pred_in == null: the MSE loss
// against frames[tgt] (loss sum in dsum[0]) and the parameter gradient in
// h->grad; otherwise the caller's dL/dpred and only the input gradient (no
// weight gradients). g_frames (nullable) receives dL/dframe.
cudaError_t backward(sur_h h, int batch, const uint16_t* frames, const int* idx, const int* tgt, float* g_frames,
                     const float* g_pred_in = nullptr) {
  const bool params = g_pred_in == nullptr;
  cudaError_t e = cudaMemsetAsync(h->grad, 0, h->np * sizeof(float), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->dsum, 0, sizeof(double), h->stream);
  if (e != cudaSuccess) return e;
  const long long po = proj_off(h->B);
  {
    Prof pr(h, "sur_proj");
    h->launches += 1;
    if (params)
      e = launch_proj(h->g, batch, 2, frames, idx, tgt, h->h[h->B], h->params + po, h->params + po + 96, nullptr,
                      h->gh[0], g_frames ? h->gpred : nullptr, h->grad + po, h->dsum, nullptr, h->stream);
    else
      e = launch_proj(h->g, batch, 8, frames, idx, nullptr, h->h[h->B], h->params + po, h->params + po + 96,
                      nullptr, h->gh[0], const_cast<float*>(g_pred_in), nullptr, nullptr, nullptr, h->stream);
  }
  int cur = 0;
  for (int b = h->B - 1; e == cudaSuccess && b >= 0; --b) {
    const size_t L1 = static_cast<size_t>(2 * b) * kConvWElems, L2 = L1 + kConvWElems;
    if (params) {
      Prof pr(h, "sur_wgrad_umma");
      h->launches += 2;
      e = launch_wgrad_umma(h->g, batch, h->r[b], h->gh[cur], h->partial, h->n_part, h->grad + w2_off(b),
                            h->mn_swap, h->err, h->stream);
    }
    if (e == cudaSuccess) e = conv(h, h->gh[cur], h->ga, h->wb + L2, nullptr, nullptr, h->r[b], 0, batch);
    if (e == cudaSuccess && params) {
      Prof pr(h, "sur_wgrad_umma");
      h->launches += 2;
      e = launch_wgrad_umma(h->g, batch, h->h[b], h->ga, h->partial, h->n_part, h->grad + w1_off(b),
                            h->mn_swap, h->err, h->stream);
    }
    if (e == cudaSuccess) e = conv(h, h->ga, h->gh[cur ^ 1], h->wb + L1, nullptr, h->gh[cur], nullptr, 0, batch);
    cur ^= 1;
  }
  if (e == cudaSuccess) {
    Prof pr(h, "sur_lift_bwd");
    h->launches += 1;
    e = launch_lift_bwd(h->g, batch, frames, idx, h->gh[cur], h->params, params ? h->gpred : g_pred_in, h->grad,
                        h->grad + 256, g_frames, h->stream);
  }
  return e;
}

sim_status read_loss(sur_h h, int batch, float* loss, const char* where) {
  sim_status s = check_err(h, where);
  if (s != SIM_OK) return s;
  if (loss) {
    double v = 0.0;
    cudaError_t e = cudaMemcpy(&v, h->dsum, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, where);
    const double count = static_cast<double>(batch) * h->g.n * h->g.n * h->g.n * 3.0;
    *loss = static_cast<float>(v / count);
  }
  return SIM_OK;
}

bool batch_ok(sur_h h, int batch, const uint16_t* frames) {
  return batch >= 1 && batch <= h->cfg.max_batch && frames != nullptr;
}

}  // namespace

extern "C" {

long long sur_param_count(const sur_config* cfg) {
  if (!valid_config(cfg)) return -1;
  return count_params(cfg->channels, cfg->blocks);
}

const char* sur_last_error(sur_h h) {
  if (!h) return "invalid handle";
  return h->last_error.c_str();
}

sim_status sur_destroy(sur_h h) {
  if (!h) return SIM_OK;
  cudaStreamSynchronize(h->stream);
  for (auto& r : h->prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (void* p : h->allocs) cudaFree(p);
  delete h;
  return SIM_OK;
}

sim_status sur_create(const sur_config* cfg, sur_h* out) {
  if (!out) return SIM_E_ARG;
  *out = nullptr;
  if (!valid_config(cfg)) return SIM_E_ARG;
  sur_h h = new mpm_surrogate();
  h->cfg = *cfg;
  h->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  h->B = cfg->blocks;
  h->np = count_params(cfg->channels, cfg->blocks);
  h->g = make_geom(cfg->grid_n, cfg->max_batch);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    sim_status s = cuda_fail(h, e, "sur_create");
    sur_destroy(h);
    return s;
  }
  sim_status st = run_selftest(h);
  if (st != SIM_OK) {
    sur_destroy(h);
    return st;
  }
  const size_t tensor = static_cast<size_t>(4) * h->g.plane * 8;  // BF16 elements
  const long long n3 = static_cast<long long>(cfg->grid_n) * cfg->grid_n * cfg->grid_n;
  h->n_part = h->num_sms;
  bool ok = dalloc(h, &h->params, h->np) && dalloc(h, &h->adam_m, h->np) && dalloc(h, &h->adam_v, h->np) &&
            dalloc(h, &h->grad, h->np) && dalloc(h, &h->wf, static_cast<size_t>(2 * h->B) * kConvWElems) &&
            dalloc(h, &h->wb, static_cast<size_t>(2 * h->B) * kConvWElems) &&
            dalloc(h, &h->gpred, static_cast<size_t>(cfg->max_batch) * n3 * 3) &&
            dalloc(h, &h->partial, static_cast<size_t>(h->n_part) * (27 * 1024 + 32)) &&
            dalloc(h, &h->feat_acc, static_cast<size_t>(n3) * 8) &&
            dalloc(h, &h->dsum, 1 + 2 * static_cast<size_t>(cfg->max_batch)) && dalloc(h, &h->err, 1);
  h->h.assign(h->B + 1, nullptr);
  h->r.assign(h->B, nullptr);
  for (int i = 0; ok && i <= h->B; ++i) ok = dalloc(h, &h->h[i], tensor);
  for (int i = 0; ok && i < h->B; ++i) ok = dalloc(h, &h->r[i], tensor);
  ok = ok && dalloc(h, &h->gh[0], tensor) && dalloc(h, &h->gh[1], tensor) && dalloc(h, &h->ga, tensor);
  if (!ok) {
    sur_destroy(h);
    return SIM_E_OOM;
  }
  // zero everything once: the halo rows of every activation tensor stay zero
  e = cudaSuccess;
  auto z = [&](void* p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, bytes, h->stream);
  };
  z(h->params, h->np * 4);
  z(h->adam_m, h->np * 4);
  z(h->adam_v, h->np * 4);
  z(h->grad, h->np * 4);
  z(h->feat_acc, static_cast<size_t>(n3) * 32);
  z(h->wf, static_cast<size_t>(2 * h->B) * kConvWElems * 2);  // the zero rows of the A layout
  z(h->wb, static_cast<size_t>(2 * h->B) * kConvWElems * 2);
  z(h->err, 4);
  for (auto* p : h->h) z(p, tensor * 2);
  for (auto* p : h->r) z(p, tensor * 2);
  z(h->gh[0], tensor * 2);
  z(h->gh[1], tensor * 2);
  z(h->ga, tensor * 2);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    sim_status s = cuda_fail(h, e, "sur_create");
    sur_destroy(h);
    return s;
  }
  *out = h;
  return SIM_OK;
}

sim_status sur_set_params(sur_h h, const float* params, int on_device) {
  if (!h || !params) return h ? fail(h, SIM_E_ARG, "sur_set_params: null pointer") : SIM_E_ARG;
  cudaError_t e = cudaMemcpyAsync(h->params, params, h->np * sizeof(float),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->adam_m, 0, h->np * sizeof(float), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->adam_v, 0, h->np * sizeof(float), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sur_set_params");
  h->t = 0;
  h->dirty = true;
  return SIM_OK;
}

sim_status sur_get_params(sur_h h, float* params, int on_device) {
  if (!h || !params) return h ? fail(h, SIM_E_ARG, "sur_get_params: null pointer") : SIM_E_ARG;
  cudaError_t e = cudaMemcpyAsync(params, h->params, h->np * sizeof(float),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sur_get_params");
  return SIM_OK;
}

static sim_status feat_args(sur_h h, int n_particles, const float* material_mass, int n_materials, FeatArgs* a) {
  if (n_particles < 0 || !material_mass || n_materials < 1 || n_materials > 8)
    return fail(h, SIM_E_ARG, "sur_features: bad particle count or materials");
  a->n = h->cfg.grid_n;
  a->N = n_particles;
  a->n_mat = n_materials;
  for (int i = 0; i < 8; ++i) a->mmass[i] = i < n_materials ? material_mass[i] : 0.0f;
  a->inv_mref = 1.0f / h->cfg.m_ref;
  a->inv_mvref = 1.0f / (h->cfg.m_ref * h->cfg.v_ref);
  return SIM_OK;
}

sim_status sur_features(sur_h h, int n_particles, const float* x, const float* v, const float* C,
                        const uint8_t* mat, const float* material_mass, int n_materials, uint16_t* frame) {
  if (!h) return SIM_E_ARG;
  FeatArgs a;
  sim_status s = feat_args(h, n_particles, material_mass, n_materials, &a);
  if (s != SIM_OK) return s;
  if (!frame || (n_particles > 0 && (!x || !v || !C || !mat)))
    return fail(h, SIM_E_ARG, "sur_features: null pointer");
  cudaError_t e;
  {
    Prof pr(h, "sur_features");
    h->launches += 2;
    e = launch_features(a, x, v, C, mat, h->feat_acc, frame, h->err, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "sur_features");
  return check_err(h, "sur_features");
}

sim_status sur_features_vjp(sur_h h, int n_particles, const float* x, const float* v, const float* C,
                            const uint8_t* mat, const float* material_mass, int n_materials, const float* g_frame,
                            float* dLdx, float* dLdv, float* dLdC) {
  if (!h) return SIM_E_ARG;
  FeatArgs a;
  sim_status s = feat_args(h, n_particles, material_mass, n_materials, &a);
  if (s != SIM_OK) return s;
  if (n_particles > 0 && (!x || !mat || !g_frame)) return fail(h, SIM_E_ARG, "sur_features_vjp: null pointer");
  cudaError_t e;
  {
    Prof pr(h, "sur_features_vjp");
    h->launches += 1;
    e = launch_features_vjp(a, x, v, C, mat, g_frame, dLdx, dLdv, dLdC, h->err, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "sur_features_vjp");
  return check_err(h, "sur_features_vjp");
}

sim_status sur_predict(sur_h h, int batch, const uint16_t* frames, const int* idx, float* pred) {
  if (!h) return SIM_E_ARG;
  if (!batch_ok(h, batch, frames) || !pred) return fail(h, SIM_E_ARG, "sur_predict: bad batch or null pointer");
  cudaError_t e = forward(h, batch, frames, idx);
  if (e == cudaSuccess) {
    Prof pr(h, "sur_proj");
    h->launches += 1;
    const long long po = proj_off(h->B);
    e = launch_proj(h->g, batch, 1, frames, idx, nullptr, h->h[h->B], h->params + po, h->params + po + 96, pred,
                    nullptr, nullptr, nullptr, nullptr, nullptr, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "sur_predict");
  return check_err(h, "sur_predict");
}

sim_status sur_loss_grad(sur_h h, int batch, const uint16_t* frames, const int* idx, const int* tgt, float* loss,
                         float* grad, float* g_frames) {
  if (!h) return SIM_E_ARG;
  if (!batch_ok(h, batch, frames) || !tgt) return fail(h, SIM_E_ARG, "sur_loss_grad: bad batch or null pointer");
  cudaError_t e = forward(h, batch, frames, idx);
  if (e == cudaSuccess) e = backward(h, batch, frames, idx, tgt, g_frames);
  if (e == cudaSuccess && grad)
    e = cudaMemcpyAsync(grad, h->grad, h->np * sizeof(float), cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sur_loss_grad");
  return read_loss(h, batch, loss, "sur_loss_grad");
}

sim_status sur_vjp(sur_h h, int batch, const uint16_t* frames, const int* idx, const float* g_pred,
                   float* g_frames) {
  if (!h) return SIM_E_ARG;
  if (!batch_ok(h, batch, frames) || !g_pred || !g_frames)
    return fail(h, SIM_E_ARG, "sur_vjp: bad batch or null pointer");
  cudaError_t e = forward(h, batch, frames, idx);
  if (e == cudaSuccess) e = backward(h, batch, frames, idx, nullptr, g_frames, g_pred);
  if (e != cudaSuccess) return cuda_fail(h, e, "sur_vjp");
  return check_err(h, "sur_vjp");
}

sim_status sur_train_step(sur_h h, int batch, const uint16_t* frames, const int* idx, const int* tgt, float lr,
                          float* loss) {
  if (!h) return SIM_E_ARG;
  if (!batch_ok(h, batch, frames) || !tgt || !(lr >= 0.0f))
    return fail(h, SIM_E_ARG, "sur_train_step: bad batch, learning rate or null pointer");
  cudaError_t e = forward(h, batch, frames, idx);
  if (e == cudaSuccess) e = backward(h, batch, frames, idx, tgt, nullptr);
  if (e == cudaSuccess) {
    Prof pr(h, "sur_adam");
    h->launches += 1;
    h->t += 1;
    e = launch_adam(h->params, h->grad, h->adam_m, h->adam_v, h->np, lr, h->cfg.adam_beta1, h->cfg.adam_beta2,
                    h->cfg.adam_eps, h->t, h->stream);
    h->dirty = true;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "sur_train_step");
  return read_loss(h, batch, loss, "sur_train_step");
}

sim_status sur_eval(sur_h h, int batch, const uint16_t* frames, const int* idx, const int* tgt, double* err2) {
  if (!h) return SIM_E_ARG;
  if (!batch_ok(h, batch, frames) || !tgt || !err2) return fail(h, SIM_E_ARG, "sur_eval: bad batch or null pointer");
  cudaError_t e = cudaMemsetAsync(h->dsum, 0, (1 + 2 * static_cast<size_t>(batch)) * sizeof(double), h->stream);
  if (e == cudaSuccess) e = forward(h, batch, frames, idx);
  if (e == cudaSuccess) {
    Prof pr(h, "sur_proj");
    h->launches += 1;
    const long long po = proj_off(h->B);
    e = launch_proj(h->g, batch, 4, frames, idx, tgt, h->h[h->B], h->params + po, h->params + po + 96, nullptr,
                    nullptr, nullptr, nullptr, nullptr, h->dsum + 1, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "sur_eval");
  sim_status s = check_err(h, "sur_eval");
  if (s != SIM_OK) return s;
  e = cudaMemcpy(err2, h->dsum + 1, 2 * static_cast<size_t>(batch) * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "sur_eval");
  return SIM_OK;
}

sim_status sur_profile_enable(sur_h h, int enable) {
  if (!h) return SIM_E_ARG;
  cudaStreamSynchronize(h->stream);
  for (auto& r : h->prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  h->prof_recs.clear();
  h->prof = enable != 0;
  return SIM_OK;
}

sim_status sur_profile_read(sur_h h, int cap, const char** names, double* total_ms, long long* launches,
                            int* n_out) {
  if (!h || !n_out) return SIM_E_ARG;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sur_profile_read");
  std::vector<const char*> nm;
  std::vector<double> ms;
  std::vector<long long> ct;
  for (auto& r : h->prof_recs) {
    float t = 0.0f;
    cudaEventElapsedTime(&t, r.a, r.b);
    size_t i = 0;
    for (; i < nm.size(); ++i)
      if (std::strcmp(nm[i], r.name) == 0) break;
    if (i == nm.size()) {
      nm.push_back(r.name);
      ms.push_back(0.0);
      ct.push_back(0);
    }
    ms[i] += t;
    ct[i] += 1;
  }
  *n_out = static_cast<int>(nm.size());
  for (int i = 0; i < cap && i < static_cast<int>(nm.size()); ++i) {
    if (names) names[i] = nm[i];
    if (total_ms) total_ms[i] = ms[i];
    if (launches) launches[i] = ct[i];
  }
  return SIM_OK;
}

long long sur_kernel_launches(sur_h h) { return h ? h->launches : -1; }

sim_status sur_selftest_mma(const float* a, const float* b, float* d, int mode) {
  if (!a || !b || !d || mode < 0 || mode > 2) return SIM_E_ARG;
  int opt = 0;
  if (mode >= 1) {
    sim_status st = run_selftest(nullptr);
    if (st != SIM_OK) return st;
    int dev = 0;
    cudaGetDevice(&dev);
    opt = (dev >= 0 && dev < 64) ? (mode == 1 ? g_mn_swap[dev] : g_apack[dev]) : 0;
  }
  std::vector<float> A(a, a + 128 * 32), Bm(b, b + 32 * 32), D(128 * 32);
  sim_status st = selftest_run(mode, opt, A, Bm, D);
  if (st != SIM_OK) return st;
  std::memcpy(d, D.data(), D.size() * sizeof(float));
  return SIM_OK;
}

long long sur_mn_major_swap(void) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_selftest_mu);
  if (dev < 0 || dev >= 64 || g_selftest_state[dev] != 1) return -1;
  return g_mn_swap[dev] | (g_apack[dev] << 1);
}

}  // extern "C"
