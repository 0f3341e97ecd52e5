// Device-side layout and launchers of the surrogate network (include/mpm_surrogate.h).
//
// Activation tensors (C = 32 channels, BF16) live in a zero-padded,
// channel-planar layout built for the implicit-GEMM convolution:
//   row(b, i, j, k) = G + b * V + ((i + 1) * P1 + (j + 1)) * P1 + (k + 1),
//   P1 = n + 2, P2 = P1^2, V = P1^3 rows per frame, G guard rows at both ends;
//   element (row, ch) at t[((ch / 8) * plane + row) * 8 + ch % 8],
//   plane = 2 G + max_batch * V rows.
// A 3x3x3 tap (a, b, c) is then the constant row offset (a-1) P2 + (b-1) P1 +
// (c-1), so the A operand of every tap is a run of consecutive rows: one
// 16-byte row per node and channel group, which is exactly the row of an
// 8 x 16-byte UMMA core matrix. Halo rows (i, j or k outside 1..n) are zero
// and never written; outputs at halo rows are computed and discarded.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace sur {

constexpr int kC = 32;          // hidden channels (the tensor-core kernels are specialised for 32)
constexpr int kCin = 8;         // frame channels
constexpr int kTile = 128;      // output rows per UMMA tile (M)
constexpr int kTaps = 27;
// convolution tiling (sur_conv.cu): 126 output rows per tile from N = 128
// input rows, marching 8 planes per work item; weights as the UMMA A operand
// (loaded into tensor memory): [128 rows (c, o), rows 96..127 zero][9 tap
// pairs (a, b)][32 input channels]
constexpr int kConvW = 126;
constexpr int kConvN = 128;
constexpr int kConvChunk = 8;
constexpr int kConvWElems = 9 * 4 * 128 * 8;
constexpr int kConvWBytes = kConvWElems * 2;

enum ErrBits { kErrTimeout = 1, kErrDomain = 2, kErrArg = 4 };

struct SurGeom {
  int n, P1, P2;
  long long V;      // rows per frame
  int G;            // guard rows before the first and after the last frame
  long long plane;  // rows per channel plane
};

inline SurGeom make_geom(int n, int max_batch) {
  SurGeom g;
  g.n = n;
  g.P1 = n + 2;
  g.P2 = g.P1 * g.P1;
  g.V = static_cast<long long>(g.P2) * g.P1;
  g.G = ((kTile + g.P1 + 1) + 7) / 8 * 8;
  g.plane = 2ll * g.G + static_cast<long long>(max_batch) * g.V;
  return g;
}

__host__ __device__ inline long long pad_row(const SurGeom& g, int b, int i, int j, int k) {
  return g.G + b * g.V + (static_cast<long long>(i + 1) * g.P1 + (j + 1)) * g.P1 + (k + 1);
}

size_t conv_smem_bytes(const SurGeom& g);

struct ConvArgs {
  const __nv_bfloat16* in;    // activation tensor (layout above)
  __nv_bfloat16* out;         // written at interior rows only
  const __nv_bfloat16* w;     // kConvWElems, the A layout above
  const float* bias;          // [32] or null
  const __nv_bfloat16* add;   // residual added before rounding, or null
  const __nv_bfloat16* mask;  // out = mask > 0 ? out : 0 (relu derivative), or null
  int relu;
  int apack;                  // BF16 pair order of A in tensor memory (self-test)
  SurGeom g;
  int batch;
  int* err;
};

// Feature transfer arguments.
struct FeatArgs {
  int n, N, n_mat;
  float mmass[8];
  float inv_mref, inv_mvref;
};

// launchers (return the cudaError of the launch)
cudaError_t launch_conv(const ConvArgs& a, int num_sms, cudaStream_t st);
// D = A B^T on the tensor cores (device pointers); mode 0 K-major operands,
// mode 1 MN-major operands with descriptor offset assignment `opt`, mode 2 A
// in tensor memory with BF16 pair order `opt`
cudaError_t selftest_mma(const float* a, const float* b, float* d, int mode, int opt);

cudaError_t launch_prep_weights(const float* params, int blocks, __nv_bfloat16* wf, __nv_bfloat16* wb,
                                cudaStream_t st);
cudaError_t launch_lift(const SurGeom& g, int batch, const uint16_t* frames, const int* idx,
                        const float* w_lift, const float* b_lift, __nv_bfloat16* h0, cudaStream_t st);
// mode bit 1: write pred; bit 2: loss (*loss_acc += sum of squares) and
// gradients; bit 4: per-frame error sums frame_sums[2b], [2b+1]; mode 8 alone:
// dL/dh from a caller-supplied dL/dpred (g_pred, read)
cudaError_t launch_proj(const SurGeom& g, int batch, int mode, const uint16_t* frames, const int* idx,
                        const int* tgt, const __nv_bfloat16* h, const float* w_proj, const float* b_proj,
                        float* pred, __nv_bfloat16* g_h, float* g_pred, float* grad_wp, double* loss_acc,
                        double* frame_sums, cudaStream_t st);
// weight + bias gradient of one conv layer on the tensor cores; grad_wb = the
// layer's weights followed by its bias in the flat gradient (overwritten);
// partial: max_ctas x (27 * 1024 + 32) floats
cudaError_t launch_wgrad_umma(const SurGeom& g, int batch, const __nv_bfloat16* x, const __nv_bfloat16* gy,
                              float* partial, int max_ctas, float* grad_wb, int mn_swap, int* err,
                              cudaStream_t st);
int wgrad_stage_rows(const SurGeom& g);
size_t wgrad_smem_bytes(const SurGeom& g);
cudaError_t launch_lift_bwd(const SurGeom& g, int batch, const uint16_t* frames, const int* idx,
                            const __nv_bfloat16* g_h0, const float* w_lift, const float* g_pred,
                            float* grad_wl, float* grad_bl, float* g_frames, cudaStream_t st);
cudaError_t launch_adam(float* p, const float* grad, float* m, float* v, long long count, float lr,
                        float beta1, float beta2, float eps, int t, cudaStream_t st);
cudaError_t launch_features(const FeatArgs& a, const float* x, const float* v, const float* C,
                            const uint8_t* mat, float* acc, uint16_t* frame, int* err, cudaStream_t st);
cudaError_t launch_features_vjp(const FeatArgs& a, const float* x, const float* v, const float* C,
                                const uint8_t* mat, const float* g_frame, float* dLdx, float* dLdv, float* dLdC,
                                int* err, cudaStream_t st);

}  // namespace sur
