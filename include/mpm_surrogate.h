/*
 * mpm_surrogate.h - C-ABI of the learned grid-space surrogate of the MLS-MPM
 * step: a 3D convolutional neural operator that predicts the grid momentum a
 * fixed number of steps ahead from the current grid state, trained on frames
 * the simulator itself generates (the paper points to learned dynamics models
 * as a cheaper differentiable stand-in, Sec. 6).
 *
 * Network (BF16 weights and activations, FP32 accumulation; C = channels,
 * B = residual blocks):
 *   frame f, 8 channels per grid node:  m, p_x, p_y, p_z, phi_0, phi_1, phi_2, 0
 *     m = sum_p W_ip m_p / m_ref, p = sum_p W_ip m_p (v_p + C_p (x_i - x_p)) / (m_ref v_ref)
 *     (the MLS-MPM transfer of Sec. 3.1 without the stress impulse),
 *     phi_k = mass fraction of material k at the node (0 where m = 0)
 *   h_0  = W_l f + b_l                        1x1x1 lift, 8 -> C
 *   r_b  = relu(conv3(h_{b-1}, W1_b) + b1_b)  3x3x3, zero padded, C -> C
 *   h_b  = h_{b-1} + conv3(r_b, W2_b) + b2_b
 *   pred = f[1:4] + W_p h_B + b_p             normalised momentum, steps ahead
 * conv3(h, W)[i,j,k,o] = sum_{a,b,c,q} W[a,b,c,o,q] h[i+a-1, j+b-1, k+c-1, q].
 * Training loss: L = mean over frames, nodes and the 3 components of
 * (pred - target)^2, target = momentum channels of the target frame. Adam
 * (Kingma and Ba 2015) updates an FP32 master copy of the parameters.
 *
 * Rounding points (the only places values are rounded to BF16): the frame,
 * every weight as used, h_b and r_b, and the activation gradients dL/dh_b,
 * dL/da_b (a_b = the pre-activation of r_b) that feed the convolutions.
 *
 * Layouts
 * -------
 * - Frame: n^3 nodes in (i, j, k) row-major order (k fastest, the simulator's
 *   grid order), 8 BF16 channels per node (16 bytes). Frame arrays are
 *   [n_frames][n^3][8]; frames are selected by int32 indices.
 * - Parameters: one flat FP32 vector, in this order: w_lift [C][8], b_lift [C],
 *   per block w1 [3][3][3][C][C] (indexed [a][b][c][out][in]), b1 [C],
 *   w2 [3][3][3][C][C], b2 [C]; then w_proj [3][C], b_proj [3].
 *   sur_param_count() gives its length.
 * - Predictions: FP32 [batch][n^3][3].
 *
 * Conventions: as in mpm_sim.h. Every function returns a sim_status;
 * sur_last_error() describes the last failure. The handle owns its device
 * memory. All array arguments are device pointers on the current device unless
 * stated otherwise; they are only used during the call. Work is enqueued on
 * config.cuda_stream, and every call synchronises that stream before
 * returning. Device-side protocol timeouts of the tensor-core kernels are
 * reported as SIM_E_TIMEOUT.
 */
#ifndef MPM_SURROGATE_H
#define MPM_SURROGATE_H

#include <stdint.h>

#include "mpm_sim.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_surrogate* sur_h;

typedef struct {
    int grid_n;         /* nodes per axis, 8 <= n <= 64 */
    int channels;       /* hidden channels C; the kernels support C = 32 */
    int blocks;         /* residual blocks B, 1..8 */
    int max_batch;      /* frames per call, >= 1 */
    float m_ref;        /* feature normalisation: mass unit */
    float v_ref;        /* feature normalisation: velocity unit */
    float adam_beta1;   /* 0.9 */
    float adam_beta2;   /* 0.999 */
    float adam_eps;     /* 1e-8 */
    void* cuda_stream;  /* cudaStream_t; NULL = legacy default stream */
} sur_config;

/* Length of the flat parameter vector for the configuration (-1 if invalid). */
long long sur_param_count(const sur_config* cfg);

/* Create a handle; allocates the activations for max_batch frames (about
 * 12 x 64 B x max_batch x (n + 2)^3 bytes). Parameters start at zero. */
sim_status sur_create(const sur_config* cfg, sur_h* out);
sim_status sur_destroy(sur_h h);

/* Replace the FP32 master parameters (sur_param_count() floats; on_device
 * selects device or host memory) and reset the Adam moments and step count. */
sim_status sur_set_params(sur_h h, const float* params, int on_device);
sim_status sur_get_params(sur_h h, float* params, int on_device);

/* Grid features of one scene's particle state: x, v [n_particles][3], C
 * [n_particles][3][3] (row-major), mat [n_particles] (material index <
 * n_materials), material_mass (HOST, n_materials floats: the particle mass of
 * each material). Writes one frame (n^3 x 8 BF16). n_materials <= 3 fills
 * phi_0..phi_2. A particle whose stencil leaves the grid: SIM_E_DOMAIN. */
sim_status sur_features(sur_h h, int n_particles, const float* x, const float* v, const float* C,
                        const uint8_t* mat, const float* material_mass, int n_materials,
                        uint16_t* frame);

/* Adjoint of the mass and momentum channels of sur_features for a cotangent
 * g_frame (FP32 [n^3][8]; channels 4..7, the material fractions, are not
 * differentiated): dL/dx, dL/dv [n_particles][3] and dL/dC [n_particles][9]
 * (each nullable, overwritten) of that scene's particles; v and C as given to
 * sur_features (nullable = 0). dL/dv_p = m_p sum_i W_ip g_i[1:4] / (m_ref v_ref). */
sim_status sur_features_vjp(sur_h h, int n_particles, const float* x, const float* v, const float* C,
                            const uint8_t* mat, const float* material_mass, int n_materials,
                            const float* g_frame, float* dLdx, float* dLdv, float* dLdC);

/* Predictions for `batch` frames: frames[idx[b]] (idx NULL = 0..batch-1). */
sim_status sur_predict(sur_h h, int batch, const uint16_t* frames, const int* idx, float* pred);

/* Loss of frames[idx[b]] against the momentum channels of frames[tgt[b]]
 * (HOST *loss), its gradient w.r.t. the flat parameters (grad, nullable,
 * overwritten) and w.r.t. the input frames (g_frames FP32 [batch][n^3][8],
 * nullable, overwritten). */
sim_status sur_loss_grad(sur_h h, int batch, const uint16_t* frames, const int* idx, const int* tgt,
                         float* loss, float* grad, float* g_frames);

/* Vector-Jacobian product of the prediction w.r.t. the input frames: for a
 * cotangent g_pred (FP32 [batch][n^3][3]) on the predictions of
 * frames[idx[b]], writes g_frames (FP32 [batch][n^3][8]) = (d pred / d
 * frame)^T g_pred. No parameter gradient is formed. */
sim_status sur_vjp(sur_h h, int batch, const uint16_t* frames, const int* idx, const float* g_pred,
                   float* g_frames);

/* One training step: loss and gradient as sur_loss_grad, then one Adam update
 * with learning rate lr. *loss (HOST, nullable) receives the loss before the update. */
sim_status sur_train_step(sur_h h, int batch, const uint16_t* frames, const int* idx, const int* tgt,
                          float lr, float* loss);

/* Error sums per frame: err2[2b] = sum (pred - target)^2, err2[2b+1] =
 * sum target^2 over the frame's nodes and components (HOST, 2 x batch
 * doubles); relative L2 = sqrt(err2[2b] / err2[2b+1]). */
sim_status sur_eval(sur_h h, int batch, const uint16_t* frames, const int* idx, const int* tgt,
                    double* err2);

/* Per-kernel CUDA-event timing, as sim_profile_enable / sim_profile_read. */
sim_status sur_profile_enable(sur_h h, int enable);
sim_status sur_profile_read(sur_h h, int cap, const char** names, double* total_ms,
                            long long* launches, int* n_out);
long long sur_kernel_launches(sur_h h);

const char* sur_last_error(sur_h h);

/* Hardware self-test of the tensor-core paths: one CTA computes D = A B^T with
 * tcgen05 (A: 128 x 32, B: 32 x 32, BF16-rounded inputs, FP32 accumulation in
 * tensor memory, two K = 16 steps). mode 0 stages both operands K-major in
 * shared memory, mode 1 both MN-major (the layout of the weight gradient),
 * mode 2 A in tensor memory and B K-major (the layout of the convolution).
 * a, b, d are HOST row-major FP32 arrays; runs on the current device and
 * synchronises. sur_create runs all modes once per process and device and
 * fails if a product is wrong. */
sim_status sur_selftest_mma(const float* a, const float* b, float* d, int mode);

/* Operand conventions the self-test found on the current device (-1 if it has
 * not run or failed): bit 0 = which shared-memory descriptor offset holds the
 * stride between MN-adjacent core matrices of an MN-major operand (0 the
 * leading-dimension offset, 1 the stride-dimension offset); bit 1 = which half
 * of a 32-bit tensor-memory column holds the even K element of an A operand
 * (0 the low half, 1 the high half). */
long long sur_mn_major_swap(void);

#ifdef __cplusplus
}
#endif

#endif /* MPM_SURROGATE_H */
