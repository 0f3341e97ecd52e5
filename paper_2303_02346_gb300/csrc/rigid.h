// Particle-represented rigid bodies (Sec. 3.2 "Rigid body"): after the G2P of
// every step the particles of each rigid object are fitted by the closest
// rigid motion and set to it; the adjoint of that projection runs before the
// G2P adjoint of the same step. Kernels in kern_rigid.cu.
//
// An object is (scene, rigid material); its index is scene * n_mat + material.
// Per object:
//   sums   S1 = sum m x, S2 = sum m x rbar^T, S3 = sum m v, S4 = sum m v rbar^T
//          (FP64 accumulators)
//   const  M, sbar = sum m rbar, K = I0^{-1} (I0 the rest inertia tensor)
//   record c, R, vbar, w, L, U, sigma, V, S4 of the step (kept per step by the
//          recompute for the adjoint)
// rbar (3 x N floats, caller order) are the rest offsets from the rest
// centroid, taken from the positions passed to sim_set_particles.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace mpm {

constexpr int kRigidConst = 16;   // M, sbar[3], K[9], pad
constexpr int kRigidSums = 24;    // S1[3], S2[9], S3[3], S4[9]
constexpr int kRigidRecord = 52;  // c[3] R[9] vbar[3] w[3] L[3] U[9] sigma[3] V[9] S4[9], pad
constexpr int kRigidGrad = 18;    // adjoint sums: gc[3] gR[9] gvbar[3] gw[3]
// The FP64 accumulators of an object are spread over kRigidReplicas lines of
// kRigidLine doubles (one 256-byte line each); a warp adds to the line picked
// by its index, so that atomics on one address do not serialise the whole
// particle pass. The solve kernels sum the lines and clear them.
constexpr int kRigidReplicas = 32;
constexpr int kRigidLine = 32;

struct RigidBuffers {
  int n_obj = 0;             // scenes x materials
  float* rest = nullptr;     // 3 x N rest offsets (caller order)
  float* cst = nullptr;      // n_obj x kRigidConst
  double* sums = nullptr;    // n_obj x kRigidReplicas x kRigidLine, zero between uses
  float* rec = nullptr;      // n_obj x kRigidRecord (forward scratch)
  double* gsums = nullptr;   // n_obj x kRigidReplicas x kRigidLine, zero between uses
  float* gout = nullptr;     // n_obj x kRigidSums: adjoints of S1..S4
};

// Rest shape of the rigid particles [lo, lo + cnt) of scene `scene` (-1: all
// scenes, [lo, lo + cnt) then covers every particle) from the caller-order
// state X0 (SoA, N stride) and tags: writes rest offsets and the objects'
// constants. 4 launches.
void launch_rigid_rest(const Params& P, const float* X0, const uint32_t* tag0, int scene, int lo, int cnt,
                       RigidBuffers rb, cudaStream_t s);

// Projection of the rigid particles of state `st` (sorted order; pid maps to
// caller order) after G2P; the step's record goes to `rec`. 3 launches.
void launch_rigid_project(const Params& P, float* st, const uint32_t* tag, const int* pid, RigidBuffers rb,
                          float* rec, cudaStream_t s);

// Adjoint of that projection, in place on the adjoint state `adj`, from the
// step's record. 3 launches.
void launch_rigid_adjoint(const Params& P, float* adj, const uint32_t* tag, const int* pid, RigidBuffers rb,
                          const float* rec, cudaStream_t s);

}  // namespace mpm
