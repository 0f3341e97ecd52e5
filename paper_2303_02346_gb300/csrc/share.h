// Host-side launchers of the neighbour kernels: gradient sharing and the
// attraction loss (paper Sec. 5.1). Internal interface between the C-ABI
// implementation and kern_share.cu / kern_misc.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"

namespace mpm {

// Cell bins of the particles at their current positions, without moving
// them: key[p] = (scene, Morton code of the stencil-origin cell), rank[p] =
// position of p among the particles of its key, bins = exclusive prefix of
// the key counts (start of each key; a key's end is the next key's start,
// or N for the last key). Uses the sort buffers.
void launch_bin(const Params& P, const float* st, const uint32_t* tag, SortBuffers sb, cudaStream_t s);

// Neighbour arrays in bin order. pk[slot] = (x, c) with c = exp(-ell[q] /
// tau) for caller index q = pid[p] - lo in [0, cnt), else c = -1 (particle
// not addressed); sidx[slot] = p; pg[slot] = (g[q], 0) if g is given.
struct NbrBuffers {
  float4* pk;
  float4* pg;
  int* sidx;
};
void launch_nbr_pack(const Params& P, const float* st, const int* pid, const SortBuffers& sb, const float* ell,
                     const float* g, int lo, int cnt, float tau, NbrBuffers nb, cudaStream_t s);

// Attraction loss: adds weight * dL_att/dx to the x fields of adj (library
// order) and weight * L_att to *loss.
void launch_attraction(const Params& P, const uint32_t* tag, const SortBuffers& sb, NbrBuffers nb, float radius,
                       float weight, float* adj, double* loss, cudaStream_t s);

// Gradient sharing: out[q] = sum_j c_j k(d / radius) g_j (caller order).
void launch_share(const Params& P, const uint32_t* tag, const int* pid, const SortBuffers& sb, NbrBuffers nb,
                  float radius, int lo, float* out, cudaStream_t s);

}  // namespace mpm
