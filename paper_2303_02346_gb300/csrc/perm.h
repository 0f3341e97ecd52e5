// Host-side launcher of the adjoint state's re-ordering between checkpoint
// orders (implemented in kern_misc.cu).
#pragma once

#include <cuda_runtime.h>

namespace mpm {

// dst[f][p'] = src[f][p] with pid_to[p'] = pid_from[p] (the same caller
// particle), for `fields` SoA fields of N particles; inv (N ints) is scratch.
// One inverse-permutation pass and one gather pass over the fields.
void launch_permute_state(const float* src, float* dst, const int* pid_from, const int* pid_to, int* inv, int N,
                          int fields, cudaStream_t s);

}  // namespace mpm
