// Grid-mass loss and its particle gradient for callers that cannot allocate
// device memory.
//
// sim_grid_mass_loss works through a simulation handle, and the handle (and
// that call, on first use) obtains its buffers with cudaMalloc. Some callers
// cannot do that: an application that has handed all device memory to its own
// pool and forbids libraries from allocating, a hard real-time control loop
// that must not enter the driver's allocator (cudaMalloc can block and
// synchronise the device), or a process running under a fixed device-memory
// cap. sim_grid_mass_loss_static serves them: the caller passes every input and
// output buffer, and the only working memory is the file-scope array below,
// which exists on every device that loads this library until the process
// exits (2 MiB + 256 B).
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "mpm_sim.h"

using namespace mpm;

namespace {

constexpr int kStaticMaxGrid = 64;
constexpr long long kStaticNodes = (long long)kStaticMaxGrid * kStaticMaxGrid * kStaticMaxGrid;
constexpr int kMaxDevices = 64;

// Working memory shared by every call on a device:
//   [0, kStaticNodes)              P2G mass field
//   [kStaticNodes, 2 kStaticNodes) dL/dm per node
//   [2 kStaticNodes, + 2 floats)   loss accumulator (one double)
static __device__ __align__(256) float g_static_scratch[2 * kStaticNodes + 64];

// Device address of g_static_scratch per device (host code cannot use the
// symbol itself as a device pointer), looked up once per device; the header
// excludes use across a cudaDeviceReset, which may move the array.
float* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_lock;

sim_status scratch_for_current_device(float** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SIM_E_CUDA;
  }
  std::lock_guard<std::mutex> guard(g_scratch_lock);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return SIM_E_CUDA;
    }
    g_scratch_addr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_addr[dev];
  return SIM_OK;
}

Params grid_params(int n) {
  Params P{};
  P.n = n;
  P.dx = 1.0f / n;
  P.inv_dx = float(n);
  return P;
}

__global__ void st_clear(float* __restrict__ scr, long long n3) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n3) scr[i] = 0.0f;
  if (i == 0) *reinterpret_cast<double*>(scr + 2 * kStaticNodes) = 0.0;
}

__global__ void st_scatter(const float* __restrict__ x, const float* __restrict__ mass, int N, Params P,
                           float* __restrict__ scr) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  float xp[3] = {x[3 * (long long)p], x[3 * (long long)p + 1], x[3 * (long long)p + 2]};
  Stencil s;
  make_stencil(xp, P, s);
  float m = mass[p];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) {
        long long idx = ((long long)(s.base[0] + a) * P.n + s.base[1] + b) * P.n + s.base[2] + c;
        atomicAdd(scr + idx, m * s.w[0][a] * s.w[1][b] * s.w[2][c]);
      }
}

__global__ void st_nodes(float* __restrict__ scr, long long n3, const float* __restrict__ tm,
                         const float* __restrict__ td, float inv_M) {
  __shared__ double ws[32];
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < n3) {
    double m = scr[i], d = m - (double)tm[i];
    l = d * d * (double)inv_M * inv_M + m * (double)td[i] * inv_M;
    scr[kStaticNodes + i] = float(2.0 * d * inv_M * inv_M + (double)td[i] * inv_M);
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if (lane == 0) ws[wid] = l;
  __syncthreads();
  if (wid == 0) {
    double s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && s != 0.0) atomicAdd(reinterpret_cast<double*>(scr + 2 * kStaticNodes), s);
  }
}

__global__ void st_grad(const float* __restrict__ x, const float* __restrict__ mass, int N, Params P,
                        const float* __restrict__ scr, float* __restrict__ dLdx) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  float xp[3] = {x[3 * (long long)p], x[3 * (long long)p + 1], x[3 * (long long)p + 2]};
  Stencil s;
  make_stencil(xp, P, s);
  float m = mass[p];
  float g[3] = {0.f, 0.f, 0.f};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) {
        long long idx = ((long long)(s.base[0] + a) * P.n + s.base[1] + b) * P.n + s.base[2] + c;
        float gm = scr[kStaticNodes + idx] * m * P.inv_dx;
        g[0] += gm * s.dw[0][a] * s.w[1][b] * s.w[2][c];
        g[1] += gm * s.w[0][a] * s.dw[1][b] * s.w[2][c];
        g[2] += gm * s.w[0][a] * s.w[1][b] * s.dw[2][c];
      }
  for (int d = 0; d < 3; ++d) dLdx[3 * (long long)p + d] = g[d];
}

__global__ void st_finish(const float* __restrict__ scr, double* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *loss = *reinterpret_cast<const double*>(scr + 2 * kStaticNodes);
}

}  // namespace

extern "C" sim_status sim_grid_mass_loss_static(const float* x, const float* mass, int n_particles,
                                                int grid_n, const float* target_mass,
                                                const float* target_dist, float total_mass, float* dLdx,
                                                double* loss, void* cuda_stream) {
  if (grid_n < 4 || grid_n > kStaticMaxGrid || n_particles < 0 || !(total_mass > 0.0f) || !target_mass ||
      !target_dist || !loss || (n_particles > 0 && (!x || !mass || !dLdx)))
    return SIM_E_ARG;
  // an error left by earlier, unrelated work stays with its owner: report it
  // without consuming it and launch nothing, so that the error check after the
  // launches below sees only this call's launches
  if (cudaPeekAtLastError() != cudaSuccess) return SIM_E_CUDA;
  float* scr = nullptr;
  sim_status st = scratch_for_current_device(&scr);
  if (st != SIM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const long long n3 = (long long)grid_n * grid_n * grid_n;
  const Params P = grid_params(grid_n);
  const int nb_nodes = int((n3 + 255) / 256);
  const int nb_part = (n_particles + 255) / 256;
  st_clear<<<nb_nodes, 256, 0, s>>>(scr, n3);
  if (n_particles > 0) st_scatter<<<nb_part, 256, 0, s>>>(x, mass, n_particles, P, scr);
  st_nodes<<<nb_nodes, 256, 0, s>>>(scr, n3, target_mass, target_dist, 1.0f / total_mass);
  if (n_particles > 0) st_grad<<<nb_part, 256, 0, s>>>(x, mass, n_particles, P, scr, dLdx);
  st_finish<<<1, 32, 0, s>>>(scr, loss);
  if (cudaGetLastError() != cudaSuccess) return SIM_E_CUDA;
  return SIM_OK;
}
