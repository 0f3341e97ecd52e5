// Host implementation of the C-ABI in include/mpm_sim.h.
//
// Device memory layout (all owned by the handle, allocated in sim_create):
//   X0        caller-order initial state (24 x N floats SoA) + tags
//   W, W2     working particle state (24 x N SoA) and its sort double buffer
//   tag/pid   per-order particle tags (material | scene << 8) and caller ids
//   Fp        projected deformation gradients of solids (9 x N), P2G -> G2P
//   acc, gv   dense block-major-addressed grids, float4 per node (S x n^3)
//   flags/list/count  active grid blocks of the current step
// Gradient mode (checkpoint_every = k > 0) adds:
//   CK[c]     checkpoint c = state, tags and caller ids at step c*k, taken right
//             after the particles are re-sorted into grid blocks
//   chunk     k states of the chunk being recomputed in the backward sweep
//   gv/gstore per step of the chunk (grid velocity after / before contact)
//   Fp/svd    per step of the chunk: projected F and the SVD of the trial F of
//             solid particles, so the adjoint kernels need no SVD
//   adj       adjoint state (24 x N), gadj_v / gadj_m adjoint grids
//   seeds     per seeded step t: loss gradients w.r.t. x, v and C of the state
//             at step t (15 x N), added into adj when the sweep reaches t
// Paper App. A: only one state per caching step is kept; the backward pass
// restores it and recomputes the local chunk before back-propagating through it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "kernels.h"
#include "perm.h"
#include "rigid.h"
#include "share.h"
#include "mpm_sim.h"

using namespace mpm;

namespace {

const char* kVersion = "mpm_sim 1.0 (sm_103a)";
constexpr int kMaxBuffers = 20;  // chunk buffers of the recompute pipeline (bits of the overflow word)

struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
  int units;  // launches the record stands for (a persistent run: its steps)
};

}  // namespace

struct mpm_sim {
  sim_config cfg;
  std::vector<int> counts, offsets;
  Params P;
  Tuning tu;  // launch shapes (sim_autotune)
  cudaStream_t stream = nullptr;
  int N = 0, S = 0, n = 0;
  long long n3tot = 0, nflags = 0;
  int k = 0, n_ckpt = 0, max_steps = 0, spa = 10;
  int resort = 8;
  int n_act_max = 1, n_actions = 0;

  float *X0 = nullptr, *W = nullptr, *W2 = nullptr, *Fp = nullptr;
  uint32_t *tag0 = nullptr, *tagA = nullptr, *tagB = nullptr, *tag_cur = nullptr;
  int *pidA = nullptr, *pidB = nullptr, *pid_cur = nullptr;
  float4 *acc = nullptr, *gv = nullptr;
  int* flags = nullptr;
  int *list = nullptr, *count = nullptr;  // two lists/counters, alternating by step parity
  // persistent forward runs: tile counters (2) and grid-barrier words (2)
  int* tile_ctr = nullptr;
  unsigned* bar = nullptr;
  int* nwater = nullptr;  // device count of water particles (set_particles)
  bool coop = false;  // the device supports cooperative launches
  // tensor maps of the grid-velocity buffers the fused G2P gathers from (staged
  // gather), one per buffer address, encoded on first use
  std::map<const float4*, CUtensorMap> gv_maps;
  bool maps_ok = true;
  // gradient mode
  float* ck_st = nullptr;
  uint32_t* ck_tag = nullptr;
  int* ck_pid = nullptr;
  // chunk buffers (up to kMaxBuffers as memory allows; with two or more the
  // recompute of chunk c-1 runs on rstream while the adjoint of chunk c runs
  // on the caller's stream, and a forward that reaches the horizon keeps its
  // last chunks in them so that the backward does not recompute those)
  int nbuf = 0;
  int chunk_ns = -1;  // non-water particle count the chunk buffers were sized for (-1: not allocated)
  float* chunk[kMaxBuffers] = {};
  float4 *gv_steps[kMaxBuffers] = {}, *gs_steps[kMaxBuffers] = {};  // gs_steps only with a tool
  // compact buffers (b >= 2, without a tool or rigid objects): instead of a
  // full-size grid per step, the grid values of the step's first `cap`
  // active-block list entries (64 nodes each, written by the grid update);
  // kernels that index the grid by node read them from gscr, a full-size grid
  // that the forward's grid update writes and the reverse sweep fills from the
  // compact copy step by step. A step whose list outgrows cap sets bit b in
  // *ovf, and the backward then recomputes that chunk instead of reading it.
  bool compact[kMaxBuffers] = {};
  float4* cgv_steps[kMaxBuffers] = {};
  int cap = 0;
  float4* gscr = nullptr;
  int* ovf = nullptr;
  float *Fp_steps[kMaxBuffers] = {}, *svd_steps[kMaxBuffers] = {};  // 9 x N, 21 x N per step
  int *list_steps[kMaxBuffers] = {}, *count_steps[kMaxBuffers] = {};
  cudaStream_t rstream = nullptr;
  cudaStream_t hstream = nullptr;  // highest priority: the reverse sweep while rstream recomputes
  cudaEvent_t ev_start = nullptr, ev_rec[kMaxBuffers] = {}, ev_adj[kMaxBuffers] = {};
  cudaEvent_t ev_join = nullptr;
  float* adj = nullptr;
  float4 *gadj_v = nullptr, *gadj_m = nullptr;
  float* rows = nullptr;  // N x 24 caller-layout staging
  int* inv = nullptr;     // N: inverse permutation scratch
  float *tool_grad = nullptr, *action_grad = nullptr;
  // tool
  float *pose0 = nullptr, *actions = nullptr, *poses = nullptr;
  bool tool_set = false;
  // sort
  SortBuffers sb{};
  // neighbour arrays of gradient sharing / attraction loss (allocated on first use)
  NbrBuffers nb{};
  // particle-represented rigid objects (allocated when a material is rigid);
  // the recompute keeps each step's projection record for the adjoint
  bool rigid = false;
  RigidBuffers rb{};
  float* rig_steps[kMaxBuffers] = {};
  // losses
  float *lm = nullptr, *ltm = nullptr, *ltd = nullptr, *ldm = nullptr;
  double* dloss = nullptr;
  int* err = nullptr;
  // first of the horizon's last chunks whose per-step data (states, grids,
  // SVDs) the forward that reached max_steps left in the chunk buffers (chunk
  // c in buffer n_ckpt - 1 - c); a backward over that horizon sweeps them
  // without recomputing them (-1: none)
  int rec_from = -1;
  // host state
  int step = 0;
  bool initialized = false, need_sort = true, seeds = false;
  // loss seeds per step (gradient mode): step t -> 15 x N floats (adjoints of
  // x, v, C of the state at step t, in the particle order that state has in
  // the forward); allocated on first use and kept, zero unless t is pending
  std::map<int, float*> seed_buf;
  std::set<int> seeded;
  std::string last_error;
  bool prof = false;
  long long launches = 0;  // kernels launched by this handle
  // CUDA graphs: step loops and backward sweeps are captured once on cstream and
  // replayed on the caller's stream (kernel arguments depend only on the keys)
  bool graphs = true;
  cudaStream_t cstream = nullptr;
  struct FwdGraph {
    int start, n;
    float *W, *W2;
    uint32_t* tag;
    int* pid;
    bool need_sort;
    cudaGraphExec_t exec;
    float *W_after, *W2_after;
    uint32_t* tag_after;
    int* pid_after;
    int rec_from_after;
    long long launches;
  };
  struct BwdGraph {
    int T, n_actions;
    int rec_from;
    std::vector<int> seeded;
    cudaGraphExec_t exec;
    long long launches;
  };
  std::vector<FwdGraph> fwd_graphs;
  std::vector<BwdGraph> bwd_graphs;
  std::vector<ProfRec> prof_recs;
  std::vector<void*> allocs;
};

namespace {

sim_status fail(sim_h h, sim_status s, const std::string& msg) {
  if (h) h->last_error = msg;
  return s;
}

sim_status cuda_fail(sim_h h, cudaError_t e, const char* where) {
  return fail(h, SIM_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <class T>
bool dalloc(sim_h h, T** p, size_t count) {
  if (count == 0) count = 1;
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  h->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return true;
}

template <class T>
void dfree(sim_h h, T** p) {
  if (!*p) return;
  auto it = std::find(h->allocs.begin(), h->allocs.end(), static_cast<void*>(*p));
  if (it != h->allocs.end()) h->allocs.erase(it);
  cudaFree(*p);
  *p = nullptr;
}

// Time the kernels of a stage when profiling is on.
struct Prof {
  sim_h h;
  const char* name;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  int units = 1;
  Prof(sim_h hh, const char* nm, cudaStream_t s = nullptr, int u = 1)
      : h(hh), name(nm), st(s ? s : hh->stream), units(u) {
    if (h->prof) {
      cudaEventCreate(&a);
      cudaEventRecord(a, st);
    }
  }
  ~Prof() {
    if (h->prof) {
      cudaEvent_t b;
      cudaEventCreate(&b);
      cudaEventRecord(b, st);
      h->prof_recs.push_back({name, a, b, units});
    }
  }
};

size_t state_floats(sim_h h) { return (size_t)kStateFields * h->N; }
float* ck_state(sim_h h, int c) { return h->ck_st + (size_t)c * state_floats(h); }
uint32_t* ck_tags(sim_h h, int c) { return h->ck_tag + (size_t)c * h->N; }
int* ck_pids(sim_h h, int c) { return h->ck_pid + (size_t)c * h->N; }
// State j (1..L) of a chunk of L steps in chunk buffer b. Without rigid
// materials the states 1..L-1 keep 16 fields (x, v, C, J / F[0][0]: what the
// adjoint kernels read; the fused recompute writes no more) and the chunk's
// end state, which also seeds the next checkpoint, keeps all 24 in the
// buffer's last slot; with rigid materials (whose recompute rereads F) every
// state keeps 24.
constexpr int kChunkFields = 16;
float* chunk_state(sim_h h, int b, int j, int L) {
  if (h->rigid) return h->chunk[b] + (size_t)(j - 1) * state_floats(h);
  const size_t slot = (size_t)kChunkFields * h->N;
  const int ksteps = std::min(h->k, h->max_steps);
  return h->chunk[b] + (size_t)(j == L ? ksteps - 1 : j - 1) * slot;
}
// floats of one chunk buffer's states
size_t chunk_floats(sim_h h) {
  const size_t ksteps = (size_t)std::min(h->k, h->max_steps);
  if (h->rigid) return ksteps * state_floats(h);
  return (ksteps - 1) * kChunkFields * h->N + state_floats(h);
}

float* rig_step(sim_h h, int b, int j) {
  return h->rig_steps[b] + (size_t)j * h->rb.n_obj * kRigidRecord;
}

GridBuffers fwd_grid(sim_h h, int parity) {
  return GridBuffers{h->acc, h->gv, nullptr, h->flags, h->list + (size_t)parity * h->nflags,
                     h->count + parity, h->Fp, nullptr};
}
GridBuffers step_grid(sim_h h, int b, int j) {
  if (h->compact[b]) {
    GridBuffers g{h->acc, h->gscr, nullptr, h->flags, h->list_steps[b] + (size_t)j * h->nflags,
                  h->count_steps[b] + j, h->Fp_steps[b] + (size_t)j * 9 * h->chunk_ns,
                  h->svd_steps[b] + (size_t)j * 21 * h->chunk_ns};
    g.cgv = h->cgv_steps[b] + (size_t)j * h->cap * 64;
    g.cap = h->cap;
    g.ovf = h->ovf;
    g.ovf_bit = 1 << b;
    return g;
  }
  return GridBuffers{h->acc, h->gv_steps[b] + (size_t)j * h->n3tot,
                     h->gs_steps[b] ? h->gs_steps[b] + (size_t)j * h->n3tot : nullptr,
                     h->flags, h->list_steps[b] + (size_t)j * h->nflags, h->count_steps[b] + j,
                     h->Fp_steps[b] + (size_t)j * 9 * h->chunk_ns, h->svd_steps[b] + (size_t)j * 21 * h->chunk_ns};
}
// Before a kernel reads step j of buffer b by node index: a compact buffer's
// values go into gscr (a full buffer's are in place).
void stage_expand(sim_h h, int b, int j, cudaStream_t s) {
  if (!h->compact[b]) return;
  Prof pr(h, "expand", s);
  launch_expand_grid(h->P, step_grid(h, b, j), h->gscr, s);
  h->launches += 1;
}

// Stages of a step. P2G of step n, grid update of step n and G2P of step n
// (which produces the state of step n + 1); between re-sorts the G2P of step
// n and the P2G of step n + 1 run as one fused kernel.
void stage_p2g(sim_h h, const float* src, const uint32_t* tag, GridBuffers g, int* reset_count,
               cudaStream_t s) {
  Prof pr(h, "p2g", s);
  launch_p2g(h->P, h->tu, src, tag, g, reset_count, h->err, s);
  h->launches += 1;
}
void stage_grid(sim_h h, int step, GridBuffers g, cudaStream_t s) {
  Prof pr(h, "grid_update", s);
  launch_grid_update(h->P, h->tu, g, h->poses, step, h->max_steps, s);
  h->launches += 1;
}
void stage_g2p(sim_h h, const float* src, float* dst, const uint32_t* tag, const float* Fp, const float4* gv,
               cudaStream_t s) {
  Prof pr(h, "g2p", s);
  launch_g2p(h->P, h->tu, src, dst, tag, Fp, gv, h->err, s);
  h->launches += h->N > 0 ? 1 : 0;
}
// lean: the fused kernel writes only the fields the next fused step or G2P reads
// (x and a liquid's J); for forward steps whose state is not kept
// Tensor map of a grid-velocity buffer for the staged gather (nullptr if the
// staged gather is off or the encoder is unavailable).
const CUtensorMap* gv_map(sim_h h, const float4* gv) {
  if (!h->tu.stage_gather || !h->maps_ok) return nullptr;
  auto it = h->gv_maps.find(gv);
  if (it != h->gv_maps.end()) return &it->second;
  CUtensorMap m;
  if (!encode_grid_map(h->P, gv, &m)) {
    h->maps_ok = false;
    return nullptr;
  }
  return &(h->gv_maps[gv] = m);
}

void stage_g2p2g(sim_h h, const float* src, float* dst, const uint32_t* tag, const float* Fp_prev,
                 const float4* gv_prev, GridBuffers g, int* reset_count, cudaStream_t s, bool lean = false) {
  Prof pr(h, "g2p2g", s);
  launch_g2p2g(h->P, h->tu, src, dst, tag, Fp_prev, gv_prev, g, reset_count, h->err, s, lean,
               gv_map(h, gv_prev));
  h->launches += 1;
}

// Steps [n0, n1) of a forward run between re-sorts as one persistent
// cooperative launch: P2G of step n0 from src, fused lean steps into W, grid
// updates inside. Profiled as "fwd_run", counted once per step.
void stage_forward_run(sim_h h, const float* src, int n0, int n1, cudaStream_t s) {
  Prof pr(h, "fwd_run", s, n1 - n0);
  GridBuffers g = fwd_grid(h, 0);
  cudaError_t e = launch_forward_run(h->P, h->tu, src, h->W, h->tag_cur, g, h->list, h->nflags, h->count,
                                     h->poses, n0, n1, h->max_steps, h->tile_ctr, h->bar, h->err, s);
  if (e != cudaSuccess) {
    // the cooperative launch was refused (nothing ran): this and later runs use
    // the per-step kernels
    cudaGetLastError();
    h->tu.persistent = 0;
    return;
  }
  h->launches += h->N > 0 ? 1 : 0;
}

// A re-sort falls on step m (checkpoint steps in gradient mode, else every
// `resort` steps).
bool sort_step(sim_h h, int m) { return h->k > 0 ? (m % h->k == 0) : (m % h->resort == 0); }

// rigidity projection of the state just written by a G2P (and its adjoint)
void stage_rigid(sim_h h, float* st, const uint32_t* tag, const int* pid, float* rec, cudaStream_t s) {
  if (!h->rigid) return;
  Prof pr(h, "rigid", s);
  launch_rigid_project(h->P, st, tag, pid, h->rb, rec, s);
  h->launches += h->N > 0 ? 3 : 0;
}
void stage_rigid_adj(sim_h h, const uint32_t* tag, const int* pid, const float* rec, cudaStream_t s) {
  if (!h->rigid) return;
  Prof pr(h, "rigid_adj", s);
  launch_rigid_adjoint(h->P, h->adj, tag, pid, h->rb, rec, s);
  h->launches += h->N > 0 ? 3 : 0;
}

void do_sort(sim_h h, const float* st_in, const uint32_t* tag_in, const int* pid_in, float* st_out,
             uint32_t* tag_out, int* pid_out, cudaStream_t s) {
  Prof pr(h, "sort", s);
  launch_sort(h->P, st_in, tag_in, pid_in, st_out, tag_out, pid_out, h->sb, s);
  h->launches += h->P.N > 0 ? 5 : 3;
}

sim_status check_err(sim_h h, const char* where) {
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, where);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, where);
  int flag = 0;
  e = cudaMemcpy(&flag, h->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, where);
  // a particle that leaves the grid is the usual root cause of later non-finite values
  if (flag & kErrDomain)
    return fail(h, SIM_E_DOMAIN, std::string(where) + ": a particle's stencil left the grid");
  if (flag & kErrNaN) return fail(h, SIM_E_NAN, std::string(where) + ": non-finite particle state");
  if (flag & kErrTimeout) return fail(h, SIM_E_TIMEOUT, std::string(where) + ": device wait timed out");
  return SIM_OK;
}

// Copy `bytes` from a caller pointer into a device buffer.
cudaError_t to_device(sim_h h, void* dst, const void* src, size_t bytes, int on_device) {
  if (bytes == 0) return cudaSuccess;
  if (on_device) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, h->stream);
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(h->stream);
}

cudaError_t to_caller(sim_h h, void* dst, const void* src, size_t bytes, int on_device) {
  if (bytes == 0) return cudaSuccess;
  if (on_device) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, h->stream);
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(h->stream);
}

bool scene_range(sim_h h, int scene, int* lo, int* cnt) {
  if (scene == -1) {
    *lo = 0;
    *cnt = h->N;
    return true;
  }
  if (scene < 0 || scene >= h->S) return false;
  *lo = h->offsets[scene];
  *cnt = h->counts[scene];
  return true;
}

// Loss seeds of the state at step t: the adjoints of x, v and C (fields 0..14
// of the adjoint state's layout), in the particle order of checkpoint
// order_of_step(t), the order that state has in the forward. Allocated on
// first use and kept, because the backward's CUDA graphs refer to it; marks
// step t pending. nullptr if the allocation fails.
constexpr int kSeedFields = 15;
int order_of_step(sim_h h, int t) { return (t - 1) / h->k; }
float* seed_buffer(sim_h h, int t) {
  float* p = nullptr;
  auto it = h->seed_buf.find(t);
  if (it != h->seed_buf.end()) {
    p = it->second;
  } else {
    if (!dalloc(h, &p, (size_t)kSeedFields * h->N)) return nullptr;
    cudaMemsetAsync(p, 0, sizeof(float) * kSeedFields * h->N, h->stream);
    h->seed_buf[t] = p;
  }
  h->seeded.insert(t);
  h->seeds = true;
  return p;
}
void clear_seeds(sim_h h) {
  for (int t : h->seeded) cudaMemsetAsync(h->seed_buf[t], 0, sizeof(float) * kSeedFields * h->N, h->stream);
  h->seeded.clear();
  h->seeds = false;
}

// Restart the trajectory from the stored initial state X0 (caller order).
void restart(sim_h h) {
  cudaMemcpyAsync(h->W, h->X0, state_floats(h) * sizeof(float), cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(h->tagA, h->tag0, (size_t)h->N * sizeof(uint32_t), cudaMemcpyDeviceToDevice, h->stream);
  h->tag_cur = h->tagA;
  h->pid_cur = h->pidA;
  launch_iota(h->pidA, h->N, h->stream);
  h->launches += h->N > 0 ? 1 : 0;
  cudaMemsetAsync(h->count, 0, 2 * sizeof(int), h->stream);
  h->step = 0;
  h->need_sort = true;
  clear_seeds(h);
  h->rec_from = -1;
  if (h->adj) cudaMemsetAsync(h->adj, 0, state_floats(h) * sizeof(float), h->stream);
  cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
}

void set_params(sim_h h) {
  const sim_config& c = h->cfg;
  Params& P = h->P;
  std::memset(&P, 0, sizeof(P));
  P.n = c.grid_n;
  P.nb = (c.grid_n + kBlockEdge - 1) / kBlockEdge;
  P.S = h->S;
  P.N = h->N;
  P.n3 = (long long)c.grid_n * c.grid_n * c.grid_n;
  P.NB = P.nb * P.nb * P.nb;
  int mb = 1;
  while (mb < P.n) mb <<= 1;
  P.MB = mb * mb * mb;
  P.dx = 1.0f / c.grid_n;
  P.inv_dx = float(c.grid_n);
  P.dt = c.dt;
  for (int i = 0; i < 3; ++i) P.g[i] = c.gravity[i];
  P.bound = c.bound;
  P.n_mat = c.n_materials;
  P.Nl = 0;
  P.Ns = h->N;
  for (int m = 0; m < c.n_materials; ++m) {
    const sim_material& sm = c.materials[m];
    MatParams& M = P.mat[m];
    M.kind = sm.kind;
    M.vol = sm.volume;
    M.mass = sm.rho * sm.volume;
    if (sm.kind == SIM_LIQUID || sm.kind == SIM_VISCOUS_LIQUID) {
      M.mu = sm.kind == SIM_VISCOUS_LIQUID ? sm.shear : 0.0f;
      M.lam = sm.bulk;
    } else {
      double E = sm.E, nu = sm.nu;
      double mu = E / (2.0 * (1.0 + nu));
      double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
      M.mu = float(mu);
      M.lam = float(lam);
      if (sm.kind == SIM_BOX_YIELD) {
        M.k_yield = sm.crit_compress;
        M.c_dp = sm.crit_stretch;
      } else {
        M.k_yield = float(sm.yield_stress / (2.0 * mu));
        double sp = std::sin(sm.friction_deg * M_PI / 180.0);
        double alpha = std::sqrt(2.0 / 3.0) * 2.0 * sp / (3.0 - sp);
        M.c_dp = float(alpha * (3.0 * lam + 2.0 * mu) / (2.0 * mu));
      }
    }
  }
  P.ext = 0;
  for (int m = 0; m < c.n_materials; ++m)
    if (c.materials[m].kind == SIM_BOX_YIELD || c.materials[m].kind == SIM_VISCOUS_LIQUID ||
        c.materials[m].kind == SIM_RIGID)
      P.ext = 1;
  P.tool = c.tool_enabled ? 1 : 0;
  for (int i = 0; i < 3; ++i) P.half[i] = c.tool_half[i];
  P.eps_c = c.contact_eps;
  P.inv_ell = c.contact_soft > 0.0f ? 1.0f / c.contact_soft : float(c.grid_n);
  P.mu_f = c.friction;
}

// Run chunk c (steps [c k, min(T, c k + k))) from its checkpoint into chunk
// buffer b on stream rs, keeping every step's state, grids, F_p, SVD and rigid
// record for the adjoint.
void recompute_chunk(sim_h h, int c, int b, int T, cudaStream_t rs) {
  const int K = h->k;
  const int s0 = c * K, L = std::min(T, s0 + K) - s0;
  const uint32_t* tag = ck_tags(h, c);
  cudaMemsetAsync(h->count_steps[b], 0, sizeof(int) * L, rs);
  for (int j = 0; j < L; ++j) {
    GridBuffers g = step_grid(h, b, j);
    if (j == 0) {
      stage_p2g(h, ck_state(h, c), tag, g, nullptr, rs);
    } else {
      GridBuffers gp = step_grid(h, b, j - 1);
      const float* src = j == 1 ? ck_state(h, c) : chunk_state(h, b, j - 1, L);
      if (h->rigid) {
        stage_g2p(h, src, chunk_state(h, b, j, L), tag, gp.Fp, gp.gv, rs);
        stage_rigid(h, chunk_state(h, b, j, L), tag, ck_pids(h, c), rig_step(h, b, j - 1), rs);
        stage_p2g(h, chunk_state(h, b, j, L), tag, g, nullptr, rs);
      } else {
        stage_g2p2g(h, src, chunk_state(h, b, j, L), tag, gp.Fp, gp.gv, g, nullptr, rs);
      }
    }
    stage_grid(h, s0 + j, g, rs);
  }
  GridBuffers gl = step_grid(h, b, L - 1);
  const float* src = L == 1 ? ck_state(h, c) : chunk_state(h, b, L - 1, L);
  stage_g2p(h, src, chunk_state(h, b, L, L), tag, gl.Fp, gl.gv, rs);
  stage_rigid(h, chunk_state(h, b, L, L), tag, ck_pids(h, c), rig_step(h, b, L - 1), rs);
}

void drop_graphs(sim_h h) {
  for (auto& g : h->fwd_graphs) cudaGraphExecDestroy(g.exec);
  for (auto& g : h->bwd_graphs) cudaGraphExecDestroy(g.exec);
  h->fwd_graphs.clear();
  h->bwd_graphs.clear();
}

// Chunk buffers for gradient mode, sized once the split of the particles into
// water and other materials is known (the F_p and SVD records of a step hold
// only the Ns non-water particles): as many as fit in 85% of the free device
// memory, at most one per chunk and kMaxBuffers, at least one. Each holds k
// states, the per-step grid velocities (with a tool also the pre-contact grid
// the contact adjoint needs; without one the grid adjoint reads the
// velocities), active-block lists, F_p and the SVDs; buffers 2 and up keep the
// grid velocities as a compact copy when the scene has no tool and no rigid
// objects. Reallocated (dropping the captured graphs that refer to them) when
// Ns changes.
sim_status ensure_chunk_buffers(sim_h h) {
  if (h->k <= 0 || h->chunk_ns == h->P.Ns) return SIM_OK;
  cudaStreamSynchronize(h->stream);
  if (h->rstream) cudaStreamSynchronize(h->rstream);
  if (h->hstream) cudaStreamSynchronize(h->hstream);
  drop_graphs(h);
  auto free_buffer = [&](int b) {
    dfree(h, &h->chunk[b]);
    dfree(h, &h->gv_steps[b]);
    dfree(h, &h->gs_steps[b]);
    dfree(h, &h->cgv_steps[b]);
    dfree(h, &h->list_steps[b]);
    dfree(h, &h->count_steps[b]);
    dfree(h, &h->Fp_steps[b]);
    dfree(h, &h->svd_steps[b]);
    dfree(h, &h->rig_steps[b]);
    h->compact[b] = false;
  };
  for (int b = 0; b < kMaxBuffers; ++b) free_buffer(b);
  dfree(h, &h->gscr);
  dfree(h, &h->ovf);
  h->nbuf = 0;
  h->chunk_ns = -1;
  h->rec_from = -1;
  const size_t Ns = (size_t)std::max(h->P.Ns, 1);
  const size_t ksteps = (size_t)std::min(h->k, h->max_steps);
  const int ngrids = h->P.tool ? 2 : 1;
  const size_t rig = h->rigid ? (size_t)h->rb.n_obj * kRigidRecord * sizeof(float) : 0;
  const size_t step_common = sizeof(int) * ((size_t)h->nflags + 1) + 30 * sizeof(float) * Ns;
  const size_t chunk_bytes = chunk_floats(h) * sizeof(float) +
                             ksteps * (ngrids * sizeof(float4) * (size_t)h->n3tot + step_common + rig);
  // compact buffers hold an eighth of the grid's blocks per step
  const int cap = int(std::max<size_t>(1, ((size_t)h->nflags + 7) / 8));
  const size_t compact_bytes = chunk_floats(h) * sizeof(float) +
                               ksteps * (sizeof(float4) * (size_t)cap * 64 + step_common);
  const int most = int(std::min<size_t>(h->n_ckpt, kMaxBuffers));
  const bool use_compact = !h->P.tool && !h->rigid && most > 2;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const size_t budget = free_b / 20 * 17;
  size_t used = use_compact ? sizeof(float4) * (size_t)h->n3tot : 0;  // gscr
  int want = 0;
  for (int b = 0; b < most; ++b) {
    const size_t sz = (use_compact && b >= 2) ? compact_bytes : chunk_bytes;
    if (used + sz > budget) break;
    used += sz;
    ++want;
  }
  want = std::max(want, 1);
  h->cap = cap;
  if (use_compact && want > 2 &&
      !(dalloc(h, &h->gscr, (size_t)h->n3tot) && dalloc(h, &h->ovf, 1))) {
    dfree(h, &h->gscr);
    dfree(h, &h->ovf);
    want = 2;
  }
  int got = 0;
  for (int b = 0; b < want; ++b) {
    const bool cb = h->gscr != nullptr && b >= 2;
    bool ok = dalloc(h, &h->chunk[b], chunk_floats(h)) &&
              (cb ? dalloc(h, &h->cgv_steps[b], (size_t)cap * 64 * ksteps)
                  : dalloc(h, &h->gv_steps[b], (size_t)h->n3tot * ksteps)) &&
              (cb || !h->P.tool || dalloc(h, &h->gs_steps[b], (size_t)h->n3tot * ksteps)) &&
              dalloc(h, &h->list_steps[b], (size_t)h->nflags * ksteps) && dalloc(h, &h->count_steps[b], ksteps) &&
              dalloc(h, &h->Fp_steps[b], 9 * Ns * ksteps) && dalloc(h, &h->svd_steps[b], 21 * Ns * ksteps) &&
              (!h->rigid || dalloc(h, &h->rig_steps[b], ksteps * h->rb.n_obj * kRigidRecord));
    if (!ok) {
      free_buffer(b);
      break;
    }
    h->compact[b] = cb;
    ++got;
  }
  if (got == 0) return fail(h, SIM_E_OOM, "chunk buffers: out of device memory");
  h->nbuf = got;
  if (h->nbuf >= 2 && !h->rstream) {
    int least = 0, greatest = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
              cudaStreamCreateWithPriority(&h->rstream, cudaStreamNonBlocking, least) == cudaSuccess &&
              cudaStreamCreateWithPriority(&h->hstream, cudaStreamNonBlocking, greatest) == cudaSuccess &&
              cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return cuda_fail(h, cudaGetLastError(), "chunk buffers: streams");
  }
  for (int b = 0; h->nbuf >= 2 && b < h->nbuf; ++b) {
    if (!h->ev_rec[b] && cudaEventCreateWithFlags(&h->ev_rec[b], cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(h, cudaGetLastError(), "chunk buffers: events");
    if (!h->ev_adj[b] && cudaEventCreateWithFlags(&h->ev_adj[b], cudaEventDisableTiming) != cudaSuccess)
      return cuda_fail(h, cudaGetLastError(), "chunk buffers: events");
  }
  h->chunk_ns = h->P.Ns;
  return SIM_OK;
}

// Chunks a forward that reaches the horizon keeps for the backward (in their
// own buffers; the rest are recomputed through two alternating buffers, while
// the sweep runs unless the handle is profiling, or through the one buffer in
// order when only one exists).
int recorded_chunks(sim_h h) {
  if (h->k <= 0) return 0;
  if (h->nbuf < 2) return 1;
  return std::min(h->nbuf, h->n_ckpt);
}

// Buffer of chunk c in the backward of a horizon of nch chunks whose chunks
// [rec_from, nch) were kept by the forward (rec_from = nch: none kept).
int chunk_buffer(sim_h h, int c, int nch, int rec_from) {
  if (c >= rec_from) return nch - 1 - c;
  if (h->nbuf < 2) return 0;
  // alternate between buffers 0 and 1, starting with the one the sweep of
  // chunk rec_from does not read
  const int R = nch - rec_from;
  return (R + (rec_from - 1 - c)) % 2;
}

// Enqueue n MLS-MPM steps on stream s (re-sorting into grid blocks at every
// checkpoint, or every `resort` steps without checkpoints) and advance the
// host-side bookkeeping. The G2P of the last step completes the state. With
// checkpoints, a call that runs the horizon's whole last chunk runs it as the
// backward's recompute would, into the chunk buffer the backward reads first,
// and copies the final state out.
void enqueue_steps(sim_h h, int n_steps, cudaStream_t s) {
  const float* cur = nullptr;  // buffer holding the state whose P2G ran last
  for (int it = 0; it < n_steps; ++it) {
    const int n = h->step;
    const int rec_first = h->n_ckpt - recorded_chunks(h);  // first chunk the forward keeps
    if (h->k > 0 && n == rec_first * h->k && n + (n_steps - it) == h->max_steps) {
      // the horizon's last chunks run as the backward's recompute would, each
      // into the buffer its sweep reads; the final state is copied out
      if (it > 0) {
        stage_g2p(h, cur, h->W, h->tag_cur, h->Fp, h->gv, s);
        stage_rigid(h, h->W, h->tag_cur, h->pid_cur, h->rb.rec, s);
      }
      const float* src = h->W;
      if (h->ovf) cudaMemsetAsync(h->ovf, 0, sizeof(int), s);
      for (int c = rec_first; c < h->n_ckpt; ++c) {
        const int b = chunk_buffer(h, c, h->n_ckpt, rec_first);
        do_sort(h, src, h->tag_cur, h->pid_cur, ck_state(h, c), ck_tags(h, c), ck_pids(h, c), s);
        h->tag_cur = ck_tags(h, c);
        h->pid_cur = ck_pids(h, c);
        recompute_chunk(h, c, b, h->max_steps, s);
        const int Lc = std::min(h->max_steps, (c + 1) * h->k) - c * h->k;
        src = chunk_state(h, b, Lc, Lc);
      }
      h->need_sort = false;
      cudaMemcpyAsync(h->W, src, state_floats(h) * sizeof(float), cudaMemcpyDeviceToDevice, s);
      h->step = h->max_steps;
      h->rec_from = rec_first;
      return;
    }
    const bool sort_now = h->k > 0 ? (n % h->k == 0) : (h->need_sort || n % h->resort == 0);
    GridBuffers g = fwd_grid(h, n & 1);
    int* reset = h->count + ((n + 1) & 1);
    if (it > 0 && !sort_now && !h->rigid) {
      // the state written here is read only by the next fused step or by the
      // G2P that completes it (before a re-sort and at the end of the call)
      stage_g2p2g(h, cur, h->W, h->tag_cur, h->Fp, h->gv, g, reset, s, /*lean=*/true);
      cur = h->W;
    } else {
      if (it > 0) {
        stage_g2p(h, cur, h->W, h->tag_cur, h->Fp, h->gv, s);
        stage_rigid(h, h->W, h->tag_cur, h->pid_cur, h->rb.rec, s);
      }
      const float* src = h->W;
      if (sort_now && h->k > 0) {
        int c = n / h->k;
        do_sort(h, h->W, h->tag_cur, h->pid_cur, ck_state(h, c), ck_tags(h, c), ck_pids(h, c), s);
        h->tag_cur = ck_tags(h, c);
        h->pid_cur = ck_pids(h, c);
        src = ck_state(h, c);
      } else if (sort_now) {
        uint32_t* tag_out = (h->tag_cur == h->tagA) ? h->tagB : h->tagA;
        int* pid_out = (h->pid_cur == h->pidA) ? h->pidB : h->pidA;
        do_sort(h, h->W, h->tag_cur, h->pid_cur, h->W2, tag_out, pid_out, s);
        std::swap(h->W, h->W2);
        h->tag_cur = tag_out;
        h->pid_cur = pid_out;
        src = h->W;
      }
      h->need_sort = false;
      if (h->tu.persistent && h->coop && !h->rigid && h->N > 0) {
        // this step and the fused steps up to the next re-sort (or the end of
        // the call) in one persistent launch, grid updates included
        int L = 1;
        while (it + L < n_steps && !sort_step(h, n + L)) ++L;
        stage_forward_run(h, src, n, n + L, s);
        if (h->tu.persistent) {
          cur = L == 1 ? src : h->W;
          h->step += L;
          it += L - 1;
          continue;
        }
      }
      stage_p2g(h, src, h->tag_cur, g, reset, s);
      cur = src;
    }
    stage_grid(h, n, g, s);
    h->step++;
  }
  if (n_steps > 0) {
    stage_g2p(h, cur, h->W, h->tag_cur, h->Fp, h->gv, s);
    stage_rigid(h, h->W, h->tag_cur, h->pid_cur, h->rb.rec, s);
  }
}

// Capture `fn(cstream)` into a graph and instantiate it. Returns nullptr on
// failure (the caller then runs the work directly).
template <class Fn>
cudaGraphExec_t capture(sim_h h, Fn fn, bool node_priority = false) {
  if (!h->cstream && cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (cudaStreamBeginCapture(h->cstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  fn(h->cstream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cstream, &graph);
  if (e != cudaSuccess || !graph) {
    cudaGetLastError();
    return nullptr;
  }
  cudaGraphExec_t exec = nullptr;
  // node_priority: kernels keep the priority of the stream they were captured
  // on (the backward's sweep and recompute streams) instead of taking the
  // launch stream's
  e = cudaGraphInstantiate(&exec, graph, node_priority ? cudaGraphInstantiateFlagUseNodePriority : 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return exec;
}

// A checkpoint before the current step holds the state of step t = c*k
// (c >= 1), in checkpoint c's particle order; false for any other step.
bool retained_checkpoint(sim_h h, int t, int* c) {
  if (h->k <= 0 || t <= 0 || t >= h->step || t % h->k != 0) return false;
  *c = t / h->k;
  return *c < h->n_ckpt;
}

// Step t of a loss seed: step = -1 is the current step; seeds need gradient
// mode and 1 <= t <= the current step.
sim_status seed_step(sim_h h, const char* where, int step, int* t) {
  if (h->k <= 0) return fail(h, SIM_E_STATE, std::string(where) + ": checkpointing is off (forward only)");
  if (h->step == 0) return fail(h, SIM_E_STATE, std::string(where) + ": no step taken");
  if (step < -1) return fail(h, SIM_E_ARG, std::string(where) + ": step must be -1 (current) or >= 1");
  const int tt = step < 0 ? h->step : step;
  if (tt < 1 || tt > h->step)
    return fail(h, SIM_E_STATE, std::string(where) + ": step " + std::to_string(tt) +
                                    " is not in [1, current step " + std::to_string(h->step) + "]");
  *t = tt;
  return SIM_OK;
}

// Caller-order gradients (row-major [count][ncomp[i]] per source) added to the
// seeds of step t at adjoint fields field[i].
sim_status add_seeds(sim_h h, const char* where, int scene, int step, const float* const* srcs, const int* field,
                     const int* ncomp, int n_src, int on_device) {
  int t = 0;
  sim_status st = seed_step(h, where, step, &t);
  if (st != SIM_OK) return st;
  int lo, cnt;
  if (!scene_range(h, scene, &lo, &cnt)) return fail(h, SIM_E_ARG, std::string(where) + ": bad scene");
  float* seed = seed_buffer(h, t);
  if (!seed) return fail(h, SIM_E_OOM, std::string(where) + ": out of device memory");
  const int c = order_of_step(h, t);
  for (int f = 0; f < n_src; ++f) {
    if (!srcs[f]) continue;
    cudaError_t e = to_device(h, h->rows, srcs[f], sizeof(float) * ncomp[f] * cnt, on_device);
    if (e != cudaSuccess) return cuda_fail(h, e, where);
    launch_add_seed(seed + (size_t)field[f] * h->N, h->rows, ck_pids(h, c), ck_tags(h, c), scene, lo, cnt, h->N,
                    h->stream, ncomp[f]);
    h->launches += h->N > 0 ? 1 : 0;
  }
  return check_err(h, where);
}

// Where a state loss of step t reads its state and writes dL/dx. At the
// current step: the working state, straight into the seeds of t. At a
// retained checkpoint c*k before it: the checkpoint (order c), into scratch
// (the first 3N floats of rows) that finish_loss_site re-orders to the order
// of the seeds of t (checkpoint c - 1) and adds.
struct LossSite {
  const float* st;
  const uint32_t* tag;
  float* grad;
  float* seed;
  int ckpt;  // -1: the current step
};
sim_status loss_site(sim_h h, const char* where, int step, LossSite* out) {
  int t = 0;
  if (h->k <= 0) return fail(h, SIM_E_STATE, std::string(where) + ": checkpointing is off (forward only)");
  if (h->step == 0) return fail(h, SIM_E_STATE, std::string(where) + ": no step taken");
  if (step < -1) return fail(h, SIM_E_ARG, std::string(where) + ": step must be -1 (current) or >= 1");
  t = step < 0 ? h->step : step;
  int c = -1;
  if (t != h->step && !retained_checkpoint(h, t, &c))
    return fail(h, SIM_E_STATE, std::string(where) + ": the state of step " + std::to_string(t) +
                                    " is not retained (the current step or a checkpoint step c*k before it)");
  float* seed = seed_buffer(h, t);
  if (!seed) return fail(h, SIM_E_OOM, std::string(where) + ": out of device memory");
  if (c < 0) {
    *out = LossSite{h->W, h->tag_cur, seed, seed, -1};
  } else {
    cudaMemsetAsync(h->rows, 0, sizeof(float) * 3 * h->N, h->stream);
    *out = LossSite{ck_state(h, c), ck_tags(h, c), h->rows, seed, c};
  }
  return SIM_OK;
}
void finish_loss_site(sim_h h, const LossSite& s) {
  if (s.ckpt < 0 || h->N == 0) return;
  float* tmp = h->rows + (size_t)3 * h->N;
  launch_permute_state(h->rows, tmp, ck_pids(h, s.ckpt), ck_pids(h, s.ckpt - 1), h->inv, h->N, 3, h->stream);
  launch_add_fields(s.seed, tmp, (long long)3 * h->N, 0, h->stream);
  h->launches += 3;
}

constexpr size_t kMaxGraphs = 16;

}  // namespace

extern "C" {

const char* sim_version(void) { return kVersion; }

const char* sim_last_error(sim_h h) {
  if (!h) return "invalid handle";
  return h->last_error.c_str();
}

sim_status sim_destroy(sim_h h) {
  if (!h) return SIM_OK;
  cudaStreamSynchronize(h->stream);
  for (auto& r : h->prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (h->rstream) cudaStreamSynchronize(h->rstream);
  if (h->hstream) cudaStreamSynchronize(h->hstream);
  for (auto& g : h->fwd_graphs) cudaGraphExecDestroy(g.exec);
  for (auto& g : h->bwd_graphs) cudaGraphExecDestroy(g.exec);
  if (h->cstream) cudaStreamDestroy(h->cstream);
  for (void* p : h->allocs) cudaFree(p);
  for (int b = 0; b < kMaxBuffers; ++b) {
    if (h->ev_rec[b]) cudaEventDestroy(h->ev_rec[b]);
    if (h->ev_adj[b]) cudaEventDestroy(h->ev_adj[b]);
  }
  if (h->ev_start) cudaEventDestroy(h->ev_start);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->rstream) cudaStreamDestroy(h->rstream);
  if (h->hstream) cudaStreamDestroy(h->hstream);
  delete h;
  return SIM_OK;
}

sim_status sim_create(const sim_config* c, sim_h* out) {
  if (!out) return SIM_E_ARG;
  *out = nullptr;
  if (!c) return SIM_E_ARG;
  if (c->grid_n < 4 || c->grid_n > 1024 || !(c->dt > 0.0f) || c->n_scenes < 1 ||
      c->n_scenes > (1 << 23) || !c->scene_counts || c->n_materials < 1 ||
      c->n_materials > SIM_MAX_MATERIALS || c->bound < 0 || c->checkpoint_every < 0 ||
      c->max_steps < 0 || c->substeps_per_action < 0 || c->resort_every < 0)
    return SIM_E_ARG;
  for (int m = 0; m < c->n_materials; ++m) {
    const sim_material& sm = c->materials[m];
    if (sm.kind < 0 || sm.kind > SIM_RIGID || !(sm.rho > 0.0f) || !(sm.volume > 0.0f)) return SIM_E_ARG;
    if (sm.kind == SIM_VISCOUS_LIQUID && !(sm.shear >= 0.0f)) return SIM_E_ARG;
    if (sm.kind == SIM_BOX_YIELD &&
        (!(sm.crit_compress >= 0.0f && sm.crit_compress < 1.0f) || !(sm.crit_stretch >= 0.0f)))
      return SIM_E_ARG;
    if (sm.kind != SIM_LIQUID && sm.kind != SIM_VISCOUS_LIQUID && sm.kind != SIM_RIGID &&
        (!(sm.E > 0.0f) || !(sm.nu > -1.0f && sm.nu < 0.5f)))
      return SIM_E_ARG;
  }
  long long Ntot = 0;
  for (int s = 0; s < c->n_scenes; ++s) {
    if (c->scene_counts[s] < 0) return SIM_E_ARG;
    Ntot += c->scene_counts[s];
  }
  if (Ntot >= (1LL << 31) / kStateFields) return SIM_E_ARG;
  if (c->checkpoint_every > 0 && c->max_steps < 1) return SIM_E_ARG;
  if (c->tool_enabled && c->max_steps < 1) return SIM_E_ARG;
  sim_h h = new mpm_sim();
  h->cfg = *c;
  h->cfg.scene_counts = nullptr;
  h->S = c->n_scenes;
  h->counts.assign(c->scene_counts, c->scene_counts + c->n_scenes);
  h->offsets.resize(h->S + 1);
  h->offsets[0] = 0;
  for (int s = 0; s < h->S; ++s) h->offsets[s + 1] = h->offsets[s] + h->counts[s];
  h->N = int(Ntot);
  h->n = c->grid_n;
  h->stream = static_cast<cudaStream_t>(c->cuda_stream);
  h->k = c->checkpoint_every;
  h->max_steps = c->max_steps;
  h->spa = c->substeps_per_action > 0 ? c->substeps_per_action : 1;
  h->resort = c->resort_every > 0 ? c->resort_every : 8;
  h->graphs = c->no_graphs == 0;
  {
    int dev = 0, coop = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess)
      h->coop = coop != 0;
    cudaGetLastError();
  }
  set_params(h);
  h->n3tot = (long long)h->S * h->P.n3;
  h->nflags = (long long)h->S * h->P.NB;
  long long nbins = (long long)h->S * h->P.MB;
  // sort keys (class, scene, Morton code) are 32-bit: 2 x nbins of them
  if (nbins >= (1LL << 31) || 2 * nbins > (1LL << 32)) {
    delete h;
    return SIM_E_ARG;
  }
  const size_t NS = state_floats(h);
  const int N = h->N;
  bool ok = dalloc(h, &h->X0, NS) && dalloc(h, &h->W, NS) && dalloc(h, &h->W2, NS) &&
            dalloc(h, &h->Fp, (size_t)9 * N) && dalloc(h, &h->tag0, N) && dalloc(h, &h->tagA, N) &&
            dalloc(h, &h->tagB, N) && dalloc(h, &h->pidA, N) && dalloc(h, &h->pidB, N) &&
            dalloc(h, &h->acc, h->n3tot) && dalloc(h, &h->gv, h->n3tot) &&
            dalloc(h, &h->flags, h->nflags) && dalloc(h, &h->list, 2 * h->nflags) &&
            dalloc(h, &h->count, 2) && dalloc(h, &h->err, 1) && dalloc(h, &h->dloss, h->S) &&
            dalloc(h, &h->tile_ctr, 2) && dalloc(h, &h->bar, 2) && dalloc(h, &h->nwater, 1) &&
            dalloc(h, &h->rows, (size_t)N * kStateFields) && dalloc(h, &h->inv, N);
  h->sb.n_bins = int(nbins);
  ok = ok && dalloc(h, &h->sb.key, N) && dalloc(h, &h->sb.rank, N) && dalloc(h, &h->sb.bins, 2 * nbins + 1) &&
       dalloc(h, &h->sb.tile_sums, 2 * nbins / 4096 + 2);
  if (ok && h->P.tool) {
    h->n_act_max = (h->max_steps + h->spa - 1) / h->spa;
    ok = dalloc(h, &h->pose0, (size_t)7 * h->S) && dalloc(h, &h->actions, (size_t)h->S * h->n_act_max * 6) &&
         dalloc(h, &h->poses, (size_t)h->S * h->max_steps * kToolFields) &&
         dalloc(h, &h->action_grad, (size_t)h->S * h->n_act_max * 6);
  }
  if (ok && h->k > 0) {
    h->n_ckpt = (h->max_steps + h->k - 1) / h->k;
    ok = dalloc(h, &h->ck_st, NS * h->n_ckpt) && dalloc(h, &h->ck_tag, (size_t)N * h->n_ckpt) &&
         dalloc(h, &h->ck_pid, (size_t)N * h->n_ckpt) && dalloc(h, &h->adj, NS) &&
         dalloc(h, &h->gadj_v, h->n3tot) && dalloc(h, &h->gadj_m, h->n3tot) &&
         dalloc(h, &h->tool_grad, (size_t)h->S * h->max_steps * kToolGradFields);
  }
  for (int m = 0; m < c->n_materials; ++m) h->rigid = h->rigid || c->materials[m].kind == SIM_RIGID;
  if (ok && h->rigid) {
    const size_t no = (size_t)h->S * c->n_materials;
    h->rb.n_obj = int(no);
    ok = dalloc(h, &h->rb.rest, (size_t)3 * N) && dalloc(h, &h->rb.cst, no * kRigidConst) &&
         dalloc(h, &h->rb.sums, no * kRigidReplicas * kRigidLine) && dalloc(h, &h->rb.rec, no * kRigidRecord);
    if (ok && h->k > 0)
      ok = dalloc(h, &h->rb.gsums, no * kRigidReplicas * kRigidLine) && dalloc(h, &h->rb.gout, no * kRigidSums);
    if (ok) {
      cudaMemsetAsync(h->rb.rest, 0, sizeof(float) * 3 * N, h->stream);
      cudaMemsetAsync(h->rb.cst, 0, sizeof(float) * no * kRigidConst, h->stream);
      cudaMemsetAsync(h->rb.sums, 0, sizeof(double) * no * kRigidReplicas * kRigidLine, h->stream);
      if (h->rb.gsums) cudaMemsetAsync(h->rb.gsums, 0, sizeof(double) * no * kRigidReplicas * kRigidLine, h->stream);
    }
  }
  if (!ok) {
    sim_destroy(h);
    return SIM_E_OOM;
  }
  // zero-initialised invariants: acc, flags, gadj_v; X0 = rest state at the origin
  cudaMemsetAsync(h->acc, 0, sizeof(float4) * h->n3tot, h->stream);
  cudaMemsetAsync(h->gv, 0, sizeof(float4) * h->n3tot, h->stream);
  cudaMemsetAsync(h->flags, 0, sizeof(int) * h->nflags, h->stream);
  cudaMemsetAsync(h->count, 0, 2 * sizeof(int), h->stream);
  cudaMemsetAsync(h->X0, 0, NS * sizeof(float), h->stream);
  launch_init_state(h->X0, N, h->stream);
  std::vector<uint32_t> tags(N);
  for (int s = 0; s < h->S; ++s)
    for (int i = h->offsets[s]; i < h->offsets[s + 1]; ++i) tags[i] = uint32_t(s) << 8;
  if (N) cudaMemcpy(h->tag0, tags.data(), sizeof(uint32_t) * N, cudaMemcpyHostToDevice);
  if (h->k > 0) {
    cudaMemsetAsync(h->gadj_v, 0, sizeof(float4) * h->n3tot, h->stream);
    cudaMemsetAsync(h->adj, 0, NS * sizeof(float), h->stream);
  }
  if (h->P.tool) {
    std::vector<float> p0(7 * h->S, 0.0f);
    for (int s = 0; s < h->S; ++s) {
      p0[7 * s + 0] = p0[7 * s + 1] = p0[7 * s + 2] = -10.0f;  // far away until set
      p0[7 * s + 3] = 1.0f;
    }
    cudaMemcpy(h->pose0, p0.data(), sizeof(float) * p0.size(), cudaMemcpyHostToDevice);
    cudaMemsetAsync(h->actions, 0, sizeof(float) * h->S * h->n_act_max * 6, h->stream);
    h->n_actions = h->n_act_max;
    launch_tool_forward(h->P, h->pose0, h->actions, h->n_actions, h->spa, h->max_steps, h->max_steps,
                        h->poses, h->stream);
  }
  restart(h);
  sim_status st = check_err(h, "sim_create");
  if (st != SIM_OK) {
    sim_destroy(h);
    return st;
  }
  *out = h;
  return SIM_OK;
}

sim_status sim_set_particles(sim_h h, int scene, const float* x, const float* v, const uint8_t* mat,
                             int on_device) {
  if (!h) return SIM_E_ARG;
  int lo, cnt;
  if (!scene_range(h, scene, &lo, &cnt)) return fail(h, SIM_E_ARG, "sim_set_particles: bad scene");
  if (cnt > 0 && (!x || !v || !mat)) return fail(h, SIM_E_ARG, "sim_set_particles: null pointer");
  const int N = h->N;
  // staging in the N x 24 rows buffer: x at 0, v at 3N, material bytes at 6N
  float* stage = h->rows;
  uint8_t* mstage = reinterpret_cast<uint8_t*>(stage + (size_t)6 * N);
  cudaError_t e = to_device(h, stage, x, sizeof(float) * 3 * cnt, on_device);
  if (e == cudaSuccess) e = to_device(h, stage + (size_t)3 * N, v, sizeof(float) * 3 * cnt, on_device);
  if (e == cudaSuccess) e = to_device(h, mstage, mat, cnt, on_device);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_set_particles");
  cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
  // rows -> SoA fields of X0 at [lo, lo + cnt); C = 0, F = I, material tags
  launch_gather_rows(stage, h->X0 + lo, nullptr, cnt, 3, 0, N, 0, h->stream);
  launch_gather_rows(stage + (size_t)3 * N, h->X0 + (size_t)3 * N + lo, nullptr, cnt, 3, 0, N, 0, h->stream);
  launch_init_particles(h->X0, h->tag0, mstage, lo, cnt, N, h->cfg.n_materials, h->err, h->stream);
  h->launches += cnt > 0 ? 3 : 0;
  // water / other materials split of all scenes (the sort puts the water first)
  launch_count_water(h->P, h->tag0, h->nwater, h->stream);
  h->launches += N > 0 ? 1 : 0;
  if (h->rigid) {
    // rest shape of the scene's rigid objects: these positions
    launch_rigid_rest(h->P, h->X0, h->tag0, scene, lo, cnt, h->rb, h->stream);
    h->launches += cnt > 0 ? 4 : 0;
  }
  int flag = 0, nw = 0;
  e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemcpy(&flag, h->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&nw, h->nwater, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_set_particles");
  if (flag & kErrArg) {
    h->initialized = false;
    return fail(h, SIM_E_ARG, "sim_set_particles: material index out of range");
  }
  if (nw != h->P.Nl) {
    // the kernels' slot layout changed: captured graphs hold the old one
    h->P.Nl = nw;
    h->P.Ns = N - nw;
    drop_graphs(h);
  }
  restart(h);
  h->initialized = true;
  return check_err(h, "sim_set_particles");
}

sim_status sim_set_state(sim_h h, int scene, const float* x, const float* v, const float* C, const float* F,
                         const uint8_t* mat, int on_device) {
  sim_status st = sim_set_particles(h, scene, x, v, mat, on_device);
  if (st != SIM_OK || (!C && !F)) return st;
  int lo, cnt;
  scene_range(h, scene, &lo, &cnt);
  const int N = h->N;
  // rows -> SoA: C at fields 6..14, F at 15..23 (a liquid keeps F[0] = J)
  const float* src[2] = {C, F};
  for (int f = 0; f < 2; ++f) {
    if (!src[f] || cnt == 0) continue;
    cudaError_t e = to_device(h, h->rows, src[f], sizeof(float) * 9 * cnt, on_device);
    if (e != cudaSuccess) return cuda_fail(h, e, "sim_set_state");
    launch_gather_rows(h->rows, h->X0 + (size_t)(6 + 9 * f) * N + lo, nullptr, cnt, 9, 0, N, 0, h->stream);
    h->launches += 1;
  }
  restart(h);
  return check_err(h, "sim_set_state");
}

sim_status sim_set_tool(sim_h h, int scene, const float* pose0, const float* actions, int n_actions,
                        int on_device) {
  if (!h) return SIM_E_ARG;
  if (!h->P.tool) return fail(h, SIM_E_STATE, "sim_set_tool: tool disabled in the config");
  if (n_actions < 1 || n_actions > h->n_act_max || !pose0 || !actions)
    return fail(h, SIM_E_ARG, "sim_set_tool: bad arguments (n_actions must be in [1, ceil(max_steps/spa)])");
  int s0 = scene, ns = 1;
  if (scene == -1) {
    s0 = 0;
    ns = h->S;
  } else if (scene < 0 || scene >= h->S) {
    return fail(h, SIM_E_ARG, "sim_set_tool: bad scene");
  }
  if (ns != h->S && n_actions != h->n_actions)
    return fail(h, SIM_E_ARG, "sim_set_tool: all scenes share one action count");
  if (ns == h->S && n_actions != h->n_actions) {
    cudaMemsetAsync(h->actions, 0, sizeof(float) * h->S * h->n_act_max * 6, h->stream);
    h->n_actions = n_actions;
  }
  cudaError_t e = to_device(h, h->pose0 + 7 * s0, pose0, sizeof(float) * 7 * ns, on_device);
  if (e == cudaSuccess)
    e = to_device(h, h->actions + (size_t)s0 * n_actions * 6, actions, sizeof(float) * ns * n_actions * 6,
                  on_device);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_set_tool");
  launch_tool_forward(h->P, h->pose0, h->actions, h->n_actions, h->spa, h->max_steps, h->max_steps,
                      h->poses, h->stream);
  h->launches += 1;
  h->tool_set = true;
  restart(h);
  return check_err(h, "sim_set_tool");
}

int sim_current_step(sim_h h) { return h ? h->step : -1; }

// After a forward that kept chunks: a compact buffer whose steps outgrew its
// capacity (bit b of *ovf) holds an incomplete grid copy, so that chunk and
// every earlier one are left to the backward's recompute.
static sim_status drop_overflowed_chunks(sim_h h) {
  if (!h->ovf || h->rec_from < 0 || h->rec_from >= h->n_ckpt) return SIM_OK;
  int bits = 0;
  cudaError_t e = cudaMemcpy(&bits, h->ovf, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_step");
  int from = h->rec_from;
  for (int c = h->rec_from; c < h->n_ckpt; ++c) {
    const int b = h->n_ckpt - 1 - c;
    if (h->compact[b] && (bits & (1 << b))) from = c + 1;
  }
  h->rec_from = from;
  return SIM_OK;
}

static sim_status step_impl(sim_h h, int n_steps);

sim_status sim_step(sim_h h, int n_steps) {
  const sim_status st = step_impl(h, n_steps);
  return st == SIM_OK ? drop_overflowed_chunks(h) : st;
}

static sim_status step_impl(sim_h h, int n_steps) {
  if (!h) return SIM_E_ARG;
  if (n_steps < 0) return fail(h, SIM_E_ARG, "sim_step: negative step count");
  if (!h->initialized) return fail(h, SIM_E_STATE, "sim_step: no particles set");
  if ((h->k > 0 || h->P.tool) && h->step + n_steps > h->max_steps)
    return fail(h, SIM_E_STATE, "sim_step: trajectory would exceed max_steps");
  if (n_steps == 0) return check_err(h, "sim_step");
  {
    const sim_status cs = ensure_chunk_buffers(h);
    if (cs != SIM_OK) return cs;
  }
  if (!h->graphs || h->prof) {
    enqueue_steps(h, n_steps, h->stream);
    return check_err(h, "sim_step");
  }
  for (auto& g : h->fwd_graphs) {
    if (g.start == h->step && g.n == n_steps && g.W == h->W && g.W2 == h->W2 && g.tag == h->tag_cur &&
        g.pid == h->pid_cur && g.need_sort == h->need_sort) {
      cudaError_t e = cudaGraphLaunch(g.exec, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "sim_step");
      h->W = g.W_after;
      h->W2 = g.W2_after;
      h->tag_cur = g.tag_after;
      h->pid_cur = g.pid_after;
      h->need_sort = false;
      h->step += n_steps;
      h->rec_from = g.rec_from_after;
      h->launches += g.launches;
      return check_err(h, "sim_step");
    }
  }
  mpm_sim::FwdGraph g{h->step, n_steps, h->W, h->W2, h->tag_cur, h->pid_cur, h->need_sort, nullptr,
                      nullptr, nullptr, nullptr, nullptr, -1, 0};
  const long long l0 = h->launches;
  // host bookkeeping runs during the capture; keep a copy in case it fails
  float *W = h->W, *W2 = h->W2;
  uint32_t* tag = h->tag_cur;
  int* pid = h->pid_cur;
  const int step0 = h->step;
  const bool ns = h->need_sort;
  const int lr = h->rec_from;
  g.exec = capture(h, [&](cudaStream_t cs) { enqueue_steps(h, n_steps, cs); });
  if (!g.exec) {
    h->W = W;
    h->W2 = W2;
    h->tag_cur = tag;
    h->pid_cur = pid;
    h->step = step0;
    h->need_sort = ns;
    h->rec_from = lr;
    h->launches = l0;
    h->graphs = false;
    enqueue_steps(h, n_steps, h->stream);
    return check_err(h, "sim_step");
  }
  g.W_after = h->W;
  g.W2_after = h->W2;
  g.tag_after = h->tag_cur;
  g.pid_after = h->pid_cur;
  g.rec_from_after = h->rec_from;
  g.launches = h->launches - l0;
  if (h->fwd_graphs.size() >= kMaxGraphs) {
    cudaGraphExecDestroy(h->fwd_graphs.front().exec);
    h->fwd_graphs.erase(h->fwd_graphs.begin());
  }
  h->fwd_graphs.push_back(g);
  cudaError_t e = cudaGraphLaunch(g.exec, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_step");
  return check_err(h, "sim_step");
}

sim_status sim_get_state(sim_h h, int scene, int step, float* x, float* v, float* C, float* F,
                         int on_device) {
  if (!h) return SIM_E_ARG;
  if (step < -1) return fail(h, SIM_E_ARG, "sim_get_state: step must be -1 (current) or >= 0");
  int lo, cnt;
  if (!scene_range(h, scene, &lo, &cnt)) return fail(h, SIM_E_ARG, "sim_get_state: bad scene");
  const int N = h->N;
  const int t = step < 0 ? h->step : step;
  // the retained states: the current one, the initial one (caller order) and
  // the checkpoints c*k before the current step (checkpoint order)
  const float* src = nullptr;
  const int* pid = nullptr;
  int c = 0;
  if (t == h->step) {
    src = h->W;
    pid = h->pid_cur;
  } else if (t == 0) {
    src = h->X0;
  } else if (retained_checkpoint(h, t, &c)) {
    src = ck_state(h, c);
    pid = ck_pids(h, c);
  } else {
    return fail(h, SIM_E_STATE,
                "sim_get_state: the state of step " + std::to_string(t) +
                    " is not retained (retained: step 0, the current step and the checkpoint steps before it)");
  }
  // rows (caller layout, all particles): x3 v3 C9 F9 per particle
  launch_gather_rows(src, h->rows, pid, N, kStateFields, N, 0, 1, h->stream);
  h->launches += N > 0 ? 1 : 0;
  std::vector<float> host;
  std::vector<uint32_t> tags;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return cuda_fail(h, cudaGetLastError(), "sim_get_state");
  host.resize((size_t)cnt * kStateFields);
  tags.resize(cnt);
  cudaError_t e = cudaMemcpy(host.data(), h->rows + (size_t)lo * kStateFields,
                             sizeof(float) * host.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && cnt) e = cudaMemcpy(tags.data(), h->tag0 + lo, sizeof(uint32_t) * cnt, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_get_state");
  std::vector<float> ox(x ? 3 * (size_t)cnt : 0), ov(v ? 3 * (size_t)cnt : 0), oC(C ? 9 * (size_t)cnt : 0),
      oF(F ? 9 * (size_t)cnt : 0);
  for (int i = 0; i < cnt; ++i) {
    const float* r = host.data() + (size_t)i * kStateFields;
    bool liquid = is_liquid(h->P.mat[tag_mat(tags[i])].kind);
    for (int c = 0; c < 3; ++c) {
      if (x) ox[3 * i + c] = r[c];
      if (v) ov[3 * i + c] = r[3 + c];
    }
    for (int c = 0; c < 9; ++c) {
      if (C) oC[9 * i + c] = r[6 + c];
      if (F) oF[9 * i + c] = liquid ? (c == 0 ? r[15] : ((c % 4 == 0) ? 1.0f : 0.0f)) : r[15 + c];
    }
  }
  struct {
    float* dst;
    std::vector<float>* src;
  } outs[4] = {{x, &ox}, {v, &ov}, {C, &oC}, {F, &oF}};
  for (auto& o : outs) {
    if (!o.dst) continue;
    e = on_device ? cudaMemcpy(o.dst, o.src->data(), sizeof(float) * o.src->size(), cudaMemcpyHostToDevice)
                  : (std::memcpy(o.dst, o.src->data(), sizeof(float) * o.src->size()), cudaSuccess);
    if (e != cudaSuccess) return cuda_fail(h, e, "sim_get_state");
  }
  return SIM_OK;
}

sim_status sim_get_tool_pose(sim_h h, int scene, int step, float* pose, int on_device) {
  if (!h) return SIM_E_ARG;
  if (!h->P.tool) return fail(h, SIM_E_STATE, "sim_get_tool_pose: tool disabled in the config");
  if (!pose || step < 0 || step >= h->max_steps)
    return fail(h, SIM_E_ARG, "sim_get_tool_pose: need pose and 0 <= step < max_steps");
  int s0 = scene, ns = 1;
  if (scene == -1) {
    s0 = 0;
    ns = h->S;
  } else if (scene < 0 || scene >= h->S) {
    return fail(h, SIM_E_ARG, "sim_get_tool_pose: bad scene");
  }
  // pose records are [scene][step][kToolFields]: one strided copy over the scenes
  const size_t rec = sizeof(float) * kToolFields;
  cudaError_t e = cudaMemcpy2DAsync(pose, rec, h->poses + ((size_t)s0 * h->max_steps + step) * kToolFields,
                                    rec * h->max_steps, rec, ns,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_get_tool_pose");
  return check_err(h, "sim_get_tool_pose");
}

sim_status sim_add_loss_grad(sim_h h, int scene, int step, const float* dLdx, const float* dLdv,
                             int on_device) {
  if (!h) return SIM_E_ARG;
  const float* srcs[2] = {dLdx, dLdv};
  const int field[2] = {0, 3}, ncomp[2] = {3, 3};
  return add_seeds(h, "sim_add_loss_grad", scene, step, srcs, field, ncomp, 2, on_device);
}

sim_status sim_add_state_grad(sim_h h, int scene, int step, const float* dLdx, const float* dLdv,
                              const float* dLdC, int on_device) {
  if (!h) return SIM_E_ARG;
  const float* srcs[3] = {dLdx, dLdv, dLdC};
  const int field[3] = {0, 3, 6}, ncomp[3] = {3, 3, 9};
  return add_seeds(h, "sim_add_state_grad", scene, step, srcs, field, ncomp, 3, on_device);
}

sim_status sim_position_loss(sim_h h, int scene, int step, const float* target, float weight,
                             double* loss_out) {
  if (!h) return SIM_E_ARG;
  if (!target || !loss_out) return fail(h, SIM_E_ARG, "sim_position_loss: null pointer");
  if (scene < -1 || scene >= h->S) return fail(h, SIM_E_ARG, "sim_position_loss: bad scene");
  LossSite site;
  sim_status st = loss_site(h, "sim_position_loss", step, &site);
  if (st != SIM_OK) return st;
  cudaMemsetAsync(h->dloss, 0, sizeof(double) * h->S, h->stream);
  {
    Prof pr(h, "loss");
    launch_position_loss(h->P, site.st, site.tag, scene, target[0], target[1], target[2], weight, site.grad,
                         h->dloss, h->stream);
  }
  h->launches += h->N > 0 ? 1 : 0;
  finish_loss_site(h, site);
  int nout = scene < 0 ? h->S : 1;
  cudaError_t e = cudaMemcpyAsync(loss_out, h->dloss, sizeof(double) * nout, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_position_loss");
  return check_err(h, "sim_position_loss");
}

sim_status sim_grid_mass_loss(sim_h h, int scene, int step, const float* target_mass, const float* target_dist,
                              float total_mass, int on_device, double* loss_out) {
  if (!h) return SIM_E_ARG;
  if (scene < 0 || scene >= h->S || !target_mass || !target_dist || !loss_out || !(total_mass > 0.0f))
    return fail(h, SIM_E_ARG, "sim_grid_mass_loss: bad arguments");
  const long long n3 = h->P.n3;
  LossSite site;
  sim_status st = loss_site(h, "sim_grid_mass_loss", step, &site);
  if (st != SIM_OK) return st;
  if (!h->lm) {
    if (!(dalloc(h, &h->lm, n3) && dalloc(h, &h->ltm, n3) && dalloc(h, &h->ltd, n3) && dalloc(h, &h->ldm, n3)))
      return fail(h, SIM_E_OOM, "sim_grid_mass_loss: out of device memory");
  }
  cudaError_t e = to_device(h, h->ltm, target_mass, sizeof(float) * n3, on_device);
  if (e == cudaSuccess) e = to_device(h, h->ltd, target_dist, sizeof(float) * n3, on_device);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_grid_mass_loss");
  cudaMemsetAsync(h->lm, 0, sizeof(float) * n3, h->stream);
  cudaMemsetAsync(h->dloss, 0, sizeof(double), h->stream);
  {
    Prof pr(h, "loss");
    launch_mass_scatter(h->P, site.st, site.tag, scene, h->lm, h->stream);
    launch_mass_loss_nodes(n3, h->lm, h->ltm, h->ltd, 1.0f / total_mass, h->ldm, h->dloss, h->stream);
    launch_mass_loss_grad(h->P, site.st, site.tag, scene, h->ldm, site.grad, h->stream);
  }
  h->launches += h->N > 0 ? 3 : 1;
  finish_loss_site(h, site);
  e = cudaMemcpyAsync(loss_out, h->dloss, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_grid_mass_loss");
  return check_err(h, "sim_grid_mass_loss");
}

// Neighbour arrays of the current positions for the particles of `scene`
// (caller range [lo, lo + cnt)): cell bins, then positions with the weights
// c = exp(-ell / tau) (and the gradients g, if given) in bin order. ell and g
// are staged in the rows buffer (ell at 0, g at N, 3 x cnt floats).
static sim_status nbr_prepare(sim_h h, const char* where, int scene, const float* ell, const float* g, float radius,
                       float tau, int on_device, int* lo, int* cnt) {
  if (!scene_range(h, scene, lo, cnt)) return fail(h, SIM_E_ARG, std::string(where) + ": bad scene");
  if (!ell || !(radius > 0.0f) || radius > h->P.dx * 1.0001f || !(tau > 0.0f))
    return fail(h, SIM_E_ARG, std::string(where) + ": need ell, 0 < radius <= 1 / grid_n and tau > 0");
  const int N = h->N;
  if (!h->nb.pk) {
    if (!(dalloc(h, &h->nb.pk, N) && dalloc(h, &h->nb.pg, N) && dalloc(h, &h->nb.sidx, N)))
      return fail(h, SIM_E_OOM, std::string(where) + ": out of device memory");
  }
  float* s_ell = h->rows;
  float* s_g = h->rows + N;
  cudaError_t e = to_device(h, s_ell, ell, sizeof(float) * (*cnt), on_device);
  if (e == cudaSuccess && g) e = to_device(h, s_g, g, sizeof(float) * 3 * (*cnt), on_device);
  if (e != cudaSuccess) return cuda_fail(h, e, where);
  launch_bin(h->P, h->W, h->tag_cur, h->sb, h->stream);
  launch_nbr_pack(h->P, h->W, h->pid_cur, h->sb, s_ell, g ? s_g : nullptr, *lo, *cnt, tau, h->nb, h->stream);
  h->launches += N > 0 ? 6 : 3;
  return SIM_OK;
}

sim_status sim_attraction_loss(sim_h h, int scene, const float* ell, float radius, float tau, float weight,
                               int on_device, double* loss_out) {
  if (!h) return SIM_E_ARG;
  if (!loss_out) return fail(h, SIM_E_ARG, "sim_attraction_loss: null loss_out");
  if (h->k <= 0) return fail(h, SIM_E_STATE, "sim_attraction_loss: checkpointing is off (forward only)");
  if (h->step == 0) return fail(h, SIM_E_STATE, "sim_attraction_loss: no step taken");
  int lo, cnt;
  sim_status st = nbr_prepare(h, "sim_attraction_loss", scene, ell, nullptr, radius, tau, on_device, &lo, &cnt);
  if (st != SIM_OK) return st;
  cudaMemsetAsync(h->dloss, 0, sizeof(double), h->stream);
  {
    Prof pr(h, "attraction");
    float* seed = seed_buffer(h, h->step);
    if (!seed) return fail(h, SIM_E_OOM, "sim_attraction_loss: out of device memory");
    launch_attraction(h->P, h->tag_cur, h->sb, h->nb, radius, weight, seed, h->dloss, h->stream);
  }
  h->launches += h->N > 0 ? 1 : 0;
  cudaError_t e = cudaMemcpyAsync(loss_out, h->dloss, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_attraction_loss");
  return check_err(h, "sim_attraction_loss");
}

sim_status sim_share_gradients(sim_h h, int scene, const float* ell, float radius, float tau, const float* g,
                               float* out, int on_device) {
  if (!h) return SIM_E_ARG;
  if (!g || !out) return fail(h, SIM_E_ARG, "sim_share_gradients: null g or out");
  int lo, cnt;
  sim_status st = nbr_prepare(h, "sim_share_gradients", scene, ell, g, radius, tau, on_device, &lo, &cnt);
  if (st != SIM_OK) return st;
  float* s_out = h->rows + (size_t)4 * h->N;
  {
    Prof pr(h, "share");
    launch_share(h->P, h->tag_cur, h->pid_cur, h->sb, h->nb, radius, lo, s_out, h->stream);
  }
  h->launches += h->N > 0 ? 1 : 0;
  cudaError_t e = to_caller(h, out, s_out, sizeof(float) * 3 * cnt, on_device);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_share_gradients");
  return check_err(h, "sim_share_gradients");
}

sim_status sim_backward(sim_h h, float* dLdx0, float* dLdv0, float* dLdactions, int on_device) {
  if (!h) return SIM_E_ARG;
  if (h->k <= 0) return fail(h, SIM_E_STATE, "sim_backward: checkpointing is off (forward only)");
  if (h->step == 0) return fail(h, SIM_E_STATE, "sim_backward: no step taken");
  const int T = h->step, K = h->k, N = h->N;
  const Params& P = h->P;
  // Device work of the reverse sweep on stream s (forks to rstream for the
  // overlapped recompute and joins back): ends with the adjoint of the initial
  // state in caller order in `rows`, the action gradients in `action_grad`,
  // and the adjoint state cleared.
  const bool overlap = h->nbuf >= 2 && !h->prof;
  // the forward that reached max_steps left its last chunks [rec_from, nch)
  // in the buffers their sweeps read (rec_from = nch: every chunk is recomputed)
  const int nch_all = (T + K - 1) / K;
  // (later than the forward's first kept chunk when a compact buffer overflowed)
  const int rec_from = (h->rec_from >= 0 && T == h->max_steps && h->rec_from >= h->n_ckpt - recorded_chunks(h))
                           ? std::min(h->rec_from, nch_all)
                           : nch_all;
  // steps whose loss seeds the sweep adds into the adjoint state (and clears)
  const std::vector<int> seeded(h->seeded.begin(), h->seeded.end());
  auto has_seed = [&](int t) { return h->seeded.count(t) > 0; };
  auto inject = [&](int t, cudaStream_t st) {
    if (!has_seed(t)) return;
    Prof pr(h, "seed", st);
    launch_add_fields(h->adj, h->seed_buf[t], (long long)kSeedFields * N, 1, st);
    h->launches += N > 0 ? 1 : 0;
  };
  auto enqueue = [&](cudaStream_t s_in) {
    // with the overlapped recompute the sweep (the critical path) runs on the
    // highest-priority stream and the recompute on the lowest, so that the
    // recompute's CTAs fill the SMs around the sweep instead of delaying it
    cudaStream_t s = s_in;
    if (overlap) {
      cudaEventRecord(h->ev_start, s_in);
      cudaStreamWaitEvent(h->hstream, h->ev_start, 0);
      s = h->hstream;
    }
    if (h->P.tool) cudaMemsetAsync(h->tool_grad, 0, sizeof(float) * h->S * h->max_steps * kToolGradFields, s);
    const int nch = (T + K - 1) / K;
    auto recompute = [&](int c, int b, cudaStream_t rs) { recompute_chunk(h, c, b, T, rs); };
    auto buf = [&](int c) { return chunk_buffer(h, c, nch, rec_from); };
    // pipeline: the recompute of chunk c-1 (stream rs) overlaps the reverse
    // sweep of chunk c (caller stream); events keep a buffer from being
    // overwritten while an earlier sweep still reads it (swept[b]: a sweep in
    // buffer b was enqueued by this backward) and a sweep from starting before
    // its chunk's recompute has finished
    bool swept[kMaxBuffers] = {};
    cudaStream_t rs = overlap ? h->rstream : s;
    if (overlap) cudaStreamWaitEvent(rs, h->ev_start, 0);
    if (rec_from > nch - 1) {
      recompute(nch - 1, buf(nch - 1), rs);
      if (overlap) cudaEventRecord(h->ev_rec[buf(nch - 1)], rs);
    }
    for (int c = nch - 1; c >= 0; --c) {
      const int b = buf(c);
      if (overlap && c >= 1 && c - 1 < rec_from) {
        const int bp = buf(c - 1);
        if (swept[bp]) cudaStreamWaitEvent(rs, h->ev_adj[bp], 0);
        recompute(c - 1, bp, rs);
        cudaEventRecord(h->ev_rec[bp], rs);
      }
      if (overlap && c < rec_from) cudaStreamWaitEvent(s, h->ev_rec[b], 0);
      const int s0 = c * K, L = std::min(T, s0 + K) - s0;
      const uint32_t* tag = ck_tags(h, c);
      auto state = [&](int j) -> const float* { return j == 0 ? ck_state(h, c) : chunk_state(h, b, j, L); };
      // reverse sweep: G2P adjoint of the last step, then per step the grid
      // adjoint and the P2G adjoint of step n fused with the G2P adjoint of
      // step n - 1, ending with the P2G adjoint of the chunk's first step.
      // The seeds of the state at step s0 + j join the adjoint state once it
      // is complete (after the P2G adjoint of that step; for j = L, which is
      // the first state of the next chunk, at the start of this sweep) and
      // before the G2P adjoint of step s0 + j - 1 reads it; a seeded step
      // runs the two adjoints unfused to make room for that.
      const int* pids = ck_pids(h, c);
      inject(s0 + L, s);
      stage_rigid_adj(h, tag, pids, rig_step(h, b, L - 1), s);
      // a compact buffer's grid of step j is expanded into gscr before the
      // G2P adjoint of step j + 1 reads it; it stays there for the grid
      // adjoint of step j
      stage_expand(h, b, L - 1, s);
      {
        GridBuffers g = step_grid(h, b, L - 1);
        Prof pr(h, "g2p_adj", s);
        launch_g2p_adj(P, h->tu, state(L - 1), state(L), tag, g.Fp, h->adj, g.gv, h->gadj_v, s);
        h->launches += N > 0 ? 1 : 0;
      }
      for (int j = L - 1; j >= 0; --j) {
        GridBuffers g = step_grid(h, b, j);
        {
          Prof pr(h, "grid_adj", s);
          launch_grid_adj(P, h->tu, g, h->gadj_v, h->gadj_m, h->poses, h->tool_grad, s0 + j, h->max_steps, s);
          h->launches += 1;
        }
        if (j > 0 && (!h->tu.fuse_adjoint || h->rigid || has_seed(s0 + j))) {
          GridBuffers gp = step_grid(h, b, j - 1);
          {
            Prof pr(h, "p2g_adj", s);
            launch_p2g_adj(P, h->tu, state(j), state(j + 1), tag, g.svd, h->adj, h->gadj_m, s);
          }
          inject(s0 + j, s);
          stage_rigid_adj(h, tag, pids, rig_step(h, b, j - 1), s);
          stage_expand(h, b, j - 1, s);
          {
            Prof pr(h, "g2p_adj", s);
            launch_g2p_adj(P, h->tu, state(j - 1), state(j), tag, gp.Fp, h->adj, gp.gv, h->gadj_v, s);
          }
          h->launches += N > 0 ? 2 : 0;
        } else if (j > 0) {
          GridBuffers gp = step_grid(h, b, j - 1);
          stage_expand(h, b, j - 1, s);
          Prof pr(h, "adj_fused", s);
          launch_adj_fused(P, h->tu, state(j - 1), state(j), state(j + 1), tag, g.svd, gp.Fp, h->adj,
                           h->gadj_m, gp.gv, h->gadj_v, s);
          h->launches += N > 0 ? 1 : 0;
        } else {
          Prof pr(h, "p2g_adj", s);
          launch_p2g_adj(P, h->tu, state(0), state(1), tag, g.svd, h->adj, h->gadj_m, s);
          h->launches += N > 0 ? 1 : 0;
        }
      }
      if (overlap) {
        cudaEventRecord(h->ev_adj[b], s);
        swept[b] = true;
      }
      if (!overlap && c > 0 && c - 1 < rec_from) {
        // single buffer: the next chunk's recompute follows this sweep in order
        recompute(c - 1, buf(c - 1), s);
      }
      if (c > 0) {
        // adjoint of the re-sort at step s0: order of checkpoint c -> order of chunk c - 1
        Prof pr(h, "permute", s);
        launch_permute_state(h->adj, h->rows, ck_pids(h, c), ck_pids(h, c - 1), h->inv, N, kStateFields, s);
        cudaMemcpyAsync(h->adj, h->rows, state_floats(h) * sizeof(float), cudaMemcpyDeviceToDevice, s);
        h->launches += N > 0 ? 2 : 0;
      }
    }
    launch_gather_rows(h->adj, h->rows, ck_pids(h, 0), N, kStateFields, N, 0, 1, s);
    h->launches += N > 0 ? 1 : 0;
    if (h->P.tool) {
      cudaMemsetAsync(h->action_grad, 0, sizeof(float) * h->S * h->n_actions * 6, s);
      {
        Prof pr(h, "tool_adj", s);
        launch_tool_backward(P, h->pose0, h->actions, h->n_actions, h->spa, T, h->max_steps, h->poses,
                             h->tool_grad, h->action_grad, s);
      }
      h->launches += 1;
    }
    cudaMemsetAsync(h->adj, 0, state_floats(h) * sizeof(float), s);
    if (overlap) {
      cudaEventRecord(h->ev_join, s);
      cudaStreamWaitEvent(s_in, h->ev_join, 0);
    }
  };
  bool done = false;
  if (h->graphs && !h->prof) {
    for (auto& g : h->bwd_graphs)
      if (g.T == T && g.n_actions == h->n_actions && g.rec_from == rec_from && g.seeded == seeded) {
        cudaError_t e = cudaGraphLaunch(g.exec, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "sim_backward");
        h->launches += g.launches;
        done = true;
        break;
      }
    if (!done) {
      const long long l0 = h->launches;
      cudaGraphExec_t exec = capture(h, enqueue, overlap);
      if (exec) {
        if (h->bwd_graphs.size() >= kMaxGraphs) {
          cudaGraphExecDestroy(h->bwd_graphs.front().exec);
          h->bwd_graphs.erase(h->bwd_graphs.begin());
        }
        h->bwd_graphs.push_back({T, h->n_actions, rec_from, seeded, exec, h->launches - l0});
        cudaError_t e = cudaGraphLaunch(exec, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "sim_backward");
        done = true;
      } else {
        h->launches = l0;
        h->graphs = false;
      }
    }
  }
  if (!done) enqueue(h->stream);
  h->rec_from = -1;  // the sweep's recomputes reuse the chunk buffers
  h->seeded.clear();   // the sweep added and cleared every pending seed
  // outputs in caller order
  sim_status st = check_err(h, "sim_backward");
  if (st != SIM_OK) return st;
  cudaError_t e = cudaSuccess;
  if ((dLdx0 || dLdv0) && N > 0) {
    // rows holds the initial state's adjoint in caller order, kStateFields
    // floats per particle: x at 0..2, v at 3..5; one strided copy each
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t pitch = kStateFields * sizeof(float), w = 3 * sizeof(float);
    if (dLdx0) e = cudaMemcpy2DAsync(dLdx0, w, h->rows, pitch, w, N, kind, h->stream);
    if (e == cudaSuccess && dLdv0) e = cudaMemcpy2DAsync(dLdv0, w, h->rows + 3, pitch, w, N, kind, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sim_backward");
  }
  if (dLdactions && h->P.tool) {
    e = to_caller(h, dLdactions, h->action_grad, sizeof(float) * h->S * h->n_actions * 6, on_device);
    if (e != cudaSuccess) return cuda_fail(h, e, "sim_backward");
  }
  h->seeds = false;
  return check_err(h, "sim_backward");
}

long long sim_kernel_launches(sim_h h) { return h ? h->launches : -1; }

sim_status sim_set_launch(sim_h h, const int* choices) {
  if (!h || !choices) return SIM_E_ARG;
  if ((choices[0] != 128 && choices[0] != 256) ||
      (choices[1] != 128 && choices[1] != 256 && choices[1] != 512) ||
      (choices[2] != 1 && choices[2] != 2 && choices[2] != 4) || choices[3] < 1 ||
      (choices[4] != 0 && choices[4] != 1) || (choices[5] != 0 && choices[5] != 1) ||
      (choices[6] != 0 && choices[6] != 1) || (choices[7] != 3 && choices[7] != 4))
    return fail(h, SIM_E_ARG, "sim_set_launch: unsupported launch shape");
  if (choices[5] && !h->coop)
    return fail(h, SIM_E_ARG, "sim_set_launch: the device has no cooperative launch (persistent forward)");
  cudaStreamSynchronize(h->stream);
  h->tu.scatter_threads = choices[0];
  h->tu.gather_threads = choices[1];
  h->tu.grid_blocks = choices[2];
  h->resort = choices[3];
  h->tu.fuse_adjoint = choices[4];
  h->tu.persistent = choices[5];
  h->tu.stage_gather = choices[6];
  h->tu.scatter_ctas = choices[7];
  // captured graphs hold the old shapes
  for (auto& g : h->fwd_graphs) cudaGraphExecDestroy(g.exec);
  for (auto& g : h->bwd_graphs) cudaGraphExecDestroy(g.exec);
  h->fwd_graphs.clear();
  h->bwd_graphs.clear();
  return SIM_OK;
}

sim_status sim_autotune(sim_h h, int n_steps, int* choices) {
  if (!h) return SIM_E_ARG;
  if (!h->initialized) return fail(h, SIM_E_STATE, "sim_autotune: no particles set");
  if (h->seeds) return fail(h, SIM_E_STATE, "sim_autotune: loss gradients are pending");
  {
    const sim_status cs = ensure_chunk_buffers(h);
    if (cs != SIM_OK) return cs;
  }
  static std::mutex cache_lock;
  static std::map<std::string, std::pair<Tuning, int>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return cuda_fail(h, cudaGetLastError(), "sim_autotune");
  char key[512];
  std::snprintf(key, sizeof(key), "%s|N=%d|S=%d|n=%d|k=%d|tool=%d|mats=%d", prop.name, h->N, h->S, h->n, h->k,
                h->P.tool, h->P.n_mat);
  {
    std::lock_guard<std::mutex> g(cache_lock);
    auto it = cache.find(key);
    if (it != cache.end()) {
      int c[8] = {it->second.first.scatter_threads, it->second.first.gather_threads,
                  it->second.first.grid_blocks, it->second.second, it->second.first.fuse_adjoint,
                  it->second.first.persistent, it->second.first.stage_gather, it->second.first.scatter_ctas};
      sim_set_launch(h, c);
      restart(h);
      if (choices) {
        choices[0] = h->tu.scatter_threads;
        choices[1] = h->tu.gather_threads;
        choices[2] = h->tu.grid_blocks;
        choices[3] = h->resort;
        choices[4] = h->tu.fuse_adjoint;
        choices[5] = h->tu.persistent;
        choices[6] = h->tu.stage_gather;
        choices[7] = h->tu.scatter_ctas;
      }
      return SIM_OK;
    }
  }
  int n = n_steps > 0 ? n_steps : 10;
  if (h->k > 0 || h->P.tool) n = std::min(n, h->max_steps);
  const bool was_prof = h->prof;
  // time one trial: n steps forward (+ the reverse sweep in gradient mode); the
  // score is the summed event time of the kernels listed in `names`
  auto trial = [&](std::initializer_list<const char*> names) -> double {
    restart(h);
    sim_profile_enable(h, 1);
    enqueue_steps(h, n, h->stream);
    if (h->k > 0) {
      h->seeds = true;
      sim_status st = sim_backward(h, nullptr, nullptr, nullptr, 0);
      if (st != SIM_OK) return 1e30;
    }
    double t = 0.0;
    for (auto& r : h->prof_recs) {
      for (const char* nm : names)
        if (std::strcmp(nm, r.name) == 0) {
          float ms = 0.0f;
          cudaEventSynchronize(r.b);
          cudaEventElapsedTime(&ms, r.a, r.b);
          t += ms;
        }
    }
    if (check_err(h, "sim_autotune") != SIM_OK) return 1e30;
    return t;
  };
  const int st_c[2] = {128, 256}, ga_c[3] = {128, 256, 512}, gb_c[3] = {1, 2, 4};
  double best = 1e30;
  int pick = h->tu.scatter_threads;
  for (int c : st_c) {
    h->tu.scatter_threads = c;
    double t = trial({"p2g", "g2p2g", "g2p_adj", "adj_fused"});
    if (t < best) best = t, pick = c;
  }
  h->tu.scatter_threads = pick;
  if (h->tu.scatter_threads == 256) {
    // resident CTAs of the fused step and the G2P adjoint: 3 (80 registers)
    // or 4 (64 registers, some spills)
    best = 1e30;
    pick = h->tu.scatter_ctas;
    for (int c : {3, 4}) {
      h->tu.scatter_ctas = c;
      double t = trial({"p2g", "g2p2g", "g2p_adj", "adj_fused"});
      if (t < best) best = t, pick = c;
    }
    h->tu.scatter_ctas = pick;
  }
  best = 1e30;
  pick = h->tu.gather_threads;
  for (int c : ga_c) {
    h->tu.gather_threads = c;
    double t = trial({"g2p", "p2g_adj"});
    if (t < best) best = t, pick = c;
  }
  h->tu.gather_threads = pick;
  best = 1e30;
  pick = h->tu.grid_blocks;
  for (int c : gb_c) {
    h->tu.grid_blocks = c;
    double t = trial({"grid_update", "grid_adj"});
    if (t < best) best = t, pick = c;
  }
  h->tu.grid_blocks = pick;
  if (h->k > 0) {
    best = 1e30;
    pick = h->tu.fuse_adjoint;
    for (int c = 0; c < 2; ++c) {
      h->tu.fuse_adjoint = c;
      double t = trial({"adj_fused", "p2g_adj", "g2p_adj"});
      if (t < best) best = t, pick = c;
    }
    h->tu.fuse_adjoint = pick;
  }
  {
    // the fused G2P's gather from global memory or from a TMA-staged box
    best = 1e30;
    pick = h->tu.stage_gather;
    for (int c = 0; c < 2; ++c) {
      h->tu.stage_gather = c;
      double t = trial({"g2p2g"});
      if (c == 1 && !h->maps_ok) t = 1e30;
      if (t < best) best = t, pick = c;
    }
    h->tu.stage_gather = pick;
  }
  if (h->coop && !h->rigid) {
    // the forward's step loop: per-step kernels or one persistent launch per run
    best = 1e30;
    pick = h->tu.persistent;
    const int n_fwd = h->k > 0 ? std::min(n, h->k) : n;
    for (int c = 0; c < 2; ++c) {
      h->tu.persistent = c;
      restart(h);
      sim_profile_enable(h, 1);
      enqueue_steps(h, n_fwd, h->stream);
      double t = 0.0;
      for (auto& r : h->prof_recs) {
        for (const char* nm : {"p2g", "g2p2g", "grid_update", "g2p", "fwd_run"})
          if (std::strcmp(nm, r.name) == 0) {
            float ms = 0.0f;
            cudaEventSynchronize(r.b);
            cudaEventElapsedTime(&ms, r.a, r.b);
            t += ms;
          }
      }
      if (check_err(h, "sim_autotune") != SIM_OK || (c == 1 && !h->tu.persistent)) t = 1e30;
      if (t < best) best = t, pick = c;
    }
    h->tu.persistent = pick;
  }
  if (h->k == 0) {
    const int rs_c[4] = {4, 8, 16, 32};
    best = 1e30;
    pick = h->resort;
    for (int c : rs_c) {
      h->resort = c;
      double t = trial({"p2g", "g2p2g", "g2p", "grid_update", "sort"});
      if (t < best) best = t, pick = c;
    }
    h->resort = pick;
  }
  sim_profile_enable(h, was_prof ? 1 : 0);
  int final_choice[8] = {h->tu.scatter_threads, h->tu.gather_threads, h->tu.grid_blocks, h->resort,
                         h->tu.fuse_adjoint, h->tu.persistent, h->tu.stage_gather, h->tu.scatter_ctas};
  sim_set_launch(h, final_choice);
  restart(h);
  {
    std::lock_guard<std::mutex> g(cache_lock);
    cache[key] = {h->tu, h->resort};
  }
  if (choices) {
    choices[0] = h->tu.scatter_threads;
    choices[1] = h->tu.gather_threads;
    choices[2] = h->tu.grid_blocks;
    choices[3] = h->resort;
    choices[4] = h->tu.fuse_adjoint;
    choices[5] = h->tu.persistent;
    choices[6] = h->tu.stage_gather;
    choices[7] = h->tu.scatter_ctas;
  }
  return check_err(h, "sim_autotune");
}

sim_status sim_selftest_grid_barrier(int blocks, int extra_arrivals, int rounds, double timeout_ms,
                                     int* passed) {
  if (blocks < 1 || blocks > 4096 || extra_arrivals < 0 || rounds < 1 || !(timeout_ms > 0.0) ||
      timeout_ms > 60000.0 || !passed)
    return SIM_E_ARG;
  int dev = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
    cudaGetLastError();
    return SIM_E_CUDA;
  }
  unsigned* bar = nullptr;
  int* words = nullptr;  // err, passed
  if (cudaMalloc(&bar, 2 * sizeof(unsigned)) != cudaSuccess) return SIM_E_OOM;
  if (cudaMalloc(&words, 2 * sizeof(int)) != cudaSuccess) {
    cudaFree(bar);
    return SIM_E_OOM;
  }
  int host[2] = {0, 0};
  cudaError_t e = cudaMemset(words, 0, 2 * sizeof(int));
  if (e == cudaSuccess)
    e = launch_barrier_selftest(bar, blocks, unsigned(blocks + extra_arrivals), rounds, words,
                                (unsigned long long)(timeout_ms * 1e6), words + 1, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(host, words, 2 * sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(bar);
  cudaFree(words);
  if (e != cudaSuccess) return SIM_E_CUDA;
  *passed = host[1];
  return (host[0] & kErrTimeout) ? SIM_E_TIMEOUT : SIM_OK;
}

sim_status sim_sync(sim_h h) {
  if (!h) return SIM_E_ARG;
  return check_err(h, "sim_sync");
}

sim_status sim_profile_enable(sim_h h, int enable) {
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

sim_status sim_profile_read(sim_h h, int cap, const char** names, double* total_ms, long long* launches,
                            int* n_out) {
  if (!h || !n_out) return SIM_E_ARG;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "sim_profile_read");
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
    ct[i] += r.units;
  }
  *n_out = int(nm.size());
  for (int i = 0; i < cap && i < (int)nm.size(); ++i) {
    if (names) names[i] = nm[i];
    if (total_ms) total_ms[i] = ms[i];
    if (launches) launches[i] = ct[i];
  }
  return SIM_OK;
}

}  // extern "C"
