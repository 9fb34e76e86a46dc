// Serving layer: many simulations resident in one device-memory arena, advanced together.
//
// Each admitted request becomes a simulation (slot) whose workspace, steady-state
// snapshot and check partials are carved from the batch's arena (first fit).  A batch
// step is three launches whatever the number of slots, each over a work-list spanning all
// slots: the moments of every slot; ONE cooperative launch that runs the potential loops
// of all slots on chip (each slot synchronises only its own tiles and stops at its own
// sub-iteration count); the coupled pass of every slot.  The steps are captured in CUDA
// graphs of several steps.  All slots of a batch tile their potential loop alike (64 x
// rows tiles, rows fixed while any slot is live) and get the blocks of their own
// launches, so a request computes exactly the same numbers alone and in any mix.  The
// tile height and the steps per graph are the batch's schedule (ehd_batch_set_schedule,
// e.g. chosen by an autotuner).
//
// Admission needs a free slot, room in the arena and room in the co-resident tile
// capacity of the shared launch; otherwise EHD_ERR_BUSY and nothing changes.  Requests that
// arrive while others run are admitted between check windows (continuous batching); the
// host-side scheduler lives in the caller (see serve.py), this file provides the slots.
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "sim_internal.h"

using namespace ehd;

namespace {

constexpr int STEADY_THREADS = 256;
constexpr int STEPS_PER_GRAPH = 16;  // default; even: a multi-step graph ends on the copy it
                                     // began with

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

struct Slot {
  bool live = false;
  ehd_sim* sim = nullptr;
  size_t off = 0, bytes = 0;
  float* snap = nullptr;      // [3][N]: phi, ux, uy at the last check
  double* dpart = nullptr;    // [blocks][4]: per-block sums of the steady check
  int nblocks = 0;
  int64_t request_id = 0;
  int64_t steps = 0;
  int64_t iters = 0;
  int steady = 0;
  int have_snap = 0;
  int status = EHD_OK;
  double rel_phi = INFINITY, rel_u = INFINITY;
  int ntiles = 0;
};

// Relative change of phi and u since the snapshot, then a new snapshot; per-block FP64
// sums (phi: sum dphi^2, sum phi^2; u: sum |du|^2, sum |u|^2), reduced on the host in order.
template <bool HALF>
__global__ void __launch_bounds__(STEADY_THREADS)
    k_steady(KParams k, Pops pops, const float* __restrict__ hist, float* __restrict__ snap,
             int have_snap, double* __restrict__ dpart) {
  const int N = k.N;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  float a = 0.0f, b = 0.0f, c = 0.0f, d = 0.0f;
  if (idx < N) {
    const float phi = phi_of<HALF>(k, pops, idx);
    float mx = 0.0f, my = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float fi = ld_pop<HALF>(k, pops, 2, i, idx);
      mx += cx(i) * fi;
      my += cy(i) * fi;
    }
    const float rho = k.rho_v + k.drho * phi;
    const float ux = (mx + 0.5f * hist[4 * (size_t)N + idx]) / rho;
    const float uy = (my + 0.5f * hist[5 * (size_t)N + idx]) / rho;
    if (have_snap) {
      const float dp = phi - snap[idx];
      const float dx = ux - snap[(size_t)N + idx], dy = uy - snap[2 * (size_t)N + idx];
      a = dp * dp;
      c = dx * dx + dy * dy;
    }
    b = phi * phi;
    d = ux * ux + uy * uy;
    snap[idx] = phi;
    snap[(size_t)N + idx] = ux;
    snap[2 * (size_t)N + idx] = uy;
  }
  __shared__ double s[STEADY_THREADS / 32][4];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s[threadIdx.x >> 5][0] = a;
    s[threadIdx.x >> 5][1] = b;
    s[threadIdx.x >> 5][2] = c;
    s[threadIdx.x >> 5][3] = d;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int w = 0; w < STEADY_THREADS / 32; ++w)
      for (int j = 0; j < 4; ++j) t[j] += s[w][j];
    for (int j = 0; j < 4; ++j) dpart[(size_t)blockIdx.x * 4 + j] = t[j];
  }
}

}  // namespace

struct ehd_batch {
  cudaStream_t stream = nullptr;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  bool own_arena = false;
  size_t heap_start = 0;                 // after the device tables
  std::map<size_t, size_t> used;         // offset -> bytes
  std::vector<Slot> slots;
  int cur = 0;                           // population copy shared by every slot
  double steady_tol = 1e-6;
  int64_t step_cap = 300000;
  int rows = BATCH_ROWS;                 // tile height of every slot
  int steps_per_graph = STEPS_PER_GRAPH;
  int tile_capacity = 0;                 // co-resident CTAs of the shared potential launch
  int rthreads = 0;
  size_t rsmem = 0;
  int cap[3] = {0, 0, 0};                // tile capacity, threads and shared memory per
  int thr[3] = {0, 0, 0};                // choice of BATCH_ROW_CHOICES
  size_t smm[3] = {0, 0, 0};
  int tiles_used = 0;
  bool dirty = true;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};    // one step from copy c
  cudaGraphExec_t execm[2] = {nullptr, nullptr};   // steps_per_graph steps from copy c
  ResidentSlot* d_slots = nullptr;       // [max_slots]
  int2* d_work = nullptr;                // [largest tile capacity]
  StepSlot* d_step = nullptr;            // [max_slots]
  int2* d_mwork = nullptr;               // [mwork_cap]: moments blocks of all slots
  int2* d_cwork = nullptr;               // [cwork_cap]: coupled blocks of all slots
  int mwork_cap = 0, cwork_cap = 0;
  int64_t steps_run = 0;
  int64_t launches = 0;
};

namespace {

bool arena_alloc(ehd_batch* b, size_t bytes, size_t* off) {
  size_t at = b->heap_start;
  for (const auto& u : b->used) {
    if (u.first >= at + bytes) break;
    at = al256(u.first + u.second);
  }
  if (at + bytes > b->arena_bytes) return false;
  b->used[at] = bytes;
  *off = at;
  return true;
}

void arena_free(ehd_batch* b, size_t off) { b->used.erase(off); }

void destroy_batch_graphs(ehd_batch* b) {
  for (int c = 0; c < 2; ++c) {
    if (b->exec[c]) cudaGraphExecDestroy(b->exec[c]);
    if (b->execm[c]) cudaGraphExecDestroy(b->execm[c]);
    b->exec[c] = nullptr;
    b->execm[c] = nullptr;
  }
}

struct BatchLaunch {
  void* rfunc;
  int ntiles, rthreads;
  size_t rsmem;
  ResidentSlot* slots;
  int2* work;
  StepSlot* step;
  int2* mwork;
  int2* cwork;       // the FP32 slots' coupled blocks, then the FP16 slots'
  int nm, nc, nc16;  // nc16 of the nc items are of FP16 slots
};

// Appends one batch step from copy `cur` after `dep` (null: no dependency); its last node
// goes to `last`.
cudaError_t add_batch_step(cudaGraph_t g, const BatchLaunch& L, int cur,
                           const cudaGraphNode_t* dep, cudaGraphNode_t* last) {
  cudaGraphNode_t mn, rn;
  cudaError_t e = add_moments_batch_node(g, dep, dep ? 1 : 0, &mn, L.step, L.mwork, L.nm, cur);
  if (e != cudaSuccess) return e;
  ResidentSlot* slots = L.slots;
  int2* wk = L.work;
  void* args[] = {&slots, &wk};
  cudaKernelNodeParams p = {};
  p.func = L.rfunc;
  p.gridDim = dim3((unsigned)L.ntiles);
  p.blockDim = dim3(L.rthreads);
  p.sharedMemBytes = (unsigned)L.rsmem;
  p.kernelParams = args;
  if ((e = cudaGraphAddKernelNode(&rn, g, &mn, 1, &p)) != cudaSuccess) return e;
  cudaKernelNodeAttrValue v = {};
  v.cooperative = 1;
  if ((e = cudaGraphKernelNodeSetAttribute(rn, cudaLaunchAttributeCooperative, &v)) !=
      cudaSuccess)
    return e;
  // the coupled pass in one launch per storage precision present (the two touch
  // disjoint slots)
  const int n32 = L.nc - L.nc16;
  if (n32 > 0 && L.nc16 > 0) {
    cudaGraphNode_t c32;
    if ((e = add_coupled_batch_node(g, &rn, 1, &c32, L.step, L.cwork, n32, cur, false)) !=
        cudaSuccess)
      return e;
    return add_coupled_batch_node(g, &c32, 1, last, L.step, L.cwork + n32, L.nc16, cur, true);
  }
  return add_coupled_batch_node(g, &rn, 1, last, L.step, L.cwork, L.nc, cur, L.nc16 > 0);
}

// A graph of `nsteps` batch steps starting from copy `cur`, instantiated.
int build_batch_graph(const BatchLaunch& L, int cur, int nsteps, cudaGraphExec_t* out) {
  cudaGraph_t g;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return EHD_ERR_CUDA;
  cudaGraphNode_t last = nullptr;
  for (int k = 0; k < nsteps; ++k) {
    cudaGraphNode_t prev = last;
    if (add_batch_step(g, L, (cur + k) & 1, k ? &prev : nullptr, &last) != cudaSuccess) {
      cudaGraphDestroy(g);
      return EHD_ERR_CUDA;
    }
  }
  const cudaError_t e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e == cudaSuccess ? EHD_OK : EHD_ERR_CUDA;
}

// Builds the step graphs for the current set of live slots.
int rebuild(ehd_batch* b) {
  destroy_batch_graphs(b);
  b->dirty = false;
  std::vector<int> live;
  for (int i = 0; i < (int)b->slots.size(); ++i)
    if (b->slots[i].live) live.push_back(i);
  if (live.empty()) return EHD_OK;
  // device tables: per live slot its resident-loop view and its step view, and the work
  // lists of the three launches
  std::vector<ResidentSlot> rs(live.size());
  std::vector<StepSlot> ss(live.size());
  std::vector<int2> work, mwork, cwork, cwork16;
  for (size_t j = 0; j < live.size(); ++j) {
    ehd_sim* s = b->slots[live[j]].sim;
    ResidentSlot& r = rs[j];
    r.k = s->kp;
    r.rg = s->rg;
    r.h = s->b.h;
    r.aq = s->b.aq;
    r.exports = s->b.exports;
    r.rpartials = s->b.rpartials;
    r.ctl = s->b.ctl;
    const int nt = s->rg.ntx * s->rg.nty;
    for (int t = 0; t < nt; ++t) work.push_back(make_int2((int)j, t));
    StepSlot& q = ss[j];
    q.k = s->kp;
    q.b = s->b;
    q.tol = s->P.poisson_tol;
    q.min_iter = s->P.poisson_min_iter;
    q.max_iter = s->P.poisson_max_iter;
    q.fixed_iter = s->P.poisson_fixed_iter;
    q.quad = moments4_ok(s->kp) ? 1 : 0;
    q.mblocks = q.quad ? (s->kp.N / 4 + 255) / 256 : moments_blocks(s->kp.N);
    for (int t = 0; t < q.mblocks; ++t) mwork.push_back(make_int2((int)j, t));
    const int cb = (s->kp.N + 127) / 128;
    for (int t = 0; t < cb; ++t) (s->kp.half ? cwork16 : cwork).push_back(make_int2((int)j, t));
  }
  const int nc16 = (int)cwork16.size();
  cwork.insert(cwork.end(), cwork16.begin(), cwork16.end());
  if ((int)work.size() > b->tile_capacity || (int)mwork.size() > b->mwork_cap ||
      (int)cwork.size() > b->cwork_cap)
    return EHD_ERR_BUSY;
  if (cudaMemcpyAsync(b->d_slots, rs.data(), sizeof(ResidentSlot) * rs.size(),
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(b->d_work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess ||
      cudaMemcpyAsync(b->d_step, ss.data(), sizeof(StepSlot) * ss.size(), cudaMemcpyHostToDevice,
                      b->stream) != cudaSuccess ||
      cudaMemcpyAsync(b->d_mwork, mwork.data(), sizeof(int2) * mwork.size(),
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(b->d_cwork, cwork.data(), sizeof(int2) * cwork.size(),
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    return EHD_ERR_CUDA;
  BatchLaunch L;
  L.rfunc = (void*)resident_batch_kernel(b->rows);
  L.ntiles = (int)work.size();
  L.rthreads = b->rthreads;
  L.rsmem = b->rsmem;
  L.slots = b->d_slots;
  L.work = b->d_work;
  L.step = b->d_step;
  L.mwork = b->d_mwork;
  L.cwork = b->d_cwork;
  L.nm = (int)mwork.size();
  L.nc = (int)cwork.size();
  L.nc16 = nc16;
  for (int c = 0; c < 2; ++c) {
    int st = build_batch_graph(L, c, 1, &b->exec[c]);
    if (st == EHD_OK) st = build_batch_graph(L, c, b->steps_per_graph, &b->execm[c]);
    if (st != EHD_OK) {
      destroy_batch_graphs(b);
      b->dirty = true;
      return st;
    }
  }
  return EHD_OK;
}

}  // namespace

extern "C" {

int ehd_batch_create(size_t hbm_budget, int max_slots, double steady_tol, int64_t step_cap,
                     void* arena, void* stream, ehd_batch** out) {
  if (!out || max_slots < 1 || hbm_budget < (1u << 20) || !(steady_tol > 0) || step_cap < 1)
    return EHD_ERR_INVALID_ARG;
  *out = nullptr;
  ehd_batch* b = new (std::nothrow) ehd_batch();
  if (!b) return EHD_ERR_NOMEM;
  b->stream = static_cast<cudaStream_t>(stream);
  b->steady_tol = steady_tol;
  b->step_cap = step_cap;
  b->slots.resize(max_slots);
  // co-resident capacity of the shared potential launch for every tile height
  {
    int dev = 0, sms = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
      cudaGetLastError();
      delete b;
      return EHD_ERR_CUDA;
    }
    for (int c = 0; c < 3; ++c) {
      const int rows = BATCH_ROW_CHOICES[c];
      KParams kp{};
      kp.nx = 64;
      kp.ny = rows;
      ResidentGeom g;
      int th, per_sm = 0;
      size_t sm;
      if (!resident_geometry(kp, 1, &g, &th, &sm, rows) ||
          cudaFuncSetAttribute(resident_batch_kernel(rows),
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resident_batch_kernel(rows), th,
                                                        sm) != cudaSuccess ||
          per_sm < 1) {
        cudaGetLastError();
        delete b;
        return EHD_ERR_CUDA;
      }
      b->cap[c] = per_sm * sms;
      b->thr[c] = th;
      b->smm[c] = sm;
    }
    b->tile_capacity = b->cap[1];
    b->rthreads = b->thr[1];
    b->rsmem = b->smm[1];
  }
  if (arena) {
    b->arena = static_cast<char*>(arena);
    b->own_arena = false;
  } else {
    if (cudaMalloc(&b->arena, hbm_budget) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return EHD_ERR_NOMEM;
    }
    b->own_arena = true;
  }
  b->arena_bytes = hbm_budget;
  // device tables at the start of the arena; a slot's nodes never exceed its tiles x 2048,
  // which bounds the work lists of the moments (256 nodes a block) and coupled (128) passes
  size_t max_nodes = 0;
  int max_tiles = 0;
  for (int c = 0; c < 3; ++c) {
    const size_t n = (size_t)b->cap[c] * 64 * BATCH_ROW_CHOICES[c];
    if (n > max_nodes) max_nodes = n;
    if (b->cap[c] > max_tiles) max_tiles = b->cap[c];
  }
  b->mwork_cap = (int)(max_nodes / 256) + max_slots;  // moments_blocks(N) <= N / 256 + 1
  b->cwork_cap = (int)(max_nodes / 128) + max_slots;
  const size_t t1 = al256(sizeof(ResidentSlot) * (size_t)max_slots);
  const size_t t2 = al256(sizeof(int2) * (size_t)max_tiles);
  const size_t t3 = al256(sizeof(StepSlot) * (size_t)max_slots);
  const size_t t4 = al256(sizeof(int2) * (size_t)b->mwork_cap);
  const size_t t5 = al256(sizeof(int2) * (size_t)b->cwork_cap);
  if (t1 + t2 + t3 + t4 + t5 >= hbm_budget) {
    ehd_batch_destroy(b);
    return EHD_ERR_NOMEM;
  }
  b->d_slots = reinterpret_cast<ResidentSlot*>(b->arena);
  b->d_work = reinterpret_cast<int2*>(b->arena + t1);
  b->d_step = reinterpret_cast<StepSlot*>(b->arena + t1 + t2);
  b->d_mwork = reinterpret_cast<int2*>(b->arena + t1 + t2 + t3);
  b->d_cwork = reinterpret_cast<int2*>(b->arena + t1 + t2 + t3 + t4);
  b->heap_start = t1 + t2 + t3 + t4 + t5;
  *out = b;
  return EHD_OK;
}

int ehd_batch_admit(ehd_batch* b, const ehd_params* params, const double* phi, const double* q,
                    const double* ux, const double* uy, int64_t request_id, int* slot) {
  if (!b || !params || !phi || !q || !ux || !uy || !slot) return EHD_ERR_INVALID_ARG;
  if (params->nx < 1 || params->ny < 1) return EHD_ERR_INVALID_ARG;
  // batches run the on-chip loop, which implements the paper's scheme only
  if (params->potential_scheme != EHD_SCHEME_IMPROVED) return EHD_ERR_INVALID_ARG;
  if (params->poisson_loop == EHD_LOOP_STREAM) return EHD_ERR_INVALID_ARG;
  // the shared launch runs the one-step on-chip loop for every slot (the same states as
  // the multi-step loops): the slot is laid out for it
  ehd_params pslot = *params;
  pslot.poisson_loop = EHD_LOOP_RESIDENT;
  int idx = -1;
  for (int i = 0; i < (int)b->slots.size(); ++i)
    if (!b->slots[i].live) {
      idx = i;
      break;
    }
  if (idx < 0) return EHD_ERR_BUSY;
  const int ntiles = ((params->nx + 63) / 64) * ((params->ny + b->rows - 1) / b->rows);
  if (b->tiles_used + ntiles > b->tile_capacity) return EHD_ERR_BUSY;
  const size_t N = (size_t)params->nx * params->ny;
  const int nblocks = (int)((N + STEADY_THREADS - 1) / STEADY_THREADS);
  const size_t ws = al256(sim_workspace_bytes(&pslot, b->rows));
  const size_t snap = al256(sizeof(float) * 3 * N);
  const size_t part = al256(sizeof(double) * 4 * (size_t)nblocks);
  size_t off;
  if (!arena_alloc(b, ws + snap + part, &off)) return EHD_ERR_BUSY;
  ehd_sim* s = nullptr;
  int st = sim_create(&pslot, b->arena + off, ws, b->stream, b->rows, &s);
  if (st != EHD_OK) {
    arena_free(b, off);
    return st;
  }
  if (!s->resident_ok) {
    ehd_destroy(s);
    arena_free(b, off);
    return EHD_ERR_BUSY;
  }
  s->cur = b->cur;
  st = ehd_set_fields(s, phi, q, ux, uy, nullptr, EHD_HOST);
  if (st != EHD_OK && st != EHD_ERR_NOT_CONVERGED) {
    ehd_destroy(s);
    arena_free(b, off);
    return st;
  }
  Slot& sl = b->slots[idx];
  sl = Slot();
  sl.live = true;
  sl.sim = s;
  sl.off = off;
  sl.bytes = ws + snap + part;
  sl.snap = reinterpret_cast<float*>(b->arena + off + ws);
  sl.dpart = reinterpret_cast<double*>(b->arena + off + ws + snap);
  sl.nblocks = nblocks;
  sl.request_id = request_id;
  sl.ntiles = ntiles;
  b->tiles_used += ntiles;
  b->dirty = true;
  *slot = idx;
  return EHD_OK;
}

int ehd_batch_run(ehd_batch* b, int nsteps) {
  NvtxRange range("ehd_batch_run");
  if (!b || nsteps < 1) return EHD_ERR_INVALID_ARG;
  if (b->dirty) {
    const int st = rebuild(b);
    if (st != EHD_OK) return st;
  }
  bool any = false;
  for (Slot& sl : b->slots)
    if (sl.live) {
      any = true;
      ehd_sim* s = sl.sim;
      if (!s->stats_live) {
        if (launch_stats_reset(s->b, b->stream) != cudaSuccess) return EHD_ERR_CUDA;
        s->stats_live = true;
        s->launches = 1;
        s->graph_steps = 0;
        s->host_iters = 0;
      }
    }
  if (!any) return EHD_OK;
  int k = 0;
  for (; k + b->steps_per_graph <= nsteps; k += b->steps_per_graph)
    if (cudaGraphLaunch(b->execm[b->cur], b->stream) != cudaSuccess) return EHD_ERR_CUDA;
  for (; k < nsteps; ++k) {
    if (cudaGraphLaunch(b->exec[b->cur], b->stream) != cudaSuccess) return EHD_ERR_CUDA;
    b->cur ^= 1;
  }
  b->steps_run += nsteps;
  b->launches += 3 * (int64_t)nsteps;
  // bring each slot's bookkeeping along and queue its steadiness check; one wait for all
  std::vector<std::vector<double>> parts(b->slots.size());
  for (size_t i = 0; i < b->slots.size(); ++i) {
    Slot& sl = b->slots[i];
    if (!sl.live) continue;
    ehd_sim* s = sl.sim;
    s->cur = b->cur;
    s->n += nsteps;
    s->history_valid = true;
    s->graph_steps += nsteps;
    sl.steps += nsteps;
    const Pops P = pops_copy(s->kp, s->b, s->cur);
    if (s->kp.half)
      k_steady<true><<<sl.nblocks, STEADY_THREADS, 0, b->stream>>>(s->kp, P, s->b.hist, sl.snap,
                                                                  sl.have_snap, sl.dpart);
    else
      k_steady<false><<<sl.nblocks, STEADY_THREADS, 0, b->stream>>>(s->kp, P, s->b.hist, sl.snap,
                                                                   sl.have_snap, sl.dpart);
    if (cudaGetLastError() != cudaSuccess) return EHD_ERR_CUDA;
    b->launches += 1;
    parts[i].resize((size_t)sl.nblocks * 4);
    if (cudaMemcpyAsync(parts[i].data(), sl.dpart, sizeof(double) * parts[i].size(),
                        cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
      return EHD_ERR_CUDA;
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return EHD_ERR_CUDA;
  int status = EHD_OK;
  for (size_t i = 0; i < b->slots.size(); ++i) {
    Slot& sl = b->slots[i];
    if (!sl.live) continue;
    ehd_sim* s = sl.sim;
    double t[4] = {0, 0, 0, 0};
    for (int j = 0; j < sl.nblocks; ++j)
      for (int c = 0; c < 4; ++c) t[c] += parts[i][(size_t)j * 4 + c];
    if (sl.have_snap) {
      sl.rel_phi = t[1] > 0 ? std::sqrt(t[0] / t[1]) : (t[0] > 0 ? INFINITY : 0.0);
      // velocities below 1e-6 (lattice units) count as rest in the denominator, and a flow
      // whose RMS speed is below that is at rest (steady in u whatever its change)
      const double u_floor2 = 1e-12 * (double)s->kp.N;
      sl.rel_u = std::sqrt(t[2] / std::fmax(t[3], u_floor2));
      const bool at_rest = t[3] < u_floor2;
      sl.steady = (sl.rel_phi < b->steady_tol && (sl.rel_u < b->steady_tol || at_rest)) ? 1 : 0;
    }
    sl.have_snap = 1;
    ehd_stats es;
    const int st = ehd_read_stats(s, &es);
    sl.iters += es.poisson_iters_total;
    sl.status = st;
    if (st == EHD_ERR_NONFINITE || st == EHD_ERR_CUDA || st == EHD_ERR_TIMEOUT) status = st;
  }
  return status;
}

int ehd_batch_poll(ehd_batch* b, ehd_slot_status* out, int max, int* n) {
  if (!b || !n || (max > 0 && !out)) return EHD_ERR_INVALID_ARG;
  int k = 0;
  for (int i = 0; i < (int)b->slots.size(); ++i) {
    const Slot& sl = b->slots[i];
    if (!sl.live) continue;
    if (k < max) {
      ehd_slot_status& o = out[k];
      o.slot = i;
      o.live = 1;
      o.request_id = sl.request_id;
      o.steps = sl.steps;
      o.poisson_iters = sl.iters;
      o.steady = sl.steady;
      o.capped = sl.steps >= b->step_cap ? 1 : 0;
      o.status = sl.status;
      o.rel_change_phi = sl.rel_phi;
      o.rel_change_u = sl.rel_u;
    }
    ++k;
  }
  *n = k;
  return EHD_OK;
}

int ehd_batch_read_fields(ehd_batch* b, int slot, unsigned mask, void* const* out, int mem) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].live)
    return EHD_ERR_INVALID_ARG;
  return ehd_read_fields(b->slots[slot].sim, mask, out, mem);
}

int ehd_batch_retire(ehd_batch* b, int slot) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].live)
    return EHD_ERR_INVALID_ARG;
  Slot& sl = b->slots[slot];
  ehd_destroy(sl.sim);
  arena_free(b, sl.off);
  b->tiles_used -= sl.ntiles;
  sl = Slot();
  b->dirty = true;
  return EHD_OK;
}

int ehd_batch_set_schedule(ehd_batch* b, int tile_rows, int steps_per_graph) {
  if (!b || steps_per_graph < 2 || steps_per_graph > 64 || (steps_per_graph & 1))
    return EHD_ERR_INVALID_ARG;
  int c = -1;
  for (int j = 0; j < 3; ++j)
    if (BATCH_ROW_CHOICES[j] == tile_rows) c = j;
  if (c < 0) return EHD_ERR_INVALID_ARG;
  for (const Slot& sl : b->slots)
    if (sl.live) return EHD_ERR_BUSY;
  b->rows = tile_rows;
  b->steps_per_graph = steps_per_graph;
  b->tile_capacity = b->cap[c];
  b->rthreads = b->thr[c];
  b->rsmem = b->smm[c];
  b->dirty = true;
  return EHD_OK;
}

int ehd_batch_info(ehd_batch* b, ehd_batch_info_t* info) {
  if (!b || !info) return EHD_ERR_INVALID_ARG;
  int live = 0;
  for (const Slot& sl : b->slots) live += sl.live ? 1 : 0;
  size_t used = 0;
  for (const auto& u : b->used) used += u.second;
  info->live_slots = live;
  info->max_slots = (int)b->slots.size();
  info->arena_bytes = b->arena_bytes;
  info->arena_used = used + b->heap_start;
  info->tiles_used = b->tiles_used;
  info->tile_capacity = b->tile_capacity;
  info->tile_rows = b->rows;
  info->steps_per_graph = b->steps_per_graph;
  info->steps_run = b->steps_run;
  info->kernel_launches = b->launches;
  return EHD_OK;
}

void ehd_batch_destroy(ehd_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (Slot& sl : b->slots)
    if (sl.live) ehd_destroy(sl.sim);
  destroy_batch_graphs(b);
  if (b->own_arena && b->arena) cudaFree(b->arena);
  delete b;
}

}  // extern "C"
