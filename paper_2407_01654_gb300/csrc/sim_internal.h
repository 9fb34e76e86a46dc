// The simulation object behind the C ABI's ehd_sim handle, shared by api.cu and batch.cu.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "../../include/ehd.h"
#include "ehd_internal.cuh"

// A named NVTX range over a scope: the host-side phases of the library (each API call,
// and the moments pass, potential loop and coupled pass of steps queued from the host) on
// an Nsight timeline.  Header-only NVTX: without a tool attached each push / pop is a
// check of one pointer.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct ehd_sim {
  using KParams = ehd::KParams;
  using Buffers = ehd::Buffers;
  using Ctl = ehd::Ctl;
  using DevStats = ehd::DevStats;
  using ResidentGeom = ehd::ResidentGeom;
  ehd_params P;
  KParams kp;
  Buffers b;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;
  cudaStream_t stream = nullptr;
  int cur = 0;              // which population copy is current
  int64_t n = 0;            // step counter
  bool history_valid = false;
  int last_k = 1;           // sub-iterations of the last potential solve
  Ctl* h_ctl = nullptr;     // pinned mirror of the loop control
  DevStats* h_stats = nullptr;
  float* h_stage = nullptr; // pinned staging for host field I/O, NIO * N floats
  int64_t launches = 0;     // kernel launches queued since the statistics were cleared
  int64_t graph_steps = 0;  // steps run as graphs since then
  int64_t host_iters = 0;   // potential sub-iterations run from the host loop since then
  bool stats_live = false;  // device statistics are accumulating
  // per-launch event timing
  bool profiling = false;
  bool expire_barrier = false;  // diagnostics: the next on-chip solve's barrier never completes
  std::vector<cudaEvent_t> ev;     // start/stop pairs
  std::vector<int> ev_kind;        // kind per pair
  size_t ev_used = 0;              // pairs recorded and not yet accumulated
  double prof_ms[4] = {0, 0, 0, 0};
  int64_t prof_n[4] = {0, 0, 0, 0};
  // one step graph per population copy (moments -> while{potential} -> coupled)
  bool graphs_tried = false;
  bool graphs_ok = false;
  bool no_graphs = false;     // steps queued kernel by kernel from the host (ehd_use_graphs)
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  // MULTI_STEPS consecutive steps in one graph (from copy 0 and from copy 1): runs of that
  // many steps pay one graph launch instead of one per step
  static constexpr int MULTI_STEPS = 8;
  static_assert(MULTI_STEPS % 2 == 0, "a run must leave the copy index unchanged");
  cudaGraphExec_t mexec[2] = {nullptr, nullptr};
  bool mgraphs_ok = false;
  // the same step graphs with event-record nodes around the three parts, for profiling
  bool pgraphs_tried = false;
  bool pgraphs_ok = false;
  cudaGraphExec_t pexec[2] = {nullptr, nullptr};
  cudaEvent_t pev[4] = {nullptr, nullptr, nullptr, nullptr};
  // resident (on-chip) potential loop, when the lattice fits
  bool resident_ok = false;
  ResidentGeom rg{};
  int rthreads = 0;
  size_t rsmem = 0;
};


// Creates a simulation; fixed_ty > 0 tiles the resident potential loop with 64 x fixed_ty
// tiles (batch slots tile the same way in any mix).
int sim_create(const ehd_params* params, void* workspace, size_t workspace_bytes, void* stream,
               int fixed_ty, ehd_sim** out);
size_t sim_workspace_bytes(const ehd_params* params, int fixed_ty);
