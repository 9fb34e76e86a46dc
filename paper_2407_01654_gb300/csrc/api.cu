// Host side of the C ABI declared in include/ehd.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "../../include/ehd.h"
#include "ehd_internal.cuh"

using namespace ehd;

#include "sim_internal.h"

namespace {

constexpr double CS2D = 1.0 / 3.0;
constexpr uint64_t STATE_MAGIC = 0x4548443153544154ull;  // "EHD1STAT"

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
  size_t ss, pops, pops16, h, hist, phi, aq, io, tmp, partials, ctl, stats, exports, rpartials, total;
  size_t export_floats, rtiles;
};

// SM count the resident loop tiles for: the current device's (every SM gets tiles), or
// the GB300's 152 when no device can be queried (e.g. sizing a workspace on a host
// without a GPU).  The export space reserved for it covers that many tiles.
constexpr int DEFAULT_SMS = 152;
int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    return DEFAULT_SMS;
  }
  return sms;
}

// Sub-iterations per halo exchange of the on-chip loop a poisson_loop value asks for (0:
// one, the one-step loop; also for the automatic choice and the streaming loop).
int loop_depth(int poisson_loop) {
  return poisson_loop == EHD_LOOP_RESIDENT3 ? 3 : (poisson_loop == EHD_LOOP_RESIDENT2 ? 2 : 0);
}

Layout layout_for(const ehd_params& P, int fixed_ty = 0) {
  const int64_t N = (int64_t)P.nx * P.ny;
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  L.ss = take(sizeof(StepState) * 2);
  if (P.precision == EHD_FP16DEV) {
    L.pops = take(sizeof(float) * 2 * NP32_HALF * (size_t)N);
    L.pops16 = take(sizeof(__half) * 2 * 24 * (size_t)N);
  } else {
    L.pops = take(sizeof(float) * 2 * NP32 * (size_t)N);
    L.pops16 = take(256);
  }
  L.h = take(sizeof(float) * 2 * NH * (size_t)N);
  L.hist = take(sizeof(float) * NHIST * (size_t)N);
  L.phi = take(sizeof(float) * (size_t)N);
  L.aq = take(sizeof(float2) * (size_t)N);
  L.io = take(sizeof(float) * NIO * (size_t)N);
  L.tmp = take(sizeof(float) * (size_t)N);
  L.partials = take(sizeof(double2) * MAX_PARTIALS);
  L.ctl = take(sizeof(Ctl));
  L.stats = take(sizeof(DevStats));
  ResidentGeom g;
  int th;
  size_t sm;
  KParams kp{};
  kp.nx = P.nx;
  kp.ny = P.ny;
  L.export_floats = 0;
  L.rtiles = 0;
  if (resident_geometry(kp, device_sms(), &g, &th, &sm, fixed_ty, loop_depth(P.poisson_loop))) {
    L.rtiles = (size_t)g.ntx * g.nty;
    L.export_floats = 2 * L.rtiles * 8 * (size_t)g.pmax;
  }
  L.exports = take(sizeof(float) * (L.export_floats ? L.export_floats : 1));
  // [2][tiles] float2 partial sums (multi-step loop: [2][tiles] one or two float4,
  // 16-byte aligned)
  L.rpartials = take(sizeof(float2) * 8 * (L.rtiles > 0 ? L.rtiles : 1));
  L.total = o;
  return L;
}

bool sizes_ok(const ehd_params* p) {
  if (p->nx < 1 || p->ny < 1) return false;
  const int64_t N = (int64_t)p->nx * p->ny;
  // the one-pass reductions hold one partial per CTA: the moments pass (at most one per
  // 256 nodes) and the streaming potential kernel (one per 64 x 16 tile, which for narrow
  // lattices is far more than N / 256)
  if ((N + 255) / 256 > MAX_PARTIALS) return false;
  if (stream_tiles(p->nx, p->ny) > MAX_PARTIALS) return false;
  // the kernels index nodes with 32-bit integers
  if (N > 0x7fffffffLL) return false;
  return true;
}

int validate(const ehd_params* p) {
  if (!p || !sizes_ok(p)) return EHD_ERR_INVALID_ARG;
  if (p->walls_y != 0 && p->walls_y != 1) return EHD_ERR_INVALID_ARG;
  if (p->precision != EHD_FP32 && p->precision != EHD_FP16DEV) return EHD_ERR_INVALID_ARG;
  if (!(p->rho_l > 0 && p->rho_v > 0 && p->mu_l > 0 && p->mu_v > 0 && p->eps_l > 0 &&
        p->eps_v > 0 && p->sigma_l >= 0 && p->sigma_v >= 0 && p->alpha > 0 && p->gamma >= 0 &&
        p->width > 0 && p->mobility > 0))
    return EHD_ERR_INVALID_ARG;
  if (p->poisson_fixed_iter < 0 || p->poisson_max_iter < 1 || p->poisson_min_iter < 1)
    return EHD_ERR_INVALID_ARG;
  if (p->poisson_fixed_iter == 0 && !(p->poisson_tol > 0)) return EHD_ERR_INVALID_ARG;
  if (p->ramp_steps < 0) return EHD_ERR_INVALID_ARG;
  if (p->poisson_loop < EHD_LOOP_AUTO || p->poisson_loop > EHD_LOOP_RESIDENT3)
    return EHD_ERR_INVALID_ARG;
  if (p->tile_rows < 0 || p->tile_rows > 64 || p->tile_rows % 8 != 0)
    return EHD_ERR_INVALID_ARG;
  if ((p->potential_scheme != EHD_SCHEME_IMPROVED &&
       p->potential_scheme != EHD_SCHEME_CONVENTIONAL) ||
      !(p->chi > 0))
    return EHD_ERR_INVALID_ARG;
  if ((p->field_mode != 0 && p->field_mode != 1) || (p->lagged_field != 0 && p->lagged_field != 1))
    return EHD_ERR_INVALID_ARG;
  const double lim = 0.5 + 1e-3;
  const double tau_g = 0.5 + p->mobility / CS2D;
  const double tau_h = 0.5 + p->eps_v / CS2D;
  const double tau_l = 0.5 + p->alpha / CS2D;
  if (tau_g <= lim || tau_h <= lim || tau_l <= lim) return EHD_ERR_UNSTABLE_PARAMS;
  for (int j = 0; j <= 100; ++j) {
    const double phi = j / 100.0;
    const double rho = p->rho_v + (p->rho_l - p->rho_v) * phi;
    const double mu = p->mu_v + (p->mu_l - p->mu_v) * phi;
    const double tau_f = 0.5 + mu / (rho * CS2D);
    const double eps = p->eps_v + phi * phi * (2 * phi - 3) * (p->eps_v - p->eps_l);
    const double sig = p->sigma_v + (p->sigma_l - p->sigma_v) * phi;
    if (tau_f <= lim) return EHD_ERR_UNSTABLE_PARAMS;
    if (sig / eps > 0.5) return EHD_ERR_UNSTABLE_PARAMS;
    if (p->potential_scheme == EHD_SCHEME_CONVENTIONAL && 0.5 + eps / (p->chi * CS2D) <= lim)
      return EHD_ERR_UNSTABLE_PARAMS;
  }
  return EHD_OK;
}

KParams make_kparams(const ehd_params& P) {
  KParams k{};
  k.nx = P.nx;
  k.ny = P.ny;
  k.N = P.nx * P.ny;
  k.nint = k.N;
  k.row0 = 0;
  k.halo_lo = 0;
  k.halo_hi = 0;
  k.slab = 0;
  k.y_global0 = 0;
  k.ny_global = P.ny;
  k.walls = P.walls_y;
  k.neutralize = P.neutralize_charge ? 1 : 0;
  k.rho_v = (float)P.rho_v;
  k.drho = (float)(P.rho_l - P.rho_v);
  k.mu_v = (float)P.mu_v;
  k.dmu = (float)(P.mu_l - P.mu_v);
  k.sig_v = (float)P.sigma_v;
  k.dsig = (float)(P.sigma_l - P.sigma_v);
  k.eps_v = (float)P.eps_v;
  k.deps = (float)(P.eps_v - P.eps_l);
  const double beta = 12.0 * P.gamma / P.width;
  const double kappa = 1.5 * P.gamma * P.width;
  k.beta4 = (float)(4.0 * beta);
  k.kappa = (float)kappa;
  k.wet_a = (float)(kappa > 0 ? std::sqrt(2.0 * beta / kappa) : 4.0 / P.width);
  const double tau_g = 0.5 + P.mobility / CS2D;
  const double tau_l = 0.5 + P.alpha / CS2D;
  const double tau_h = 0.5 + P.eps_v / CS2D;
  k.omega_g = (float)(1.0 / tau_g);
  k.omega_l = (float)(1.0 / tau_l);
  k.pref_l = (float)(1.0 - 0.5 / tau_l);
  k.omega_h = (float)(1.0 / tau_h);
  k.cs2tauh = (float)(CS2D * tau_h);
  k.scheme = P.potential_scheme;
  k.field_fd = P.field_mode;
  k.lagged = P.lagged_field;
  k.inv_chi = (float)(1.0 / P.chi);
  k.inv_chi_cs2 = (float)(1.0 / (P.chi * CS2D));
  k.gbx = (float)P.body_gx;
  k.gby = (float)P.body_gy;
  const double pi = 3.14159265358979323846;
  k.cos_yb = std::cos(P.theta_bottom_deg * pi / 180.0);
  k.cos_yt = std::cos(P.theta_top_deg * pi / 180.0);
  k.ew_signed = P.ew_sign * P.ew_bottom;
  k.varphi_b = P.varphi_bottom;
  k.varphi_t = P.varphi_top;
  k.ramp_steps = P.ramp_steps;
  k.half = P.precision == EHD_FP16DEV ? 1 : 0;
  for (int f = 0; f < 3; ++f) {
    k.psc[f] = 1.0f;
    k.ipsc[f] = 1.0f;
  }
  return k;
}

#define EHD_CUDA(call)                         \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return EHD_ERR_CUDA; \
  } while (0)

// Accumulates recorded event pairs into the totals (synchronises the stream).
int prof_flush(ehd_sim* s) {
  if (!s->ev_used) return EHD_OK;
  EHD_CUDA(cudaStreamSynchronize(s->stream));
  for (size_t j = 0; j < s->ev_used; ++j) {
    float ms = 0.0f;
    EHD_CUDA(cudaEventElapsedTime(&ms, s->ev[2 * j], s->ev[2 * j + 1]));
    s->prof_ms[s->ev_kind[j]] += ms;
    s->prof_n[s->ev_kind[j]] += 1;
  }
  s->ev_used = 0;
  return EHD_OK;
}

// Records the start event of a launch of the given kind; returns its pair index or -1.
long prof_begin(ehd_sim* s, int kind) {
  s->launches += 1;
  if (!s->profiling) return -1;
  if (s->ev_used >= 4096 && prof_flush(s) != EHD_OK) return -1;
  if (2 * (s->ev_used + 1) > s->ev.size()) {
    for (int j = 0; j < 2; ++j) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      s->ev.push_back(e);
    }
    s->ev_kind.push_back(0);
  }
  const size_t j = s->ev_used++;
  s->ev_kind[j] = kind;
  cudaEventRecord(s->ev[2 * j], s->stream);
  return (long)j;
}

void prof_end(ehd_sim* s, long j) {
  if (j >= 0) cudaEventRecord(s->ev[2 * j + 1], s->stream);
}

#define EHD_LAUNCH(s, kind, call)             \
  do {                                        \
    const long pj_ = prof_begin((s), (kind)); \
    cudaError_t e_ = (call);                  \
    prof_end((s), pj_);                       \
    if (e_ != cudaSuccess) return EHD_ERR_CUDA; \
  } while (0)

// The potential loop of one solve.  The moments kernel has reset the control.  Fixed
// count: exactly that many launches.  Stopping rule: launches are queued in chunks; a
// launch after the rule has fired returns at once; the pinned control mirror tells the
// host when to stop queueing.
int run_potential_loop(ehd_sim* s, int fixed, int max_iter) {
  if (s->resident_ok) {
    if (s->expire_barrier) {
      s->expire_barrier = false;
      EHD_CUDA(launch_expire_barrier(s->b, s->stream));
    }
    // the whole loop in one cooperative launch
    EHD_LAUNCH(s, 1, launch_poisson_resident(s->kp, s->rg, s->rthreads, s->rsmem, s->b,
                                             s->stream));
    EHD_CUDA(cudaMemcpyAsync(s->h_ctl, s->b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                             s->stream));
    EHD_CUDA(cudaStreamSynchronize(s->stream));
    if (s->h_ctl->bar_error) return EHD_ERR_TIMEOUT;
    if (!s->h_ctl->done) return EHD_ERR_CUDA;
    s->last_k = s->h_ctl->iter;
    return s->h_ctl->converged ? EHD_OK : EHD_ERR_NOT_CONVERGED;
  }
  if (fixed > 0) {
    for (int i = 0; i < fixed; ++i) EHD_LAUNCH(s, 1, launch_poisson(s->kp, s->b, s->stream));
    return EHD_OK;
  }
  int queued = 0;
  int chunk = s->last_k + 1;
  const size_t first_pair = s->ev_used;
  for (;;) {
    if (chunk > max_iter - queued + 1) chunk = max_iter - queued + 1;
    if (chunk < 1) chunk = 1;
    for (int i = 0; i < chunk; ++i) EHD_LAUNCH(s, 1, launch_poisson(s->kp, s->b, s->stream));
    queued += chunk;
    EHD_CUDA(cudaMemcpyAsync(s->h_ctl, s->b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                             s->stream));
    EHD_CUDA(cudaStreamSynchronize(s->stream));
    if (s->h_ctl->done) {
      s->last_k = s->h_ctl->iter;
      // launches after the loop finished did no work: file them under their own kind
      if (s->profiling && s->ev_used >= first_pair)
        for (size_t j = first_pair + (size_t)s->h_ctl->iter; j < s->ev_used; ++j)
          s->ev_kind[j] = 2;
      return s->h_ctl->converged ? EHD_OK : EHD_ERR_NOT_CONVERGED;
    }
    if (queued > max_iter + 2) return EHD_ERR_CUDA;  // the control never finished
    chunk = chunk * 2;
  }
}

void destroy_graphs(ehd_sim* s) {
  for (int c = 0; c < 2; ++c) {
    if (s->exec[c]) cudaGraphExecDestroy(s->exec[c]);
    if (s->graph[c]) cudaGraphDestroy(s->graph[c]);
    if (s->pexec[c]) cudaGraphExecDestroy(s->pexec[c]);
    if (s->mexec[c]) cudaGraphExecDestroy(s->mexec[c]);
    s->exec[c] = nullptr;
    s->graph[c] = nullptr;
    s->pexec[c] = nullptr;
    s->mexec[c] = nullptr;
  }
  s->graphs_ok = false;
  s->mgraphs_ok = false;
  s->pgraphs_ok = false;
  s->pgraphs_tried = false;
}

// The profiling form of the step graphs: event-record nodes before the moments pass and
// after each part, so the per-kernel times come from the graph's own execution.
void ensure_prof_graphs(ehd_sim* s) {
  if (s->pgraphs_tried) return;
  s->pgraphs_tried = true;
  const ehd_params& P = s->P;
  for (int j = 0; j < 4; ++j)
    if (!s->pev[j] && cudaEventCreate(&s->pev[j]) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
  for (int c = 0; c < 2; ++c) {
    cudaGraph_t g = nullptr;
    const bool ok =
        build_step_graph(s->kp, s->b, c, P.poisson_tol, P.poisson_min_iter, P.poisson_max_iter,
                         P.poisson_fixed_iter, s->resident_ok ? &s->rg : nullptr, s->rthreads,
                         s->rsmem, &g, s->pev) == cudaSuccess &&
        cudaGraphInstantiate(&s->pexec[c], g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      cudaGetLastError();
      for (int d = 0; d < 2; ++d) {
        if (s->pexec[d]) cudaGraphExecDestroy(s->pexec[d]);
        s->pexec[d] = nullptr;
      }
      return;
    }
  }
  s->pgraphs_ok = true;
}

// Builds the two step graphs once.  If the driver refuses (e.g. no conditional nodes),
// steps run through the host-side loop instead; both paths run the same kernels.
void ensure_graphs(ehd_sim* s) {
  if (s->graphs_tried) return;
  s->graphs_tried = true;
  const ehd_params& P = s->P;
  for (int c = 0; c < 2; ++c) {
    if (build_step_graph(s->kp, s->b, c, P.poisson_tol, P.poisson_min_iter, P.poisson_max_iter,
                         P.poisson_fixed_iter, s->resident_ok ? &s->rg : nullptr, s->rthreads,
                         s->rsmem, &s->graph[c]) != cudaSuccess ||
        cudaGraphInstantiate(&s->exec[c], s->graph[c], 0) != cudaSuccess) {
      cudaGetLastError();
      destroy_graphs(s);
      return;
    }
  }
  s->graphs_ok = true;
  // the multi-step graphs are an optimisation: without them steps run one graph each
  bool mok = true;
  for (int c = 0; c < 2 && mok; ++c) {
    cudaGraph_t g = nullptr;
    mok = build_step_graph(s->kp, s->b, c, P.poisson_tol, P.poisson_min_iter,
                           P.poisson_max_iter, P.poisson_fixed_iter,
                           s->resident_ok ? &s->rg : nullptr, s->rthreads, s->rsmem, &g,
                           nullptr, ehd_sim::MULTI_STEPS) == cudaSuccess &&
          cudaGraphInstantiate(&s->mexec[c], g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
  }
  if (!mok) {
    cudaGetLastError();
    for (int c = 0; c < 2; ++c) {
      if (s->mexec[c]) cudaGraphExecDestroy(s->mexec[c]);
      s->mexec[c] = nullptr;
    }
  }
  s->mgraphs_ok = mok;
}

// Copies one input field into the staging area; returns its largest magnitude in *amax
// (used to choose the FP16 storage scales).
// dst[j][i] = (To)src[j][i] for j < nf, i < n: the conversions between the caller's
// double arrays and the float32 staging buffers, split over up to 8 host threads when
// there are at least 2^20 values in all (below that, starting threads costs more than
// they save).
template <typename To, typename From>
void convert(To* const* dst, const From* const* src, int nf, size_t n) {
  const size_t total = (size_t)nf * n;
  const unsigned hw = std::thread::hardware_concurrency();
  const size_t nt = total < ((size_t)1 << 20) ? 1 : (hw < 2 ? 1 : (hw < 8 ? hw : 8));
  auto part = [&](size_t t) {
    const size_t a = total * t / nt, b = total * (t + 1) / nt;
    for (size_t k = a; k < b;) {  // flat index k = j n + i
      const size_t j = k / n, i0 = k - j * n, i1 = (b - j * n < n) ? b - j * n : n;
      To* d = dst[j];
      const From* f = src[j];
      for (size_t i = i0; i < i1; ++i) d[i] = (To)f[i];
      k = j * n + i1;
    }
  };
  if (nt == 1) {
    part(0);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(nt - 1);
  for (size_t t = 1; t < nt; ++t) th.emplace_back(part, t);
  part(0);
  for (auto& x : th) x.join();
}

int stage_in(ehd_sim* s, const void* src, int slot, int mem, double* amax) {
  const size_t N = (size_t)s->kp.N;
  float* dst = s->b.io + slot * N;
  float* stage = s->h_stage + slot * N;
  if (mem == EHD_DEVICE) {
    EHD_CUDA(cudaMemcpyAsync(dst, src, N * sizeof(float), cudaMemcpyDeviceToDevice,
                             s->stream));
    if (s->kp.half) {
      EHD_CUDA(cudaMemcpyAsync(stage, src, N * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
      EHD_CUDA(cudaStreamSynchronize(s->stream));
    }
  } else {
    const double* d = static_cast<const double*>(src);
    convert(&stage, &d, 1, N);
    EHD_CUDA(cudaMemcpyAsync(dst, stage, N * sizeof(float), cudaMemcpyHostToDevice,
                             s->stream));
  }
  double m = 0.0;
  if (s->kp.half)
    for (size_t i = 0; i < N; ++i) {
      const double a = std::fabs((double)stage[i]);
      m = a > m ? a : m;
    }
  *amax = m;
  return EHD_OK;
}

// Power of two 2^floor(log2(1/ref)): the FP16 scale that maps a magnitude ref to [0.5, 1).
float pow2_scale(double ref) {
  int e;
  std::frexp(1.0 / ref, &e);
  return (float)std::ldexp(1.0, e - 1);
}

// FP16 storage scales from the parameters and the initial fields: g's moving populations
// carry w_i hbar (hbar ~ beta), l's w_i q, f's w_i (3 p + 3 rho c.u).
void choose_scales(ehd_sim* s, double qmax, double umax) {
  const ehd_params& P = s->P;
  const double beta = 12.0 * P.gamma / P.width;
  const double eps_max = P.eps_l > P.eps_v ? P.eps_l : P.eps_v;
  const double rho_max = P.rho_l > P.rho_v ? P.rho_l : P.rho_v;
  double dphi = std::fabs(P.varphi_bottom - P.varphi_top);
  dphi = std::fmax(dphi, std::fmax(std::fabs(P.varphi_bottom), std::fabs(P.varphi_top)));
  const double L = (double)(P.nx < P.ny ? P.nx : P.ny);
  const double g_ref = std::fmax(beta, 1e-6);
  const double q_ref = std::fmax(std::fmax(qmax, eps_max * dphi / (L * L)), 1e-9);
  const double f_ref = std::fmax(std::fmax(3.0 * rho_max * std::fmax(umax, 1e-3),
                                           eps_max * (dphi / L) * (dphi / L)), 1e-9);
  const double refs[3] = {g_ref, q_ref, f_ref};
  for (int f = 0; f < 3; ++f) {
    s->kp.psc[f] = pow2_scale(refs[f]);
    s->kp.ipsc[f] = 1.0f / s->kp.psc[f];
  }
}

}  // namespace

extern "C" {

#ifdef EHD_CHECKED
const char* ehd_version(void) { return "ehd-gb300 0.1 (sm_103a, checked indices)"; }
#else
const char* ehd_version(void) { return "ehd-gb300 0.1 (sm_103a)"; }
#endif

int ehd_abi_sizes(size_t* params_bytes, size_t* stats_bytes) {
  if (params_bytes) *params_bytes = sizeof(ehd_params);
  if (stats_bytes) *stats_bytes = sizeof(ehd_stats);
  return EHD_OK;
}

const char* ehd_error_string(int code) {
  switch (code) {
    case EHD_OK: return "ok";
    case EHD_ERR_INVALID_ARG: return "invalid argument";
    case EHD_ERR_UNSTABLE_PARAMS: return "unstable parameters (relaxation time or sigma/eps)";
    case EHD_ERR_NOMEM: return "out of memory or workspace too small";
    case EHD_ERR_NOT_CONVERGED: return "potential loop reached its iteration cap";
    case EHD_ERR_NONFINITE: return "non-finite values in phi or q";
    case EHD_ERR_BUSY: return "no free slot or memory";
    case EHD_ERR_CUDA: return "CUDA runtime error";
    case EHD_ERR_TOO_LARGE: return "lattice exceeds the fixed scratch of the no-allocation solve";
    case EHD_ERR_TIMEOUT: return "a bounded device-side wait ran out (grid barrier)";
    default: return "unknown status";
  }
}

int ehd_workspace_bytes(const ehd_params* params, size_t* bytes) {
  if (!params || !bytes || !sizes_ok(params)) return EHD_ERR_INVALID_ARG;
  if (params->tile_rows < 0 || params->tile_rows > 64 || params->tile_rows % 8 != 0)
    return EHD_ERR_INVALID_ARG;
  *bytes = layout_for(*params, params->tile_rows).total;
  return EHD_OK;
}

}  // extern "C"

size_t sim_workspace_bytes(const ehd_params* params, int fixed_ty) {
  return layout_for(*params, fixed_ty).total;
}

int sim_create(const ehd_params* params, void* workspace, size_t workspace_bytes, void* stream,
               int fixed_ty, ehd_sim** out) {
  if (!out) return EHD_ERR_INVALID_ARG;
  *out = nullptr;
  const int v = validate(params);
  if (v != EHD_OK) return v;
  const int64_t N = (int64_t)params->nx * params->ny;
  const Layout L = layout_for(*params, fixed_ty);
  ehd_sim* s = new (std::nothrow) ehd_sim();
  if (!s) return EHD_ERR_NOMEM;
  s->P = *params;
  s->kp = make_kparams(*params);
  s->stream = static_cast<cudaStream_t>(stream);
  s->n = params->start_step;
  if (workspace) {
    if (workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255u)) {
      delete s;
      return workspace_bytes < L.total ? EHD_ERR_NOMEM : EHD_ERR_INVALID_ARG;
    }
    s->ws = workspace;
    s->own_ws = false;
  } else {
    if (cudaMalloc(&s->ws, L.total) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return EHD_ERR_NOMEM;
    }
    s->own_ws = true;
  }
  s->ws_bytes = L.total;
  char* base = static_cast<char*>(s->ws);
  s->b.ss = reinterpret_cast<StepState*>(base + L.ss);
  s->b.pops = reinterpret_cast<float*>(base + L.pops);
  s->b.pops16 = reinterpret_cast<__half*>(base + L.pops16);
  s->b.h = reinterpret_cast<float*>(base + L.h);
  s->b.hist = reinterpret_cast<float*>(base + L.hist);
  s->b.phi = reinterpret_cast<float*>(base + L.phi);
  s->b.aq = reinterpret_cast<float2*>(base + L.aq);
  s->b.io = reinterpret_cast<float*>(base + L.io);
  s->b.tmp = reinterpret_cast<float*>(base + L.tmp);
  s->b.partials = reinterpret_cast<double2*>(base + L.partials);
  s->b.ctl = reinterpret_cast<Ctl*>(base + L.ctl);
  s->b.stats = reinterpret_cast<DevStats*>(base + L.stats);
  s->b.exports = reinterpret_cast<float*>(base + L.exports);
  s->b.rpartials = reinterpret_cast<float2*>(base + L.rpartials);
  s->kp.oob = &s->b.ctl->oob;
  // resident potential loop: needs cooperative launch, one tile per SM on this device,
  // and an export area within the reserved space
  {
    int dev = 0, sms = 0, coop = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess &&
        coop && L.export_floats && params->poisson_loop != EHD_LOOP_STREAM) {
      const int use_sms = sms;
      ResidentGeom g;
      int th;
      size_t sm;
      const int depth = loop_depth(params->poisson_loop);
      // the conventional scheme runs on the one- and two-step loops
      const bool conv = params->potential_scheme == EHD_SCHEME_CONVENTIONAL;
      const void* fk = nullptr;
      if (resident_geometry(s->kp, use_sms, &g, &th, &sm, fixed_ty, depth) &&
          (fk = resident_kernel(g.TY, depth, conv)) != nullptr &&
          2 * (size_t)g.ntx * g.nty * 8 * g.pmax <= L.export_floats &&
          (size_t)g.ntx * g.nty <= L.rtiles &&
          cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) ==
              cudaSuccess) {
        int per_sm = 0;
        // the multi-step loops hold tensor memory for the whole launch: CTAs that share
        // an SM must fit its 512 columns together, or a CTA would wait in tcgen05.alloc
        // for one that only leaves at the end of the loop
        const int tcols = resident_tmem_columns(g.TY, depth);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fk, th, sm) != cudaSuccess)
          per_sm = 0;
        if (tcols < 0) per_sm = 0;
        if (tcols > 0 && per_sm > 512 / tcols) per_sm = 512 / tcols;
        if (per_sm >= 1 && (long long)g.ntx * g.nty <= (long long)per_sm * sms) {
          s->resident_ok = true;
          s->rg = g;
          s->rthreads = th;
          s->rsmem = sm;
        }
      }
    }
    cudaGetLastError();
    if ((params->poisson_loop == EHD_LOOP_RESIDENT || params->poisson_loop == EHD_LOOP_RESIDENT2 ||
         params->poisson_loop == EHD_LOOP_RESIDENT3) &&
        !s->resident_ok) {
      ehd_destroy(s);
      return EHD_ERR_INVALID_ARG;  // the lattice does not fit on chip on this device
    }
  }
  if (cudaMallocHost(&s->h_ctl, sizeof(Ctl)) != cudaSuccess ||
      cudaMallocHost(&s->h_stats, sizeof(DevStats)) != cudaSuccess ||
      cudaMallocHost(&s->h_stage, sizeof(float) * NIO * (size_t)N) != cudaSuccess) {
    cudaGetLastError();
    ehd_destroy(s);
    return EHD_ERR_NOMEM;
  }
  // zero everything once: populations, control, tickets
  if (cudaMemsetAsync(s->ws, 0, L.total, s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess) {
    ehd_destroy(s);
    return EHD_ERR_CUDA;
  }
  *out = s;
  return EHD_OK;
}

extern "C" {

int ehd_create(const ehd_params* params, void* workspace, size_t workspace_bytes, void* stream,
               ehd_sim** out) {
  return sim_create(params, workspace, workspace_bytes, stream, params ? params->tile_rows : 0,
                    out);
}

int ehd_profile(ehd_sim* s, int enable) {
  if (!s) return EHD_ERR_INVALID_ARG;
  if (prof_flush(s) != EHD_OK) return EHD_ERR_CUDA;
  s->profiling = enable != 0;
  for (int j = 0; j < 4; ++j) {
    s->prof_ms[j] = 0.0;
    s->prof_n[j] = 0;
  }
  return EHD_OK;
}

int ehd_profile_read(ehd_sim* s, ehd_kernel_times* out) {
  if (!s || !out) return EHD_ERR_INVALID_ARG;
  if (prof_flush(s) != EHD_OK) return EHD_ERR_CUDA;
  for (int j = 0; j < 4; ++j) {
    out->ms[j] = s->prof_ms[j];
    out->launches[j] = s->prof_n[j];
  }
  return EHD_OK;
}

void ehd_destroy(ehd_sim* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  destroy_graphs(s);
  for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
  for (cudaEvent_t e : s->pev)
    if (e) cudaEventDestroy(e);
  if (s->own_ws && s->ws) cudaFree(s->ws);
  if (s->h_ctl) cudaFreeHost(s->h_ctl);
  if (s->h_stats) cudaFreeHost(s->h_stats);
  if (s->h_stage) cudaFreeHost(s->h_stage);
  delete s;
}

int ehd_diag_index_errors(ehd_sim* s, unsigned* count) {
  if (!s || !count) return EHD_ERR_INVALID_ARG;
  EHD_CUDA(cudaMemcpyAsync(count, &s->b.ctl->oob, sizeof(unsigned), cudaMemcpyDeviceToHost,
                           s->stream));
  EHD_CUDA(cudaStreamSynchronize(s->stream));
  return EHD_OK;
}

int ehd_contact_line(ehd_sim* s, double level, double* out) {
  if (!s || !out || !s->kp.walls || s->kp.ny < 2 || s->kp.slab || !(level > 0.0) ||
      !(level < 1.0))
    return EHD_ERR_INVALID_ARG;
  EHD_CUDA(launch_contact_line(s->kp, s->b, s->cur, (float)level, s->stream));
  double2 r[2];
  EHD_CUDA(cudaMemcpyAsync(r, s->b.partials, sizeof(r), cudaMemcpyDeviceToHost, s->stream));
  EHD_CUDA(cudaStreamSynchronize(s->stream));
  out[0] = r[0].x;
  out[1] = r[0].y;
  out[2] = r[1].x;
  return EHD_OK;
}

int ehd_solve_potential(ehd_sim* s, double tol, int max_iter, int* iters, double* rel_change) {
  NvtxRange range("ehd_solve_potential");
  if (!s) return EHD_ERR_INVALID_ARG;
  const ehd_params& P = s->P;
  const double t = tol > 0 ? tol : P.poisson_tol;
  const int mx = max_iter > 0 ? max_iter : P.poisson_max_iter;
  const int fixed = (tol > 0 || max_iter > 0) ? 0 : P.poisson_fixed_iter;
  EHD_LAUNCH(s, 0, launch_moments(s->kp, s->b, s->cur, t, P.poisson_min_iter, mx, fixed,
                                   s->stream, s->resident_ok));
  int st = run_potential_loop(s, fixed, mx);
  if (st == EHD_ERR_CUDA) return st;
  EHD_CUDA(cudaMemcpyAsync(s->h_ctl, s->b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  EHD_CUDA(cudaStreamSynchronize(s->stream));
  if (iters) *iters = s->h_ctl->iter;
  if (rel_change) *rel_change = s->h_ctl->rel;
  if (s->h_ctl->nonfinite) return EHD_ERR_NONFINITE;
  return s->h_ctl->converged ? EHD_OK : EHD_ERR_NOT_CONVERGED;
}

int ehd_set_fields(ehd_sim* s, const void* phi, const void* q, const void* ux, const void* uy,
                   const void* p, int mem) {
  if (!s || !phi || !q || !ux || !uy || (mem != EHD_HOST && mem != EHD_DEVICE))
    return EHD_ERR_INVALID_ARG;
  NvtxRange range("ehd_set_fields");
  int st;
  double m_phi, m_q, m_ux, m_uy, m_p;
  if ((st = stage_in(s, phi, 0, mem, &m_phi)) != EHD_OK) return st;
  if ((st = stage_in(s, q, 1, mem, &m_q)) != EHD_OK) return st;
  if ((st = stage_in(s, ux, 2, mem, &m_ux)) != EHD_OK) return st;
  if ((st = stage_in(s, uy, 3, mem, &m_uy)) != EHD_OK) return st;
  if (p && (st = stage_in(s, p, 4, mem, &m_p)) != EHD_OK) return st;
  if (s->kp.half) {
    choose_scales(s, m_q, m_ux > m_uy ? m_ux : m_uy);
    // the step graphs hold the coefficients: rebuild them with the new scales
    destroy_graphs(s);
    s->graphs_tried = false;
  }
  s->n = s->P.start_step;
  s->history_valid = false;
  // the populations are written into the current copy; the potential restarts in copy 0
  EHD_CUDA(cudaMemsetAsync(&s->b.ctl->parity, 0, sizeof(int), s->stream));
  EHD_CUDA(cudaMemsetAsync(&s->b.ctl->nonfinite, 0, sizeof(int), s->stream));
  s->launches += 1;
  EHD_CUDA(launch_step_set(s->kp, s->b, s->cur, s->n, 1, s->stream));
  EHD_LAUNCH(s, 0, launch_init(s->kp, s->b, s->cur, p != nullptr, s->stream));
  s->last_k = 1;
  return ehd_solve_potential(s, 0.0, 0, nullptr, nullptr);
}

static int fill_stats(ehd_sim* s, ehd_stats* out) {
  EHD_CUDA(cudaMemcpyAsync(s->h_stats, s->b.stats, sizeof(DevStats), cudaMemcpyDeviceToHost,
                           s->stream));
  EHD_CUDA(cudaStreamSynchronize(s->stream));
  const DevStats& d = *s->h_stats;
  out->step = s->n;
  out->steps = d.steps;
  out->poisson_iters_total = d.iters_total;
  out->poisson_iters_min = d.steps ? d.iters_min : 0;
  out->poisson_iters_max = d.iters_max;
  out->not_converged_steps = d.not_converged;
  out->nonfinite = d.nonfinite;
  out->last_rel_change = d.last_rel;
  out->sum_phi = d.sum_phi;
  out->sum_q = d.sum_q;
  // host-driven launches are counted as they are queued; a graph step launches moments,
  // the potential loop (one resident kernel, or one kernel per sub-iteration) and coupled
  out->kernel_launches = s->launches + 2LL * s->graph_steps;
  if (s->resident_ok)
    out->kernel_launches += s->graph_steps;
  else
    out->kernel_launches += (int64_t)d.iters_total - s->host_iters;
  int status = EHD_OK;
  if (d.not_converged) status = EHD_ERR_NOT_CONVERGED;
  if (d.nonfinite) status = EHD_ERR_NONFINITE;
  if (d.barrier_error) status = EHD_ERR_TIMEOUT;
  return status;
}

static int reset_stats(ehd_sim* s) {
  s->launches = 1;
  s->graph_steps = 0;
  s->host_iters = 0;
  EHD_CUDA(launch_stats_reset(s->b, s->stream));
  return EHD_OK;
}

int ehd_step(ehd_sim* s, int nsteps, ehd_stats* out) {
  if (!s || nsteps < 0) return EHD_ERR_INVALID_ARG;
  NvtxRange range("ehd_step");
  const ehd_params& P = s->P;
  int status = EHD_OK;
  if (out || !s->stats_live) {
    if (reset_stats(s) != EHD_OK) return EHD_ERR_CUDA;
    s->stats_live = true;
  }
  if (!s->no_graphs) ensure_graphs(s);
  if (s->profiling && s->graphs_ok && !s->no_graphs) ensure_prof_graphs(s);
  for (int k = 0; k < nsteps; ++k) {
    // an armed diagnostic runs its step from the host (the graph has no slot for it)
    const bool use_graphs = s->graphs_ok && !s->expire_barrier && !s->no_graphs &&
                            (!s->profiling || s->pgraphs_ok);
    if (use_graphs && !s->profiling && s->mgraphs_ok && nsteps - k >= ehd_sim::MULTI_STEPS) {
      // a run of steps in one launch (an even count: the copy index is unchanged after it)
      EHD_CUDA(cudaGraphLaunch(s->mexec[s->cur], s->stream));
      s->graph_steps += ehd_sim::MULTI_STEPS;
      s->n += ehd_sim::MULTI_STEPS;
      s->history_valid = true;
      k += ehd_sim::MULTI_STEPS - 1;
      continue;
    }
    if (use_graphs && s->profiling) {
      // the profiling graph: the step's three parts timed by its own event nodes
      EHD_CUDA(cudaGraphLaunch(s->pexec[s->cur], s->stream));
      EHD_CUDA(cudaEventSynchronize(s->pev[3]));
      const int kinds[3] = {0, 1, 3};
      for (int j = 0; j < 3; ++j) {
        float ms = 0.0f;
        EHD_CUDA(cudaEventElapsedTime(&ms, s->pev[j], s->pev[j + 1]));
        s->prof_ms[kinds[j]] += ms;
        s->prof_n[kinds[j]] += 1;
      }
      s->graph_steps += 1;
    } else if (use_graphs) {
      // the whole step, potential loop included, without returning to the host
      EHD_CUDA(cudaGraphLaunch(s->exec[s->cur], s->stream));
      s->graph_steps += 1;
    } else {
      {
        NvtxRange r("moments");
        EHD_LAUNCH(s, 0, launch_moments(s->kp, s->b, s->cur, P.poisson_tol,
                                         P.poisson_min_iter, P.poisson_max_iter,
                                         P.poisson_fixed_iter, s->stream, s->resident_ok));
      }
      int st;
      {
        NvtxRange r("potential loop");
        st = run_potential_loop(s, P.poisson_fixed_iter, P.poisson_max_iter);
      }
      if (st == EHD_ERR_CUDA || st == EHD_ERR_TIMEOUT) return st;
      if (st != EHD_OK) status = st;
      if (!s->resident_ok) s->host_iters += s->h_ctl->iter;
      NvtxRange r("coupled");
      EHD_LAUNCH(s, 3, launch_coupled(s->kp, s->b, s->cur, s->stream));
    }
    s->cur ^= 1;
    s->n += 1;
    s->history_valid = true;
  }
  if (out) {
    const int st = fill_stats(s, out);
    s->stats_live = false;
    if (st != EHD_OK && status == EHD_OK) status = st;
    if (st == EHD_ERR_NONFINITE || st == EHD_ERR_CUDA || st == EHD_ERR_TIMEOUT) status = st;
  }
  return status;
}

int ehd_use_graphs(ehd_sim* s, int enable) {
  if (!s) return EHD_ERR_INVALID_ARG;
  s->no_graphs = enable == 0;
  return EHD_OK;
}

int ehd_diag_expire_barrier(ehd_sim* s) {
  if (!s || !s->resident_ok) return EHD_ERR_INVALID_ARG;
  s->expire_barrier = true;
  return EHD_OK;
}

int ehd_loop_kind(const ehd_sim* s) {
  if (!s) return -1;
  if (!s->resident_ok) return EHD_LOOP_STREAM;
  return s->rg.depth == 3 ? EHD_LOOP_RESIDENT3
                          : (s->rg.depth == 2 ? EHD_LOOP_RESIDENT2 : EHD_LOOP_RESIDENT);
}

int ehd_read_stats(ehd_sim* s, ehd_stats* out) {
  if (!s || !out) return EHD_ERR_INVALID_ARG;
  if (!s->stats_live) {
    std::memset(out, 0, sizeof(*out));
    out->step = s->n;
    return EHD_OK;
  }
  const int st = fill_stats(s, out);
  s->stats_live = false;
  return st;
}

int ehd_read_fields(ehd_sim* s, unsigned mask, void* const* out, int mem) {
  NvtxRange range("ehd_read_fields");
  if (!s || !out || (mem != EHD_HOST && mem != EHD_DEVICE) || (mask & ~((1u << EHD_NUM_FIELDS) - 1u)))
    return EHD_ERR_INVALID_ARG;
  if (!mask) return EHD_OK;
  int nf = 0;
  for (int b = 0; b < EHD_NUM_FIELDS; ++b)
    if (mask & (1u << b)) {
      if (!out[nf]) return EHD_ERR_INVALID_ARG;
      ++nf;
    }
  EHD_CUDA(launch_fields(s->kp, s->b, s->cur, mask, s->stream));
  const size_t N = (size_t)s->kp.N;
  for (int j = 0; j < nf; ++j) {
    if (mem == EHD_DEVICE) {
      EHD_CUDA(cudaMemcpyAsync(out[j], s->b.io + j * N, N * sizeof(float),
                               cudaMemcpyDeviceToDevice, s->stream));
    } else {
      EHD_CUDA(cudaMemcpyAsync(s->h_stage + j * N, s->b.io + j * N, N * sizeof(float),
                               cudaMemcpyDeviceToHost, s->stream));
    }
  }
  EHD_CUDA(cudaStreamSynchronize(s->stream));
  if (mem == EHD_HOST) {
    double* dst[EHD_NUM_FIELDS];
    const float* src[EHD_NUM_FIELDS];
    for (int j = 0; j < nf; ++j) {
      dst[j] = static_cast<double*>(out[j]);
      src[j] = s->h_stage + j * N;
    }
    convert(dst, src, nf, N);
  }
  return EHD_OK;
}

// State blob: header, then populations (27 N), potential populations (8 N), lagged
// quantities (6 N) and the phi of the last potential solve (N), all float32.
struct StateHeader {
  uint64_t magic;
  int32_t nx, ny;
  int64_t n;
  int32_t history_valid, last_k;
  int32_t precision, pad;
  float psc[3], pad2;
};

size_t pop_bytes(const KParams& k) {
  return k.half ? (sizeof(float) * NP32_HALF + sizeof(__half) * 24) * (size_t)k.N
                : sizeof(float) * NP32 * (size_t)k.N;
}

int ehd_state_bytes(const ehd_sim* s, size_t* bytes) {
  if (!s || !bytes) return EHD_ERR_INVALID_ARG;
  *bytes = sizeof(StateHeader) + pop_bytes(s->kp) + sizeof(float) * (size_t)s->kp.N * (NH + NHIST + 1);
  return EHD_OK;
}

int ehd_save_state(ehd_sim* s, void* buf, size_t bytes) {
  size_t need;
  if (!s || !buf || ehd_state_bytes(s, &need) != EHD_OK || bytes < need)
    return EHD_ERR_INVALID_ARG;
  const size_t N = (size_t)s->kp.N;
  EHD_CUDA(cudaMemcpyAsync(s->h_ctl, s->b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
  EHD_CUDA(cudaStreamSynchronize(s->stream));
  StateHeader hd{};
  hd.magic = STATE_MAGIC;
  hd.nx = s->P.nx;
  hd.ny = s->P.ny;
  hd.n = s->n;
  hd.history_valid = s->history_valid ? 1 : 0;
  hd.last_k = s->last_k;
  hd.precision = s->P.precision;
  for (int f = 0; f < 3; ++f) hd.psc[f] = s->kp.psc[f];
  char* p = static_cast<char*>(buf);
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  const Pops pc = pops_copy(s->kp, s->b, s->cur);
  const float* h = s->b.h + (size_t)s->h_ctl->parity * NH * N;
  if (s->kp.half) {
    EHD_CUDA(cudaMemcpyAsync(p, pc.p32, sizeof(float) * NP32_HALF * N, cudaMemcpyDeviceToHost,
                             s->stream));
    p += sizeof(float) * NP32_HALF * N;
    EHD_CUDA(cudaMemcpyAsync(p, pc.p16, sizeof(__half) * 24 * N, cudaMemcpyDeviceToHost, s->stream));
    p += sizeof(__half) * 24 * N;
  } else {
    EHD_CUDA(cudaMemcpyAsync(p, pc.p32, sizeof(float) * NP32 * N, cudaMemcpyDeviceToHost,
                             s->stream));
    p += sizeof(float) * NP32 * N;
  }
  EHD_CUDA(cudaMemcpyAsync(p, h, sizeof(float) * NH * N, cudaMemcpyDeviceToHost, s->stream));
  p += sizeof(float) * NH * N;
  EHD_CUDA(cudaMemcpyAsync(p, s->b.hist, sizeof(float) * NHIST * N, cudaMemcpyDeviceToHost,
                           s->stream));
  p += sizeof(float) * NHIST * N;
  EHD_CUDA(cudaMemcpyAsync(p, s->b.phi, sizeof(float) * N, cudaMemcpyDeviceToHost, s->stream));
  EHD_CUDA(cudaStreamSynchronize(s->stream));
  return EHD_OK;
}

int ehd_load_state(ehd_sim* s, const void* buf, size_t bytes) {
  size_t need;
  if (!s || !buf || ehd_state_bytes(s, &need) != EHD_OK || bytes < need)
    return EHD_ERR_INVALID_ARG;
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (hd.magic != STATE_MAGIC || hd.nx != s->P.nx || hd.ny != s->P.ny ||
      hd.precision != s->P.precision)
    return EHD_ERR_INVALID_ARG;
  const size_t N = (size_t)s->kp.N;
  const char* p = static_cast<const char*>(buf) + sizeof(hd);
  s->cur = 0;
  if (s->kp.half) {
    for (int f = 0; f < 3; ++f) {
      s->kp.psc[f] = hd.psc[f];
      s->kp.ipsc[f] = 1.0f / hd.psc[f];
    }
    destroy_graphs(s);
    s->graphs_tried = false;
  }
  const Pops pc = pops_copy(s->kp, s->b, 0);
  if (s->kp.half) {
    EHD_CUDA(cudaMemcpyAsync(pc.p32, p, sizeof(float) * NP32_HALF * N, cudaMemcpyHostToDevice,
                             s->stream));
    p += sizeof(float) * NP32_HALF * N;
    EHD_CUDA(cudaMemcpyAsync(pc.p16, p, sizeof(__half) * 24 * N, cudaMemcpyHostToDevice, s->stream));
    p += sizeof(__half) * 24 * N;
  } else {
    EHD_CUDA(cudaMemcpyAsync(pc.p32, p, sizeof(float) * NP32 * N, cudaMemcpyHostToDevice,
                             s->stream));
    p += sizeof(float) * NP32 * N;
  }
  EHD_CUDA(cudaMemcpyAsync(s->b.h, p, sizeof(float) * NH * N, cudaMemcpyHostToDevice, s->stream));
  p += sizeof(float) * NH * N;
  EHD_CUDA(cudaMemcpyAsync(s->b.hist, p, sizeof(float) * NHIST * N, cudaMemcpyHostToDevice,
                           s->stream));
  p += sizeof(float) * NHIST * N;
  EHD_CUDA(cudaMemcpyAsync(s->b.phi, p, sizeof(float) * N, cudaMemcpyHostToDevice, s->stream));
  EHD_CUDA(cudaMemsetAsync(&s->b.ctl->parity, 0, sizeof(int), s->stream));
  // the restored state is judged on its own: a non-finite flag of the replaced one goes
  EHD_CUDA(cudaMemsetAsync(&s->b.ctl->nonfinite, 0, sizeof(int), s->stream));
  s->n = hd.n;
  s->history_valid = hd.history_valid != 0;
  s->last_k = hd.last_k;
  EHD_CUDA(launch_step_set(s->kp, s->b, 0, s->n, s->history_valid ? 0 : 1, s->stream));
  EHD_CUDA(cudaStreamSynchronize(s->stream));
  return EHD_OK;
}

}  // extern "C"
