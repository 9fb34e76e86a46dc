// Slab decomposition of one lattice: the whole-lattice step computed by S slabs of
// consecutive rows, each with its own device buffers, exchanging the rows each pass needs
// from its neighbours.  This is the layout a lattice too large for one GPU takes across
// several (one slab per device); here every slab lives on the same GPU and the exchange
// is a gather kernel between the slabs' buffers.
//
// Each slab stores its interior rows plus one ghost row below and one above (stored rows
// 0 and ny_s + 1).  The kernels of the single-lattice step run on every slab unchanged in
// their arithmetic; at a cut they read the ghost row (stencils, the potential kernel's
// recomputed ring) or push into it (the coupled pass), instead of applying the wall rule
// or the periodic wrap.  What crosses a cut, per pass:
//   after the moments pass          phi and the potential coefficients (a, q): one row each
//                                   way (the stencils, the potential kernel's ring);
//   after each potential
//   sub-iteration                   the 8 potential populations of the boundary row, each
//                                   way (the next sub-iteration's ring);
//   after the coupled pass          the g, l, f populations pushed across the cut: 3
//                                   directions x 3 fields, each way.
// The global reductions -- the stopping sums of every sub-iteration and the FP64 sums of
// phi and q of the moments pass -- are formed per slab by the usual kernels and combined
// in a fixed slab order by one thread, which takes the one decision every slab follows.
// With a fixed sub-iteration count the result is the single lattice's, bit for bit
// (the per-node arithmetic and every input value are the same); with the stopping rule
// the combined sums round differently from the single lattice's, so a decision can
// differ where the relative change lies within rounding of the tolerance.
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ehd.h"
#include "ehd_internal.cuh"
#include "sim_internal.h"

namespace ehd {
namespace {

constexpr int MAX_SLABS = 64;

// One exchanged row: n floats from src to dst; with pctl set, each pointer is offset by
// its parity stride times the current parity of the potential populations.
struct HaloRow {
  const float* src;
  float* dst;
  long long src_pstride, dst_pstride;
  const Ctl* pctl;
  int n;
  int pad;
};

__global__ void k_halo(const HaloRow* __restrict__ rows) {
  const HaloRow r = rows[blockIdx.y];
  const long long par = r.pctl ? (long long)ld_cg(&r.pctl->parity) : 0;
  const float* src = r.src + par * r.src_pstride;
  float* dst = r.dst + par * r.dst_pstride;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r.n; i += gridDim.x * blockDim.x)
    dst[i] = src[i];
}

struct SlabCtls {
  Ctl* c[MAX_SLABS];
  int n;
  int pad;
  double nodes;  // interior nodes of the whole lattice
};

// After every slab's moments pass: the FP64 sums of phi and q over the whole lattice (slab
// sums added in slab order), the mean charge of the neutralised source, and one
// non-finite flag for all (with which every slab's solve stops after one sub-iteration).
__global__ void k_slab_moments(SlabCtls t) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double sp = 0.0, sq = 0.0;
  int bad = 0;
  for (int s = 0; s < t.n; ++s) {
    sp += ld_cg(&t.c[s]->sum_phi);
    sq += ld_cg(&t.c[s]->sum_q);
    bad |= ld_cg(&t.c[s]->nonfinite);
  }
  const float mean_q = (float)(sq / t.nodes);
  for (int s = 0; s < t.n; ++s) {
    Ctl* c = t.c[s];
    c->sum_phi = sp;
    c->sum_q = sq;
    c->mean_q = mean_q;
    c->nonfinite = bad;
    if (bad) {
      c->fixed_iter = 0;
      c->min_iter = 1;
      c->max_iter = 1;
    }
  }
  __threadfence();
}

// After every slab's potential sub-iteration: the stopping rule of Algorithm 1 on the
// combined sums, the same arithmetic as the single lattice's last CTA; every slab's loop
// control advances alike.
__global__ void k_slab_decide(SlabCtls t, cudaGraphConditionalHandle cond, int use_cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Ctl* c0 = t.c[0];
  if (ld_cg(&c0->done)) {
    if (use_cond) cudaGraphSetConditional(cond, 0u);
    return;
  }
  double nm = 0.0, dn = 0.0;
  for (int s = 0; s < t.n; ++s) {
    nm += ld_cg(&t.c[s]->slab_num);
    dn += ld_cg(&t.c[s]->slab_den);
  }
  double rel;
  if (nm == 0.0 && dn == 0.0)
    rel = 0.0;
  else if (dn == 0.0)
    rel = __longlong_as_double(0x7ff0000000000000ll);  // +inf
  else
    rel = sqrt(nm / dn);
  const int it = c0->iter + 1;
  const int parity = c0->parity ^ 1;
  int done, conv;
  if (c0->fixed_iter > 0) {
    done = it >= c0->fixed_iter;
    conv = 1;
  } else {
    conv = (it >= c0->min_iter) && (rel < c0->tol);
    done = conv || it >= c0->max_iter;
  }
  for (int s = 0; s < t.n; ++s) {
    Ctl* c = t.c[s];
    c->iter = it;
    c->parity = parity;
    c->rel = rel;
    c->converged = conv;
    c->done = done;
  }
  __threadfence();
  if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
}

cudaError_t add_kernel(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                       cudaGraphNode_t* out, void* func, dim3 grid, dim3 block, void** args) {
  cudaKernelNodeParams p = {};
  p.func = func;
  p.gridDim = grid;
  p.blockDim = block;
  p.kernelParams = args;
  return cudaGraphAddKernelNode(out, g, deps, nd, &p);
}

}  // namespace
}  // namespace ehd

using namespace ehd;

// Row groups of the exchange table.
enum { G_PHIAQ = 0, G_H = 1, G_POPS0 = 2, G_POPS1 = 3, G_TMP = 4, G_COUNT = 5 };

struct ehd_slabs {
  ehd_params P;                    // the whole lattice
  int S = 0;
  std::vector<ehd_sim*> sims;
  std::vector<int> y0, ny;         // first row and height of each slab
  cudaStream_t stream = nullptr;
  SlabCtls ctls{};
  HaloRow* d_rows = nullptr;       // the exchange table on the device
  int first[G_COUNT] = {}, count[G_COUNT] = {};
  int max_n = 0;                   // longest row, floats
  cudaGraphExec_t step_exec[2] = {nullptr, nullptr};
  cudaGraphExec_t solve_exec = nullptr;
  int cur = 0;
  int64_t n = 0;
};

namespace {

int destroy_and(ehd_slabs* t, int code) {
  ehd_slabs_destroy(t);
  return code;
}

// Queues one exchange group on the stream.
cudaError_t halo(ehd_slabs* t, int grp, cudaStream_t st) {
  if (t->count[grp] == 0) return cudaSuccess;
  const int bx = (t->max_n + 255) / 256;
  k_halo<<<dim3(bx, t->count[grp]), 256, 0, st>>>(t->d_rows + t->first[grp]);
  return cudaGetLastError();
}

cudaError_t add_halo(ehd_slabs* t, int grp, cudaGraph_t g, const cudaGraphNode_t* deps,
                     size_t nd, cudaGraphNode_t* out) {
  // one slab between walls has no cut: an empty node keeps the order of the graph
  if (t->count[grp] == 0) return cudaGraphAddEmptyNode(out, g, deps, nd);
  const HaloRow* rows = t->d_rows + t->first[grp];
  void* args[] = {&rows};
  return add_kernel(g, deps, nd, out, (void*)k_halo, dim3((t->max_n + 255) / 256, t->count[grp]),
                    dim3(256), args);
}

// Adds moments -> combine -> (phi, a, q) exchange -> while { potential sub-iteration on
// every slab -> decide -> exchange of h } to g after `dep` (nullable); *tail is the
// while node.
cudaError_t add_solve(ehd_slabs* t, cudaGraph_t g, int cur, const cudaGraphNode_t* dep,
                      cudaGraphNode_t* tail) {
  const ehd_params& P = t->P;
  cudaError_t e;
  std::vector<cudaGraphNode_t> mn(t->S);
  for (int s = 0; s < t->S; ++s)
    if ((e = add_moments_node(g, dep, dep ? 1 : 0, &mn[s], t->sims[s]->kp, t->sims[s]->b, cur,
                              P.poisson_tol, P.poisson_min_iter, P.poisson_max_iter,
                              P.poisson_fixed_iter)) != cudaSuccess)
      return e;
  cudaGraphNode_t comb, hx, wn;
  SlabCtls c = t->ctls;
  void* cargs[] = {&c};
  if ((e = add_kernel(g, mn.data(), mn.size(), &comb, (void*)k_slab_moments, dim3(1), dim3(32),
                      cargs)) != cudaSuccess ||
      (e = add_halo(t, G_PHIAQ, g, &comb, 1, &hx)) != cudaSuccess)
    return e;
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
    return e;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if ((e = cudaGraphAddNode(&wn, g, &hx, nullptr, 1, &cp)) != cudaSuccess) return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  std::vector<cudaGraphNode_t> pn(t->S);
  for (int s = 0; s < t->S; ++s)
    if ((e = add_poisson_node_nocond(body, nullptr, 0, &pn[s], t->sims[s]->kp, t->sims[s]->b)) !=
        cudaSuccess)
      return e;
  cudaGraphNode_t dn, hh;
  int use = 1;
  void* dargs[] = {&c, &h, &use};
  if ((e = add_kernel(body, pn.data(), pn.size(), &dn, (void*)k_slab_decide, dim3(1), dim3(32),
                      dargs)) != cudaSuccess ||
      (e = add_halo(t, G_H, body, &dn, 1, &hh)) != cudaSuccess)
    return e;
  *tail = wn;
  return cudaSuccess;
}

cudaError_t build_graphs(ehd_slabs* t) {
  cudaError_t e;
  for (int cur = 0; cur < 2; ++cur) {
    cudaGraph_t g;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
    cudaGraphNode_t wn, hp;
    std::vector<cudaGraphNode_t> cn(t->S);
    e = add_solve(t, g, cur, nullptr, &wn);
    for (int s = 0; s < t->S && e == cudaSuccess; ++s)
      e = add_coupled_node(g, &wn, 1, &cn[s], t->sims[s]->kp, t->sims[s]->b, cur);
    if (e == cudaSuccess) e = add_halo(t, cur == 0 ? G_POPS1 : G_POPS0, g, cn.data(), cn.size(), &hp);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&t->step_exec[cur], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
  }
  cudaGraph_t g;
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
  cudaGraphNode_t wn;
  e = add_solve(t, g, 0, nullptr, &wn);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&t->solve_exec, g, 0);
  cudaGraphDestroy(g);
  return e;
}

// The exchange table: for every cut (slab a below slab b), the rows each group moves.
void build_rows(ehd_slabs* t, std::vector<HaloRow> (&grp)[G_COUNT]) {
  const int nx = t->P.nx;
  const int cuts = t->P.walls_y ? t->S - 1 : (t->S > 1 ? t->S : 0);
  auto row = [&](float* base, int r) { return base + (size_t)r * nx; };
  auto add = [&](int g, const float* src, float* dst, int n, long long sps = 0,
                 long long dps = 0, const Ctl* pctl = nullptr) {
    grp[g].push_back(HaloRow{src, dst, sps, dps, pctl, n, 0});
    if (n > t->max_n) t->max_n = n;
  };
  for (int c = 0; c < cuts; ++c) {
    ehd_sim* A = t->sims[c];
    ehd_sim* B = t->sims[(c + 1) % t->S];
    const int na = t->ny[c];
    const size_t NA = (size_t)A->kp.N, NB = (size_t)B->kp.N;
    // phi and the coefficients: A's top ghost <- B's first row, B's bottom ghost <- A's last
    add(G_PHIAQ, row(B->b.phi, 1), row(A->b.phi, na + 1), nx);
    add(G_PHIAQ, row(A->b.phi, na), row(B->b.phi, 0), nx);
    float* aqa = reinterpret_cast<float*>(A->b.aq);
    float* aqb = reinterpret_cast<float*>(B->b.aq);
    add(G_PHIAQ, aqb + 2 * (size_t)nx, aqa + 2 * (size_t)(na + 1) * nx, 2 * nx);
    add(G_PHIAQ, aqa + 2 * (size_t)na * nx, aqb, 2 * nx);
    // phi of the current populations, for output
    add(G_TMP, row(B->b.tmp, 1), row(A->b.tmp, na + 1), nx);
    add(G_TMP, row(A->b.tmp, na), row(B->b.tmp, 0), nx);
    // potential populations of the current parity, each of the 8 directions
    for (int j = 0; j < NH; ++j) {
      add(G_H, row(B->b.h + j * NB, 1), row(A->b.h + j * NA, na + 1), nx, NH * (long long)NB,
          NH * (long long)NA, A->b.ctl);
      add(G_H, row(A->b.h + j * NA, na), row(B->b.h + j * NB, 0), nx, NH * (long long)NA,
          NH * (long long)NB, A->b.ctl);
    }
    // populations pushed across the cut into the ghost rows, for each population copy:
    // upward (directions 2, 5, 6) into B's first row, downward (4, 7, 8) into A's last
    for (int copy = 0; copy < 2; ++copy) {
      float* pa = pops_copy(A->kp, A->b, copy).p32;
      float* pb = pops_copy(B->kp, B->b, copy).p32;
      for (int f = 0; f < 3; ++f) {
        for (int i : {2, 5, 6})
          add(G_POPS0 + copy, row(pa + (f * 9 + i) * NA, na + 1), row(pb + (f * 9 + i) * NB, 1), nx);
        for (int i : {4, 7, 8})
          add(G_POPS0 + copy, row(pb + (f * 9 + i) * NB, 0), row(pa + (f * 9 + i) * NA, na), nx);
      }
    }
  }
}

}  // namespace

extern "C" {

int ehd_slabs_create(const ehd_params* params, int nslabs, void* stream, ehd_slabs** out) {
  if (!out) return EHD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!params || nslabs < 1 || nslabs > MAX_SLABS || params->ny < nslabs ||
      params->precision != EHD_FP32)
    return EHD_ERR_INVALID_ARG;
  ehd_slabs* t = new (std::nothrow) ehd_slabs();
  if (!t) return EHD_ERR_NOMEM;
  t->P = *params;
  t->S = nslabs;
  t->stream = static_cast<cudaStream_t>(stream);
  t->n = params->start_step;
  const int NY = params->ny;
  for (int s = 0; s < nslabs; ++s) {
    const int a = (int)((long long)NY * s / nslabs), b = (int)((long long)NY * (s + 1) / nslabs);
    t->y0.push_back(a);
    t->ny.push_back(b - a);
  }
  for (int s = 0; s < nslabs; ++s) {
    // each slab is a simulation of its rows plus the two ghost rows, on the streaming loop
    ehd_params q = *params;
    q.ny = t->ny[s] + 2;
    q.poisson_loop = EHD_LOOP_STREAM;
    q.tile_rows = 0;
    ehd_sim* sim = nullptr;
    const int st = sim_create(&q, nullptr, 0, stream, 0, &sim);
    if (st != EHD_OK) return destroy_and(t, st);
    t->sims.push_back(sim);
    KParams& k = sim->kp;
    k.ny = t->ny[s];
    k.nint = params->nx * t->ny[s];
    k.row0 = 1;
    const bool periodic_cut = !params->walls_y && nslabs > 1;
    k.halo_lo = (s > 0 || periodic_cut) ? 1 : 0;
    k.halo_hi = (s < nslabs - 1 || periodic_cut) ? 1 : 0;
    k.slab = 1;
    k.y_global0 = t->y0[s];
    k.ny_global = NY;
    t->ctls.c[s] = sim->b.ctl;
  }
  t->ctls.n = nslabs;
  t->ctls.nodes = (double)params->nx * NY;
  std::vector<HaloRow> grp[G_COUNT];
  build_rows(t, grp);
  std::vector<HaloRow> all;
  for (int g = 0; g < G_COUNT; ++g) {
    t->first[g] = (int)all.size();
    t->count[g] = (int)grp[g].size();
    all.insert(all.end(), grp[g].begin(), grp[g].end());
  }
  if (!all.empty()) {
    if (cudaMalloc(&t->d_rows, sizeof(HaloRow) * all.size()) != cudaSuccess) {
      cudaGetLastError();
      return destroy_and(t, EHD_ERR_NOMEM);
    }
    if (cudaMemcpy(t->d_rows, all.data(), sizeof(HaloRow) * all.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
      return destroy_and(t, EHD_ERR_CUDA);
  }
  if (build_graphs(t) != cudaSuccess) {
    cudaGetLastError();
    return destroy_and(t, EHD_ERR_CUDA);
  }
  *out = t;
  return EHD_OK;
}

int ehd_slabs_set_fields(ehd_slabs* t, const double* phi, const double* q, const double* ux,
                         const double* uy, const double* p) {
  if (!t || !phi || !q || !ux || !uy) return EHD_ERR_INVALID_ARG;
  const int nx = t->P.nx, NY = t->P.ny;
  const double* src[5] = {phi, q, ux, uy, p};
  const int nf = p ? 5 : 4;
  for (int s = 0; s < t->S; ++s) {
    ehd_sim* sim = t->sims[s];
    const size_t N = (size_t)sim->kp.N;
    // stored rows 0 .. ny_s + 1 are lattice rows y0 - 1 .. y0 + ny_s (wrapped; at a wall
    // the ghost row is never read, the edge row is copied there)
    for (int f = 0; f < nf; ++f) {
      float* dst = sim->h_stage + f * N;
      for (int r = 0; r < t->ny[s] + 2; ++r) {
        int gy = t->y0[s] + r - 1;
        if (gy < 0) gy = t->P.walls_y ? 0 : gy + NY;
        if (gy >= NY) gy = t->P.walls_y ? NY - 1 : gy - NY;
        const double* in = src[f] + (size_t)gy * nx;
        for (int x = 0; x < nx; ++x) dst[(size_t)r * nx + x] = (float)in[x];
      }
      if (cudaMemcpyAsync(sim->b.io + f * N, dst, N * sizeof(float), cudaMemcpyHostToDevice,
                          t->stream) != cudaSuccess)
        return EHD_ERR_CUDA;
    }
    sim->n = t->P.start_step;
    sim->cur = 0;
    if (cudaMemsetAsync(&sim->b.ctl->parity, 0, sizeof(int), t->stream) != cudaSuccess ||
        cudaMemsetAsync(&sim->b.ctl->nonfinite, 0, sizeof(int), t->stream) != cudaSuccess ||
        launch_step_set(sim->kp, sim->b, 0, sim->n, 1, t->stream) != cudaSuccess ||
        launch_init(sim->kp, sim->b, 0, p != nullptr, t->stream) != cudaSuccess ||
        launch_stats_reset(sim->b, t->stream) != cudaSuccess)
      return EHD_ERR_CUDA;
  }
  t->cur = 0;
  t->n = t->P.start_step;
  // the initial potential populations' boundary rows, then the initial solve
  if (halo(t, G_H, t->stream) != cudaSuccess ||
      cudaGraphLaunch(t->solve_exec, t->stream) != cudaSuccess)
    return EHD_ERR_CUDA;
  ehd_sim* s0 = t->sims[0];
  if (cudaMemcpyAsync(s0->h_ctl, s0->b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, t->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(t->stream) != cudaSuccess)
    return EHD_ERR_CUDA;
  if (s0->h_ctl->nonfinite) return EHD_ERR_NONFINITE;
  return s0->h_ctl->converged ? EHD_OK : EHD_ERR_NOT_CONVERGED;
}

int ehd_slabs_step(ehd_slabs* t, int nsteps, ehd_stats* out) {
  if (!t || nsteps < 0) return EHD_ERR_INVALID_ARG;
  for (int s = 0; s < t->S; ++s)
    if (launch_stats_reset(t->sims[s]->b, t->stream) != cudaSuccess) return EHD_ERR_CUDA;
  for (int k = 0; k < nsteps; ++k) {
    if (cudaGraphLaunch(t->step_exec[t->cur], t->stream) != cudaSuccess) return EHD_ERR_CUDA;
    t->cur ^= 1;
    t->n += 1;
  }
  for (ehd_sim* s : t->sims) {
    s->cur = t->cur;
    s->n = t->n;
    s->history_valid = true;
  }
  ehd_sim* s0 = t->sims[0];
  if (cudaMemcpyAsync(s0->h_stats, s0->b.stats, sizeof(DevStats), cudaMemcpyDeviceToHost,
                      t->stream) != cudaSuccess ||
      cudaStreamSynchronize(t->stream) != cudaSuccess)
    return EHD_ERR_CUDA;
  const DevStats& d = *s0->h_stats;
  if (out) {
    std::memset(out, 0, sizeof(*out));
    out->step = t->n;
    out->steps = d.steps;
    out->poisson_iters_total = d.iters_total;
    out->poisson_iters_min = d.steps ? d.iters_min : 0;
    out->poisson_iters_max = d.iters_max;
    out->not_converged_steps = d.not_converged;
    out->nonfinite = d.nonfinite;
    out->last_rel_change = d.last_rel;
    out->sum_phi = d.sum_phi;
    out->sum_q = d.sum_q;
    out->kernel_launches = (int64_t)nsteps * (2 * t->S + 4) + (int64_t)d.iters_total * (t->S + 2);
  }
  if (d.nonfinite) return EHD_ERR_NONFINITE;
  if (d.not_converged) return EHD_ERR_NOT_CONVERGED;
  return EHD_OK;
}

int ehd_slabs_read_fields(ehd_slabs* t, unsigned mask, double* const* out) {
  if (!t || !out || (mask & ~((1u << EHD_NUM_FIELDS) - 1u))) return EHD_ERR_INVALID_ARG;
  int nf = 0;
  for (int b = 0; b < EHD_NUM_FIELDS; ++b)
    if (mask & (1u << b)) {
      if (!out[nf]) return EHD_ERR_INVALID_ARG;
      ++nf;
    }
  if (!nf) return EHD_OK;
  for (ehd_sim* s : t->sims)
    if (launch_phi_now(s->kp, s->b, t->cur, t->stream) != cudaSuccess) return EHD_ERR_CUDA;
  if (halo(t, G_TMP, t->stream) != cudaSuccess) return EHD_ERR_CUDA;
  const int nx = t->P.nx;
  for (int s = 0; s < t->S; ++s) {
    ehd_sim* sim = t->sims[s];
    const size_t N = (size_t)sim->kp.N, nint = (size_t)sim->kp.nint;
    if (launch_fields_from_phi(sim->kp, sim->b, t->cur, mask, t->stream) != cudaSuccess)
      return EHD_ERR_CUDA;
    for (int j = 0; j < nf; ++j)
      if (cudaMemcpyAsync(sim->h_stage + j * N, sim->b.io + j * N + nx, nint * sizeof(float),
                          cudaMemcpyDeviceToHost, t->stream) != cudaSuccess)
        return EHD_ERR_CUDA;
  }
  if (cudaStreamSynchronize(t->stream) != cudaSuccess) return EHD_ERR_CUDA;
  for (int s = 0; s < t->S; ++s) {
    ehd_sim* sim = t->sims[s];
    const size_t N = (size_t)sim->kp.N, nint = (size_t)sim->kp.nint;
    for (int j = 0; j < nf; ++j) {
      double* dst = out[j] + (size_t)t->y0[s] * nx;
      const float* src = sim->h_stage + j * N;
      for (size_t i = 0; i < nint; ++i) dst[i] = (double)src[i];
    }
  }
  return EHD_OK;
}

int ehd_slabs_exchange_bytes(const ehd_slabs* t, size_t* per_sub_iteration, size_t* per_step) {
  if (!t) return EHD_ERR_INVALID_ARG;
  const size_t nx = (size_t)t->P.nx;
  const size_t cuts = t->P.walls_y ? t->S - 1 : (t->S > 1 ? t->S : 0);
  // per cut and sub-iteration: 8 potential populations each way; per step: phi and (a, q)
  // each way, and 9 pushed populations each way
  if (per_sub_iteration) *per_sub_iteration = cuts * 2 * NH * nx * sizeof(float);
  if (per_step) *per_step = cuts * 2 * (1 + 2 + 9) * nx * sizeof(float);
  return EHD_OK;
}

void ehd_slabs_destroy(ehd_slabs* t) {
  if (!t) return;
  if (t->stream) cudaStreamSynchronize(t->stream);
  for (int c = 0; c < 2; ++c)
    if (t->step_exec[c]) cudaGraphExecDestroy(t->step_exec[c]);
  if (t->solve_exec) cudaGraphExecDestroy(t->solve_exec);
  if (t->d_rows) cudaFree(t->d_rows);
  for (ehd_sim* s : t->sims) ehd_destroy(s);
  delete t;
}

}  // extern "C"
