// Potential solve for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc (or any allocating routine): code that runs
// inside a host-side memory budget enforced elsewhere, callers that hand out all device
// memory up front from their own pool, or plug-ins loaded into a process whose allocator
// they do not own.  ehd_potential_solve_noalloc serves them: it runs the potential
// sub-iteration loop (the same arithmetic as the library's streaming potential kernel) on
// arrays the caller passes, and keeps the only scratch the kernel needs -- one pair of
// FP64 partial sums per CTA and the loop-control block -- in a file-scope device array of
// fixed size.  That array exists on every GPU that loads this library, for the life of
// the process.
//
// Limits and behaviour:
//   * the lattice's tiling into 32 x 16 tiles may have at most NA_MAX_CTAS = 4096 tiles,
//     ceil(nx / 32) * ceil(ny / 16) <= 4096 (so at most 2,097,152 nodes, fewer when the
//     sizes are not multiples of the tile); other lattices are rejected with
//     EHD_ERR_TOO_LARGE before anything is queued.  Every kernel of the solve runs at
//     most that many CTAs, one scratch partial each;
//   * the first call on a device looks up the array's device address (once, with that
//     device current); make that first call before any stream capture begins;
//   * every call shares the one array and clears the loop control before it starts; two
//     calls whose work overlaps on the GPU (different streams, or threads) race on it and
//     must not be issued concurrently.
#include <mutex>

#include "../../include/ehd.h"
#include "ehd_internal.cuh"

namespace ehd {
namespace {

constexpr int NA_TX = 32;
constexpr int NA_TY = 16;
constexpr int NA_THREADS = 256;
constexpr int NA_MAX_CTAS = 4096;
constexpr int NA_MAX_DEVICES = 64;

struct NoAllocScratch {
  Ctl ctl;
  double2 partials[NA_MAX_CTAS];
};

// The fixed scratch.  Host code may not use this name as an address (in host code it
// names a host-side stand-in); the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_setup_mutex;
NoAllocScratch* g_scratch_ptr[NA_MAX_DEVICES] = {};

// Loop set-up for one call: control cleared, rule and wall values stored.
__global__ void k_na_setup(NoAllocScratch* sc, double tol, int min_iter, int max_iter,
                           int fixed_iter, float vw_b, float vw_t) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Ctl& c = sc->ctl;
  c.iter = 0;
  c.done = 0;
  c.converged = 0;
  c.parity = 0;
  c.rel = 0.0;
  c.tol = tol;
  c.min_iter = min_iter;
  c.max_iter = max_iter;
  c.fixed_iter = fixed_iter;
  c.nonfinite = 0;
  c.sum_phi = 0.0;
  c.sum_q = 0.0;
  c.mean_q = 0.0f;
  c.ticket_m = 0u;
  c.ticket_p = 0u;
  c.vw_b = vw_b;
  c.vw_t = vw_t;
}

// Mean of q over the lattice (for the neutralised source), FP64, last CTA writes it.
// At most NA_MAX_CTAS CTAs (one partial each in the fixed scratch), each thread striding
// over the lattice.
__global__ void __launch_bounds__(256) k_na_mean(int N, const float* __restrict__ q,
                                                 NoAllocScratch* sc) {
  __shared__ double s_w[8];
  __shared__ int s_last;
  double v = 0.0;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += gridDim.x * blockDim.x)
    v += (double)q[idx];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < 8; ++w) a += s_w[w];
    sc->partials[blockIdx.x] = make_double2(a, 0.0);
    __threadfence();
    s_last = atomicAdd(&sc->ctl.ticket_m, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double a = 0.0;
  for (int j = 0; j < (int)gridDim.x; ++j) a += __ldcg(&sc->partials[j]).x;
  sc->ctl.mean_q = (float)(a / (double)N);
  sc->ctl.ticket_m = 0u;
}

// One potential sub-iteration (Eq. weq53), the streaming kernel's arithmetic, with the
// forcing coefficient a formed from phi on the fly and the scratch in the fixed array.
__global__ void __launch_bounds__(NA_THREADS) k_poisson_noalloc(
    KParams k, const float* __restrict__ phi, const float* __restrict__ q,
    float* __restrict__ h0, float* __restrict__ h1, NoAllocScratch* sc) {
  constexpr int RX = NA_TX + 2, RY = NA_TY + 2;
  __shared__ float sm[8][RY][RX];
  __shared__ float sphi[NA_TY][NA_TX];
  __shared__ double s_w[NA_THREADS / 32][2];
  __shared__ int s_last;
  Ctl* ctl = &sc->ctl;
  // the same control words for every thread, written only by a launch's last CTA after
  // every CTA has read them: the read-only path merges them per SM
  if (__ldg(&ctl->done)) return;
  const int parity = __ldg(&ctl->parity);
  const float qshift = k.neutralize ? __ldg(&ctl->mean_q) : 0.0f;
  const float vw_b = __ldg(&ctl->vw_b), vw_t = __ldg(&ctl->vw_t);
  const int nx = k.nx, ny = k.ny;
  const size_t N = (size_t)k.N;
  const float* __restrict__ src = parity ? h1 : h0;
  float* __restrict__ dst = parity ? h0 : h1;
  const int x0 = blockIdx.x * NA_TX, y0 = blockIdx.y * NA_TY;
  const float om = k.omega_h;

  for (int t = threadIdx.x; t < RX * RY; t += NA_THREADS) {
    const int ly = t / RX, lx = t - ly * RX;
    int gy = y0 + ly - 1;
    if (k.walls) {
      if (gy < 0 || gy >= ny) continue;
    } else {
      gy = wrap(gy, ny);
    }
    const int gx = wrap(x0 + lx - 1, nx);
    const size_t idx = (size_t)gy * nx + gx;
    float h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = __ldg(src + i * N + idx);
    const float ph = __ldg(phi + idx);
    const float eh = eps_hat_of(k, ph);
    const float a = eh / (k.cs2tauh * (eh + k.cs2tauh));
    const float varphi = h_varphi(h_sum8(h));
    float m1x, m1y;
    h_moment1(h, m1x, m1y);
    const float qs = 0.125f * (__ldg(q + idx) - qshift);
#pragma unroll
    for (int i = 1; i < 9; ++i) sm[i - 1][ly][lx] = h_star(i, h[i - 1], om, varphi, a, m1x, m1y, qs);
    if (lx >= 1 && lx <= NA_TX && ly >= 1 && ly <= NA_TY) sphi[ly - 1][lx - 1] = varphi;
  }
  __syncthreads();

  float num = 0.0f, den = 0.0f;
  for (int t = threadIdx.x; t < NA_TX * NA_TY; t += NA_THREADS) {
    const int ly = t / NA_TX, lx = t - ly * NA_TX;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx >= nx || gy >= ny) continue;
    const size_t idx = (size_t)gy * nx + gx;
    float hn[8];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const int sy = gy - cy(i);
      float v;
      if (k.walls && (sy < 0 || sy >= ny)) {
        v = h_wall(i, sm[opp(i) - 1][ly + 1][lx + 1], sy < 0 ? vw_b : vw_t);
      } else {
        v = sm[i - 1][ly + 1 - cy(i)][lx + 1 - cx(i)];
      }
      dst[(i - 1) * N + idx] = v;
      hn[i - 1] = v;
    }
    h_change(h_varphi(h_sum8(hn)), sphi[ly][lx], num, den);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_w[threadIdx.x >> 5][0] = (double)num;
    s_w[threadIdx.x >> 5][1] = (double)den;
  }
  __syncthreads();
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < NA_THREADS / 32; ++w) {
      a += s_w[w][0];
      b += s_w[w][1];
    }
    sc->partials[bid] = make_double2(a, b);
    __threadfence();
    s_last = atomicAdd(&ctl->ticket_p, 1u) == (unsigned)nblocks - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ double s_red[NA_THREADS][2];
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < nblocks; j += NA_THREADS) {
    const double2 v = __ldcg(&sc->partials[j]);
    a += v.x;
    b += v.y;
  }
  s_red[threadIdx.x][0] = a;
  s_red[threadIdx.x][1] = b;
  __syncthreads();
  for (int o = NA_THREADS / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s_red[threadIdx.x][0] += s_red[threadIdx.x + o][0];
      s_red[threadIdx.x][1] += s_red[threadIdx.x + o][1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nm = s_red[0][0], dn = s_red[0][1];
    double rel;
    if (nm == 0.0 && dn == 0.0)
      rel = 0.0;
    else if (dn == 0.0)
      rel = __longlong_as_double(0x7ff0000000000000ll);
    else
      rel = sqrt(nm / dn);
    const int it = ctl->iter + 1;
    ctl->iter = it;
    ctl->parity = parity ^ 1;
    ctl->rel = rel;
    int done, conv;
    if (ctl->fixed_iter > 0) {
      done = it >= ctl->fixed_iter;
      conv = 1;
    } else {
      conv = (it >= ctl->min_iter) && (rel < ctl->tol);
      done = conv || it >= ctl->max_iter;
    }
    ctl->converged = conv;
    ctl->done = done;
    ctl->ticket_p = 0u;
    __threadfence();
  }
}

// Device address of the fixed scratch for the current device, looked up once.
int scratch_for_current_device(NoAllocScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
    return EHD_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return EHD_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_scratch_ptr[dev];
  return EHD_OK;
}

}  // namespace
}  // namespace ehd

using namespace ehd;

extern "C" int ehd_potential_solve_noalloc(const ehd_params* params, const float* phi,
                                           const float* q, float* h, float* h_work,
                                           void* stream, int* iters, double* rel_change) {
  if (!params || !phi || !q || !h || !h_work) return EHD_ERR_INVALID_ARG;
  const ehd_params& P = *params;
  if (P.nx < 1 || P.ny < 1 || (P.walls_y != 0 && P.walls_y != 1) || !(P.eps_v > 0) ||
      !(P.eps_l > 0) || P.poisson_max_iter < 1 || P.poisson_min_iter < 1 ||
      P.poisson_fixed_iter < 0 || (P.poisson_fixed_iter == 0 && !(P.poisson_tol > 0)) ||
      P.potential_scheme != EHD_SCHEME_IMPROVED)
    return EHD_ERR_INVALID_ARG;
  const int gx = (P.nx + NA_TX - 1) / NA_TX, gy = (P.ny + NA_TY - 1) / NA_TY;
  if ((long long)gx * gy > NA_MAX_CTAS) return EHD_ERR_TOO_LARGE;
  const double cs2 = 1.0 / 3.0;
  const double tau_h = 0.5 + P.eps_v / cs2;
  if (tau_h <= 0.5 + 1e-3) return EHD_ERR_UNSTABLE_PARAMS;
  KParams k{};
  k.nx = P.nx;
  k.ny = P.ny;
  k.N = P.nx * P.ny;
  k.walls = P.walls_y;
  k.neutralize = P.neutralize_charge ? 1 : 0;
  k.eps_v = (float)P.eps_v;
  k.deps = (float)(P.eps_v - P.eps_l);
  k.omega_h = (float)(1.0 / tau_h);
  k.cs2tauh = (float)(cs2 * tau_h);
  // wall potentials at the parameters' starting step (ramp fraction r, as for a step)
  double r = 1.0;
  if (P.ramp_steps > 0) {
    r = (double)P.start_step / (double)P.ramp_steps;
    r = r < 1.0 ? r : 1.0;
  }
  const float vw_b = (float)(r * P.varphi_bottom), vw_t = (float)(r * P.varphi_top);

  NoAllocScratch* sc = nullptr;
  const int st = scratch_for_current_device(&sc);
  if (st != EHD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_na_setup<<<1, 32, 0, s>>>(sc, P.poisson_tol, P.poisson_min_iter, P.poisson_max_iter,
                              P.poisson_fixed_iter, vw_b, vw_t);
  if (cudaGetLastError() != cudaSuccess) return EHD_ERR_CUDA;
  if (k.neutralize) {
    const int mean_blocks = (k.N + 255) / 256 < NA_MAX_CTAS ? (k.N + 255) / 256 : NA_MAX_CTAS;
    k_na_mean<<<mean_blocks, 256, 0, s>>>(k.N, q, sc);
    if (cudaGetLastError() != cudaSuccess) return EHD_ERR_CUDA;
  }
  const dim3 grid(gx, gy);
  Ctl host_ctl;
  auto read_ctl = [&]() -> int {
    if (cudaMemcpyAsync(&host_ctl, &sc->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return EHD_ERR_CUDA;
    return EHD_OK;
  };
  if (P.poisson_fixed_iter > 0) {
    for (int i = 0; i < P.poisson_fixed_iter; ++i)
      k_poisson_noalloc<<<grid, NA_THREADS, 0, s>>>(k, phi, q, h, h_work, sc);
    if (cudaGetLastError() != cudaSuccess || read_ctl() != EHD_OK) return EHD_ERR_CUDA;
  } else {
    int queued = 0, chunk = 2;
    for (;;) {
      for (int i = 0; i < chunk; ++i)
        k_poisson_noalloc<<<grid, NA_THREADS, 0, s>>>(k, phi, q, h, h_work, sc);
      queued += chunk;
      if (cudaGetLastError() != cudaSuccess || read_ctl() != EHD_OK) return EHD_ERR_CUDA;
      if (host_ctl.done) break;
      if (queued > P.poisson_max_iter + 2) return EHD_ERR_CUDA;
      chunk = chunk * 2;
      if (chunk > P.poisson_max_iter - host_ctl.iter + 1) chunk = P.poisson_max_iter - host_ctl.iter + 1;
      if (chunk < 1) chunk = 1;
    }
  }
  // the result ends in h_work after an odd number of sub-iterations: bring it to h
  if (host_ctl.parity == 1) {
    if (cudaMemcpyAsync(h, h_work, sizeof(float) * 8 * (size_t)k.N, cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return EHD_ERR_CUDA;
  }
  if (iters) *iters = host_ctl.iter;
  if (rel_change) *rel_change = host_ctl.rel;
  return host_ctl.converged ? EHD_OK : EHD_ERR_NOT_CONVERGED;
}
