// Kernels of the coupled step other than the potential sub-iteration:
//   k_init      equilibrium initialisation (Algorithm 1 step 1)
//   k_moments   phi, q and the potential coefficients of the current step, FP64 sums
//   k_coupled   one fused collide-and-push of the g, l and f populations (Algorithm 1
//               steps 2, 4, 5 with the field of step 3), history update
//   k_fields    macroscopic fields for output
#include "ehd_internal.cuh"

namespace ehd {

namespace {


// phi at the 3x3 neighbourhood of interior node (x, y); rows outside a wall are ghost
// values from the wetting rule n_w.grad(phi) = -sqrt(2 beta/kappa) cos(theta) (phi - phi^2)
// (Eq. weq68): ghost = phi_wall_row + a cos(theta) phi (1 - phi) with the first fluid row's
// value.  In a slab, the row beyond a cut is the stored ghost row (the neighbouring slab's
// values).
struct Stencil {
  float c, e, w, n, s, ne, nw, se, sw;
};

__device__ __forceinline__ float ghost(float v, float a_cos) { return v + a_cos * (v - v * v); }

__device__ __forceinline__ Stencil load_stencil(const KParams& k, const StepState& sa,
                                                const float* __restrict__ phi, int x, int y) {
  const int nx = k.nx, ny = k.ny;
#ifdef EHD_CHECKED
  if (x < 0 || x >= nx || y < 0 || y >= ny) {  // never in a correct launch
    checked_index(k, 1, 0);
    x = 0;
    y = 0;
  }
#endif
  if (x > 0 && x + 1 < nx && y > 0 && y + 1 < ny) {
    // away from every edge: the 3 x 3 neighbourhood at fixed offsets
    const float* r = phi + (size_t)(y + k.row0) * nx + x;
    Stencil s;
    s.c = __ldg(r);
    s.e = __ldg(r + 1);
    s.w = __ldg(r - 1);
    s.n = __ldg(r + nx);
    s.ne = __ldg(r + nx + 1);
    s.nw = __ldg(r + nx - 1);
    s.s = __ldg(r - nx);
    s.se = __ldg(r - nx + 1);
    s.sw = __ldg(r - nx - 1);
    return s;
  }
  const int xm = x == 0 ? nx - 1 : x - 1;
  const int xp = x + 1 == nx ? 0 : x + 1;
  Stencil s;
  const float* row = phi + (size_t)(y + k.row0) * nx;
  s.c = __ldg(row + x);
  s.e = __ldg(row + xp);
  s.w = __ldg(row + xm);
  if (k.walls && !k.halo_hi && y + 1 == ny) {
    const float a = k.wet_a * sa.cos_t;
    s.n = ghost(s.c, a);
    s.ne = ghost(s.e, a);
    s.nw = ghost(s.w, a);
  } else {
    // the row above: wrapped, or the stored ghost row beyond a cut (interior row ny)
    const int ry = y + 1 == ny ? (k.halo_hi ? ny : 0) : y + 1;
    const float* r = phi + (size_t)(ry + k.row0) * nx;
    s.n = __ldg(r + x);
    s.ne = __ldg(r + xp);
    s.nw = __ldg(r + xm);
  }
  if (k.walls && !k.halo_lo && y == 0) {
    const float a = k.wet_a * sa.cos_b;
    s.s = ghost(s.c, a);
    s.se = ghost(s.e, a);
    s.sw = ghost(s.w, a);
  } else {
    const int ry = y == 0 ? (k.halo_lo ? -1 : ny - 1) : y - 1;
    const float* r = phi + (size_t)(ry + k.row0) * nx;
    s.s = __ldg(r + x);
    s.se = __ldg(r + xp);
    s.sw = __ldg(r + xm);
  }
  return s;
}

// Isotropic stencils of Sec. 3.2 with w_i / c_s^2 = 1/3 (axis), 1/12 (diagonal).
__device__ __forceinline__ void grad_lap(const Stencil& s, float& gx, float& gy, float& lap) {
  gx = (s.e - s.w) * (1.0f / 3.0f) + (s.ne + s.se - s.nw - s.sw) * (1.0f / 12.0f);
  gy = (s.n - s.s) * (1.0f / 3.0f) + (s.ne + s.nw - s.se - s.sw) * (1.0f / 12.0f);
  lap = (s.e + s.w + s.n + s.s) * (2.0f / 3.0f) + (s.ne + s.nw + s.se + s.sw) * (1.0f / 6.0f) -
        s.c * (10.0f / 3.0f);
}

// varphi = 9/5 sum_{i>0} h_i (Eq. weq55) of node idx from the converged populations.
__device__ __forceinline__ float varphi_node(const float* __restrict__ hs, size_t N, int idx) {
  float h[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) h[i] = __ldg(hs + i * N + idx);
  return h_varphi(h_sum8(h));
}

// varphi at the 3x3 neighbourhood of (x, y); beyond an electrode the ghost value is the
// linear extension through the wall potential, 2 varphi_w - varphi of the first row.
__device__ __forceinline__ Stencil load_varphi_stencil(const KParams& k,
                                                       const float* __restrict__ hs, int x,
                                                       int y, float vw_b, float vw_t) {
  const int nx = k.nx, ny = k.ny;
  const size_t N = (size_t)k.N;
  const int xm = x == 0 ? nx - 1 : x - 1;
  const int xp = x + 1 == nx ? 0 : x + 1;
  Stencil s;
  const int row = (y + k.row0) * nx;
  s.c = varphi_node(hs, N, row + x);
  s.e = varphi_node(hs, N, row + xp);
  s.w = varphi_node(hs, N, row + xm);
  if (k.walls && !k.halo_hi && y + 1 == ny) {
    s.n = 2.0f * vw_t - s.c;
    s.ne = 2.0f * vw_t - s.e;
    s.nw = 2.0f * vw_t - s.w;
  } else {
    const int r = ((y + 1 == ny ? (k.halo_hi ? ny : 0) : y + 1) + k.row0) * nx;
    s.n = varphi_node(hs, N, r + x);
    s.ne = varphi_node(hs, N, r + xp);
    s.nw = varphi_node(hs, N, r + xm);
  }
  if (k.walls && !k.halo_lo && y == 0) {
    s.s = 2.0f * vw_b - s.c;
    s.se = 2.0f * vw_b - s.e;
    s.sw = 2.0f * vw_b - s.w;
  } else {
    const int r = ((y == 0 ? (k.halo_lo ? -1 : ny - 1) : y - 1) + k.row0) * nx;
    s.s = varphi_node(hs, N, r + x);
    s.se = varphi_node(hs, N, r + xp);
    s.sw = varphi_node(hs, N, r + xm);
  }
  return s;
}

// Stored index of the node a population leaving interior node (x, y) in direction i lands
// on, and the direction it lands in: periodic in x; at a wall, half-way bounce-back
// returns it to (x, y) in the opposite direction; beyond a slab's cut it lands in the
// ghost row, from which the exchange hands it to the neighbouring slab.
__device__ __forceinline__ int push_target(const KParams& k, int x, int y, int i, int& dir) {
  int ty = y + cy(i);
  dir = i;
  if (ty < 0 || ty >= k.ny) {
    if (!(ty < 0 ? k.halo_lo : k.halo_hi)) {
      if (k.walls) {
        dir = opp(i);
        return (y + k.row0) * k.nx + x;
      }
      ty = ty < 0 ? k.ny - 1 : 0;
    }
  }
  int tx = x + cx(i);
  tx = tx < 0 ? k.nx - 1 : (tx >= k.nx ? 0 : tx);
  return (ty + k.row0) * k.nx + tx;
}

// FP32 warp sum.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace

// ------------------------------------------------------------------------------------
// Initialisation: populations at equilibrium (Eqs. weq40, weq46, weq54, weq61).
// ------------------------------------------------------------------------------------
template <bool HALF>
__global__ void k_init(KParams k, const StepState* __restrict__ ss, const float* __restrict__ in,
                       int have_p, Pops pops, float* __restrict__ h, float* __restrict__ hist) {
  const int N = k.N;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;  // interior node
  if (i0 >= k.nint) return;
  const StepState sa = *ss;
  const int y = i0 / k.nx, x = i0 - y * k.nx;
  const int idx = i0 + k.row0 * k.nx;                      // its stored index
  const float* phi0 = in;
  const float q = __ldg(in + N + idx);
  const float ux = __ldg(in + 2 * N + idx);
  const float uy = __ldg(in + 3 * N + idx);
  const float p = have_p ? __ldg(in + 4 * N + idx) : 0.0f;
  Stencil s = load_stencil(k, sa, phi0, x, y);
  float gx, gy, lap;
  grad_lap(s, gx, gy, lap);
  const float phi = s.c;
  // hbar without the field term (E = 0 at initialisation)
  const float mu = k.beta4 * phi * (phi - 0.5f) * (phi - 1.0f) - k.kappa * lap;
  const float rho = k.rho_v + k.drho * phi;
  const float uu = ux * ux + uy * uy;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float cu = cx(i) * ux + cy(i) * uy;
    const float si = wgt(i) * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu);
    st_pop<HALF>(k, pops, 0, i, idx, i == 0 ? phi - (1.0f - wgt(0)) * mu : wgt(i) * mu);
    st_pop<HALF>(k, pops, 1, i, idx, wgt(i) * q * (1.0f + 3.0f * cu));
    st_pop<HALF>(k, pops, 2, i, idx, (i == 0 ? (wgt(0) - 1.0f) : wgt(i)) * 3.0f * p + rho * si);
  }
  st_g0_lo<HALF>(k, pops, idx, 0.0f);
  // potential at equilibrium with the linear wall interpolation (0 when periodic); in a
  // slab, y and ny are those of the whole lattice
  float vlin = 0.0f;
  if (k.walls) vlin = sa.vw_b + (sa.vw_t - sa.vw_b) * ((y + k.y_global0 + 0.5f) / (float)k.ny_global);
#pragma unroll
  for (int i = 1; i < 9; ++i) h[(i - 1) * (size_t)N + idx] = wgt(i) * vlin;
#pragma unroll
  for (int j = 0; j < NHIST; ++j) hist[j * (size_t)N + idx] = 0.0f;
}

// Step values for step n (ramps, first-step flag) into one slot.
__global__ void k_step_set(KParams k, StepState* ss, long long n, int first) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *ss = make_step(k, n, first);
}

// ------------------------------------------------------------------------------------
// Moments of the current step (a1): phi = sum g (Eq. weq49), q = sum l + R^{n-1}/2
// (Eq. weq62 with the lagged R of Algorithm 1).  Writes phi and the per-node potential
// coefficients; FP64 sums of phi and q; the last CTA resets the potential loop.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void moments_tail(const KParams& k, const StepState* __restrict__ ss,
                                             double2* __restrict__ partials, Ctl* ctl,
                                             double tol, int min_iter, int max_iter,
                                             int fixed_iter, int bid, int nblk, float phi_acc,
                                             float q_acc, int bad);

// Block `bid` of `nblk` blocks of 256 threads over one simulation.
template <bool HALF>
__device__ __forceinline__ void moments_body(const KParams& k, const StepState* __restrict__ ss,
                                             const Pops& pops, const float* __restrict__ hist,
                                             float* __restrict__ phi_out,
                                             float2* __restrict__ aq,
                                             double2* __restrict__ partials, Ctl* ctl,
                                             double tol, int min_iter, int max_iter,
                                             int fixed_iter, int bid, int nblk) {
  const int N = k.N;
  float phi_acc = 0.0f, q_acc = 0.0f;
  int bad = 0;
  const int off = k.row0 * k.nx;  // stored index of interior node 0
  for (int i0 = bid * blockDim.x + threadIdx.x; i0 < k.nint; i0 += nblk * blockDim.x) {
    const int idx = i0 + off;
    const float phi = phi_of<HALF>(k, pops, idx);
    float q = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) q += ld_pop<HALF>(k, pops, 1, i, idx);
    q += 0.5f * __ldg(hist + 3 * (size_t)N + idx);
    phi_out[idx] = phi;
    aq[idx] = make_float2(potential_coef(k, phi), q);
    bad |= !(isfinite(phi) && isfinite(q));
    phi_acc += phi;
    q_acc += q;
  }
  moments_tail(k, ss, partials, ctl, tol, min_iter, max_iter, fixed_iter, bid, nblk, phi_acc,
               q_acc, bad);
}

// The reduction of the moments pass: FP32 within a warp, FP64 across warps and CTAs.
__device__ __forceinline__ void moments_tail(const KParams& k, const StepState* __restrict__ ss,
                                             double2* __restrict__ partials, Ctl* ctl,
                                             double tol, int min_iter, int max_iter,
                                             int fixed_iter, int bid, int nblk, float phi_acc,
                                             float q_acc, int bad) {
  // FP32 within a warp, FP64 across warps and CTAs.  Warp 0 forms the CTA's FP64 partial
  // and takes a ticket; the CTA that takes the last one reduces every CTA's partial with
  // all its threads (a fixed order: thread t adds partials t, t + 256, ..., then a fixed
  // tree), the others leave.
  __shared__ float2 s_sum[8];
  __shared__ double2 s_red[256];
  __shared__ int s_last;
  const float wp = warp_sum(phi_acc), wq = warp_sum(q_acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_sum[warp] = make_float2(wp, wq);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&ctl->nonfinite, 1);
  __syncthreads();
  if (warp == 0) {
    const int nw = (int)(blockDim.x >> 5);
    double a = 0.0, b = 0.0;
    if (lane < nw) {
      a = (double)s_sum[lane].x;
      b = (double)s_sum[lane].y;
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {  // fixed tree over the (at most 8) warps
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      partials[bid] = make_double2(a, b);
      __threadfence();
      s_last = atomicAdd(&ctl->ticket_m, 1u) == (unsigned)nblk - 1u;
    }
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double ra = 0.0, rb = 0.0;
  for (int j = threadIdx.x; j < nblk; j += blockDim.x) {
    const double2 v = __ldcg(partials + j);
    ra += v.x;
    rb += v.y;
  }
  s_red[threadIdx.x] = make_double2(ra, rb);
  __syncthreads();
  for (int o = (int)blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const double2 u = s_red[threadIdx.x + o];
      s_red[threadIdx.x].x += u.x;
      s_red[threadIdx.x].y += u.y;
    }
    __syncthreads();
  }
  const double sa = s_red[0].x, sb = s_red[0].y;
  if (threadIdx.x == 0) {
    // a non-finite phi or q (flagged by any CTA before its ticket) can never satisfy the
    // stopping rule: the solve then makes one sub-iteration and reports not converged,
    // and the call reports EHD_ERR_NONFINITE
    const bool bad_state = ld_cg(&ctl->nonfinite) != 0;
    ctl->sum_phi = sa;
    ctl->sum_q = sb;
    ctl->mean_q = (float)(sb / (double)k.nint);
    ctl->iter = 0;
    ctl->done = 0;
    ctl->converged = 0;
    ctl->rel = 0.0;
    ctl->tol = tol;
    ctl->min_iter = bad_state ? 1 : min_iter;
    ctl->max_iter = bad_state ? 1 : max_iter;
    ctl->fixed_iter = bad_state ? 0 : fixed_iter;
    ctl->vw_b = ss->vw_b;
    ctl->vw_t = ss->vw_t;
    ctl->ticket_m = 0u;
    ctl->bar_count = 0u;
    ctl->mpart_n = 0;
    __threadfence();
  }
}

// The moments pass without the cross-CTA reduction (an on-chip potential loop without a
// neutralised source needs neither the mean charge nor the sums before it runs): each CTA
// leaves its FP64 partial, the coupled pass reduces them for the statistics, and block 0
// sets the loop control.  (A non-finite flag is applied by the loop itself.)
__device__ __forceinline__ void moments_partial_only(const KParams& k,
                                                     const StepState* __restrict__ ss,
                                                     double2* __restrict__ partials, Ctl* ctl,
                                                     double tol, int min_iter, int max_iter,
                                                     int fixed_iter, int bid, int nblk,
                                                     float phi_acc, float q_acc, int bad) {
  __shared__ float2 s_sum[8];
  const float wp = warp_sum(phi_acc), wq = warp_sum(q_acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_sum[warp] = make_float2(wp, wq);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&ctl->nonfinite, 1);
  __syncthreads();
  if (warp != 0) return;
  const int nw = (int)(blockDim.x >> 5);
  double a = 0.0, b = 0.0;
  if (lane < nw) {
    a = (double)s_sum[lane].x;
    b = (double)s_sum[lane].y;
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {  // the same fixed tree as moments_tail
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) partials[bid] = make_double2(a, b);
  if (bid == 0 && lane == 0) {
    ctl->iter = 0;
    ctl->done = 0;
    ctl->converged = 0;
    ctl->rel = 0.0;
    ctl->tol = tol;
    ctl->min_iter = min_iter;
    ctl->max_iter = max_iter;
    ctl->fixed_iter = fixed_iter;
    ctl->vw_b = ss->vw_b;
    ctl->vw_t = ss->vw_t;
    ctl->ticket_m = 0u;
    ctl->bar_count = 0u;
    ctl->mpart_n = nblk;
  }
}

template <bool HALF>
__global__ void __launch_bounds__(256) k_moments(KParams k, const StepState* __restrict__ ss,
                                                 Pops pops,
                                                 const float* __restrict__ hist,
                                                 float* __restrict__ phi_out,
                                                 float2* __restrict__ aq,
                                                 double2* __restrict__ partials, Ctl* ctl,
                                                 double tol, int min_iter, int max_iter,
                                                 int fixed_iter) {
  moments_body<HALF>(k, ss, pops, hist, phi_out, aq, partials, ctl, tol, min_iter, max_iter,
                     fixed_iter, blockIdx.x, gridDim.x);
}

// The moments pass for FP32 storage with N a multiple of 4: four consecutive nodes per
// thread with 16-byte loads, so a thread has its 20 loads in flight at once (the scalar
// form's grid-stride loop waited on one node's loads before the next).  Per node the
// arithmetic is moments_body's, in the same order; only the FP32 partial sums group the
// nodes differently.
// Four consecutive FP16-stored moving populations of plane (field, i), as the FP32 values
// ld_pop<true> reads for each of them (one 8-byte load).
__device__ __forceinline__ float4 ld_pop4_half(const KParams& k, const Pops& P, int field, int i,
                                               size_t q4) {
  const uint2 raw = __ldg(reinterpret_cast<const uint2*>(P.p16 + (size_t)(field * 8 + i - 1) * k.N) + q4);
  const __half2 a = *reinterpret_cast<const __half2*>(&raw.x);
  const __half2 b = *reinterpret_cast<const __half2*>(&raw.y);
  const float s = __fmul_rn(k.ipsc[field], wgt(i));
  return make_float4(__fmul_rn(__low2float(a), s), __fmul_rn(__high2float(a), s),
                     __fmul_rn(__low2float(b), s), __fmul_rn(__high2float(b), s));
}

// Four consecutive nodes per thread (N a multiple of 4): 16-byte loads of each FP32 plane
// and 8-byte loads of each FP16 plane; per node the arithmetic of moments_body.
template <bool TAIL, bool HALF>
__device__ __forceinline__ void moments4_body(const KParams& k, const StepState* __restrict__ ss,
                                              const Pops& pops, const float* __restrict__ hist,
                                              float* __restrict__ phi_out,
                                              float2* __restrict__ aq,
                                              double2* __restrict__ partials, Ctl* ctl,
                                              double tol, int min_iter, int max_iter,
                                              int fixed_iter, int bid, int nblk) {
  const size_t N4 = (size_t)k.N / 4;
  const size_t q4 = (size_t)bid * blockDim.x + threadIdx.x;
  float phi_acc = 0.0f, q_acc = 0.0f;
  int bad = 0;
  if (q4 < N4) {
    const float4* P = reinterpret_cast<const float4*>(pops.p32) + q4;
    float4 g[9], l[9], lo;
    if (HALF) {
      // FP32 planes: the rest populations of g and l, then g0's low part in plane 3
      g[0] = __ldg(P);
      l[0] = __ldg(P + N4);
      lo = __ldg(P + 3 * N4);
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        g[i] = ld_pop4_half(k, pops, 0, i, q4);
        l[i] = ld_pop4_half(k, pops, 1, i, q4);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        g[i] = __ldg(P + i * N4);
        l[i] = __ldg(P + (9 + i) * N4);
      }
      lo = __ldg(P + NPOP * N4);
    }
    const float4 R = __ldg(reinterpret_cast<const float4*>(hist + 3 * (size_t)k.N) + q4);
    float ph[4], qq[4];
    const float* gf = reinterpret_cast<const float*>(g);
    const float* lf = reinterpret_cast<const float*>(l);
    const float lov[4] = {lo.x, lo.y, lo.z, lo.w}, Rv[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float gc[9], lc[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        gc[i] = gf[4 * i + c];
        lc[i] = lf[4 * i + c];
      }
      moments_of(gc, lov[c], lc, Rv[c], ph[c], qq[c]);
      bad |= !(isfinite(ph[c]) && isfinite(qq[c]));
      phi_acc += ph[c];
      q_acc += qq[c];
    }
    reinterpret_cast<float4*>(phi_out)[q4] = make_float4(ph[0], ph[1], ph[2], ph[3]);
    float4* a4 = reinterpret_cast<float4*>(aq) + 2 * q4;
    a4[0] = make_float4(potential_coef(k, ph[0]), qq[0], potential_coef(k, ph[1]), qq[1]);
    a4[1] = make_float4(potential_coef(k, ph[2]), qq[2], potential_coef(k, ph[3]), qq[3]);
  }
  if (TAIL)
    moments_tail(k, ss, partials, ctl, tol, min_iter, max_iter, fixed_iter, bid, nblk, phi_acc,
                 q_acc, bad);
  else
    moments_partial_only(k, ss, partials, ctl, tol, min_iter, max_iter, fixed_iter, bid, nblk,
                         phi_acc, q_acc, bad);
}
template <bool TAIL, bool HALF>
__global__ void __launch_bounds__(256) k_moments4(KParams k, const StepState* __restrict__ ss,
                                                  Pops pops, const float* __restrict__ hist,
                                                  float* __restrict__ phi_out,
                                                  float2* __restrict__ aq,
                                                  double2* __restrict__ partials, Ctl* ctl,
                                                  double tol, int min_iter, int max_iter,
                                                  int fixed_iter) {
  moments4_body<TAIL, HALF>(k, ss, pops, hist, phi_out, aq, partials, ctl, tol, min_iter,
                            max_iter, fixed_iter, blockIdx.x, gridDim.x);
}
// The k_moments4 form for a lattice: with or without the cross-CTA tail, by storage.
static inline const void* moments4_kernel(const KParams& kp, bool tail) {
  if (kp.half)
    return tail ? (const void*)k_moments4<true, true> : (const void*)k_moments4<false, true>;
  return tail ? (const void*)k_moments4<true, false> : (const void*)k_moments4<false, false>;
}
// Whether a lattice takes k_moments4 (moments4_ok, in the header), and its grid.
static inline int moments4_blocks(const KParams& kp) { return (kp.N / 4 + 255) / 256; }

// ------------------------------------------------------------------------------------
// The fused coupled pass (a1, a2, a4-a9): stencils on phi, field from the converged
// potential populations, chemical potential, forces, charge source, then collision of
// g (Eq. weq45), l (Eq. weq58) and f (Eq. weq38) and the push to the neighbours with
// half-way bounce-back; history for the next step.
// ------------------------------------------------------------------------------------
// Where the per-node kernel reads the node's post-stream populations, converged potential
// populations and lagged quantities (device memory, one node per thread).
// The populations and lagged values the pass reads are read once: they go through L2
// evict-first (ld.global.cs), and so do its stores of the hydrodynamic populations and of
// the lagged values other than R (st_pop, below), which only the next coupled pass reads;
// the converged potential populations, phi and the loop's data, and the g and l
// populations and R that the next moments pass reads, keep their place in L2.  Measured at
// 512 x 1024: a step 5 us shorter than with every access at the default policy (the
// coupled pass 26.6 against 30.2 us, the moments pass 6.4 against 8.2 us), the same bits.
template <bool HALF>
struct GlobalSrc {
  const KParams& k;
  const Pops& pin;
  const float* __restrict__ hs;
  const float* __restrict__ hist;
  int idx;
  // with FP16 storage the value ld_pop<true> reads, through the same evict-first loads
  __device__ __forceinline__ float pop(int field, int i) const {
    const size_t j = EHD_IDX(k, idx, k.N);
    if (!HALF) return __ldcs(pin.p32 + (size_t)(field * 9 + i) * k.N + j);
    if (i == 0) return __ldcs(pin.p32 + (size_t)field * k.N + j);
    const __half v = __ldcs(pin.p16 + (size_t)(field * 8 + i - 1) * k.N + j);
    return __half2float(v) * (k.ipsc[field] * wgt(i));
  }
  __device__ __forceinline__ float g0_lo() const {
    return __ldcs(pin.p32 + (size_t)(HALF ? 3 : NPOP) * k.N + EHD_IDX(k, idx, k.N));
  }
  __device__ __forceinline__ float h(int i) const {
    return __ldg(hs + i * (size_t)k.N + EHD_IDX(k, idx, k.N));
  }
  __device__ __forceinline__ float hist_in(int j) const {
    return __ldcs(hist + j * (size_t)k.N + EHD_IDX(k, idx, k.N));
  }
};

// The statistics and next-step values one thread of the pass records (the potential loop
// of this step has finished).
__device__ __forceinline__ void coupled_record(const KParams& k, StepState* ss, int cur,
                                               const StepState& sa, const Ctl* ctl,
                                               DevStats* stats) {
  // values of the next step, in the other slot (this step's slot is being read)
  ss[cur ^ 1] = make_step(k, sa.n + 1, 0);
  const int it = ld_cg(&ctl->iter);
  stats->iters_total += it;
  stats->iters_min = min(stats->iters_min, it);
  stats->iters_max = max(stats->iters_max, it);
  stats->not_converged += ld_cg(&ctl->converged) ? 0 : 1;
  stats->nonfinite |= ld_cg(&ctl->nonfinite);
  stats->last_rel = ld_cg(&ctl->rel);
  stats->sum_phi = ld_cg(&ctl->sum_phi);
  stats->sum_q = ld_cg(&ctl->sum_q);
  stats->barrier_error |= ld_cg(&ctl->bar_error);
  stats->steps += 1;
}

// The coupled pass at interior node (x, y), stored index idx: everything after the loads.
template <bool HALF, class Src>
__device__ __forceinline__ void coupled_node(const KParams& k, const StepState& sa,
                                             const Pops& pout, const float* __restrict__ phi_f,
                                             const float* __restrict__ hs,
                                             float* __restrict__ hist, const Ctl* ctl, int x,
                                             int y, int idx, const Src& src) {
  const int N = k.N;
  // a2: stencils on phi
  const Stencil st = load_stencil(k, sa, phi_f, x, y);
  float gphx, gphy, lap;
  grad_lap(st, gphx, gphy, lap);
  const float phi = st.c;

  // populations at this node (post-stream)
  float g[9], l[9], f[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    g[i] = src.pop(0, i);
    l[i] = src.pop(1, i);
    f[i] = src.pop(2, i);
  }
  float hv[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) hv[i] = src.h(i);
  const float s_prev_in = src.hist_in(0);
  const float jx_prev_in = src.hist_in(1);
  const float jy_prev_in = src.hist_in(2);
  const float R_prev = src.hist_in(3);
  const float Fx_prev = src.hist_in(4);
  const float Fy_prev = src.hist_in(5);

  // a1: moments and properties
  float lsum = 0.0f, mx = 0.0f, my = 0.0f, fsum_nr = 0.0f;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    lsum += l[i];
    mx += cx(i) * f[i];
    my += cy(i) * f[i];
    if (i) fsum_nr += f[i];
  }
  const float q = lsum + 0.5f * R_prev;
  const float rho = k.rho_v + k.drho * phi;
  const float inv_rho = 1.0f / rho;
  const float ux = (mx + 0.5f * Fx_prev) * inv_rho;
  const float uy = (my + 0.5f * Fy_prev) * inv_rho;

  // a4: E = -grad(varphi) from the converged potential populations: the local first
  // moment (Eq. eqA.16), or the stencil on varphi (variant)
  const float eh = eps_hat_of(k, phi);
  float Ex, Ey;
  if (k.field_fd) {
    const Stencil sv = load_varphi_stencil(k, hs, x, y, __ldg(&ctl->vw_b), __ldg(&ctl->vw_t));
    float gvx, gvy, lv;
    grad_lap(sv, gvx, gvy, lv);
    Ex = -gvx;
    Ey = -gvy;
  } else {
    const float m1x = hv[0] - hv[2] + hv[4] - hv[5] - hv[6] + hv[7];
    const float m1y = hv[1] - hv[3] + hv[4] + hv[5] - hv[6] - hv[7];
    const float inv_den = 1.0f / potential_den(k, phi);
    Ex = m1x * inv_den;
    Ey = m1y * inv_den;
  }
  // the field in hbar: this step's, or (variant) the previous step's, as Algorithm 1
  // lists the Cahn-Hilliard LBE before the potential solve (the same at the first step)
  float Emx = Ex, Emy = Ey;
  if (k.lagged) {
    if (!sa.first) {
      Emx = hist[6 * (size_t)N + idx];
      Emy = hist[7 * (size_t)N + idx];
    }
    hist[6 * (size_t)N + idx] = Ex;
    hist[7 * (size_t)N + idx] = Ey;
  }

  // a5: chemical potential (Eq. weq31), force (Eq. weq30), charge source (Eq. weq57)
  const float de = deps_of(k, phi);
  const float mu = k.beta4 * phi * (phi - 0.5f) * (phi - 1.0f) - k.kappa * lap -
                   0.5f * de * (Emx * Emx + Emy * Emy);
  const float Fx = mu * gphx + q * Ex + rho * k.gbx;
  const float Fy = mu * gphy + q * Ey + rho * k.gby;
  const float eps = k.eps_v + eh;
  const float sig = k.sig_v + k.dsig * phi;
  const float gE = gphx * Ex + gphy * Ey;
  const float R = (sig / eps) * (de * gE - q) - k.dsig * gE;

  // a9 inputs: advection term and charge flux; zero backward differences at the start
  const float s_adv = ux * gphx + uy * gphy;
  const float Jx = q * ux, Jy = q * uy;
  const float s_prev = sa.first ? s_adv : s_prev_in;
  const float jx_prev = sa.first ? Jx : jx_prev_in;
  const float jy_prev = sa.first ? Jy : jy_prev_in;

  // pressure (Eq. eq32): c_s^2/(1 - w0) [sum_{i!=0} f + u.grad(rho)/2 + rho s_0(u)],
  // s_0(u) = -w0 u.u / (2 c_s^2), grad rho = drho grad phi
  const float uu = ux * ux + uy * uy;
  const float p = 0.6f * (fsum_nr + 0.5f * k.drho * s_adv - (2.0f / 3.0f) * rho * uu);

  // relaxation rates
  const float mu_dyn = k.mu_v + k.dmu * phi;
  const float tau_f = 0.5f + 3.0f * mu_dyn * inv_rho;
  const float om_f = 1.0f / tau_f;
  const float pref_f = 1.0f - 0.5f * om_f;
  const float om_g = k.omega_g, om_l = k.omega_l, pref_l = k.pref_l;

  // CH source: G_i + (G_i - G_i^{n-1})/2 = w_i k_i (3 s - s_prev)/2
  const float gsrc = 1.5f * s_adv - 0.5f * s_prev;
  const float djx = 3.0f * (Jx - jx_prev), djy = 3.0f * (Jy - jy_prev);
  const float grx = k.drho * gphx, gry = k.drho * gphy;

  // The rest population g_0 carries phi, O(1), while a step near a steady state changes
  // it by far less than its FP32 spacing; it is kept as hi + lo, and its change is the
  // collision's phi balance: sum_i g_i* = sum_i g_i - (3 s - s_prev)/2 (sum_i g_eq_i =
  // phi, sum_i w_i k_i = -1), so g_0* - g_0 = sum_{i>0} (g_i - g_i*) - (3 s - s_prev)/2,
  // the value that relaxing g_0 by Eq. weq45 gives in exact arithmetic, added to hi + lo
  // without rounding error.  The moving populations enter as stored (with FP16 storage,
  // rounded), so phi's total over the lattice changes by the source alone.
  // Per-node coefficients of the three collisions by lattice-weight class (axis, diagonal,
  // rest), so that a direction costs a few fused multiply-adds:
  //   g_i* = g_i + om_g (w_i mu - g_i) + w_i k_i gsrc                     (Eq. weq45)
  //   l_i* = l_i + om_l (l_eq_i - l_i) + pref_l w_i (R + c_i.dJ),
  //          l_eq_i = w_i q + 3 w_i q (c_i.u)                               (Eqs. weq58-61)
  //   f_i* = f_i + om_f (f_eq_i - f_i) + 3 pref_f w_i (c_i.F + (c_i.u)(c_i.grad rho)),
  //          f_eq_i = 3 w_i p + rho w_i ((c_i.u)(3 + 4.5 c_i.u) - 1.5 u.u),  (Eqs. weq38-40)
  //          with w_0 - 1 in place of w_0 in the pressure term of f_eq_0
  const float wa = wgt(1), wd = wgt(5), w0 = wgt(0);
  const float wmu_a = __fmul_rn(wa, mu), wmu_d = __fmul_rn(wd, mu);
  const float wks_a = __fmul_rn(wa * ch_k(1), gsrc), wks_d = __fmul_rn(wd * ch_k(5), gsrc);
  const float wq_a = __fmul_rn(wa, q), wq_d = __fmul_rn(wd, q), wq_0 = __fmul_rn(w0, q);
  const float wq3_a = __fmul_rn(3.0f, wq_a), wq3_d = __fmul_rn(3.0f, wq_d);
  const float plw_a = __fmul_rn(pref_l, wa), plw_d = __fmul_rn(pref_l, wd);
  const float plwR_a = __fmul_rn(plw_a, R), plwR_d = __fmul_rn(plw_d, R);
  const float plwR_0 = __fmul_rn(__fmul_rn(pref_l, w0), R);
  const float p3 = __fmul_rn(3.0f, p);
  const float w3p_a = __fmul_rn(wa, p3), w3p_d = __fmul_rn(wd, p3), w3p_0 = __fmul_rn(w0 - 1.0f, p3);
  const float rw_a = __fmul_rn(rho, wa), rw_d = __fmul_rn(rho, wd), rw_0 = __fmul_rn(rho, w0);
  const float pf3 = __fmul_rn(3.0f, pref_f);
  const float pf3w_a = __fmul_rn(pf3, wa), pf3w_d = __fmul_rn(pf3, wd);
  const float m15uu = __fmul_rn(-1.5f, uu);
  // c_i.v for the diagonal directions: v_x + v_y and v_x - v_y
  const float upp = __fadd_rn(ux, uy), upm = __fsub_rn(ux, uy);
  const float jpp = __fadd_rn(djx, djy), jpm = __fsub_rn(djx, djy);
  const float Fpp = __fadd_rn(Fx, Fy), Fpm = __fsub_rn(Fx, Fy);
  const float gpp = __fadd_rn(grx, gry), gpm = __fsub_rn(grx, gry);

  // The rest population g_0 carries phi, O(1), while a step near a steady state changes
  // it by far less than its FP32 spacing; it is kept as hi + lo, and its change is the
  // collision's phi balance: sum_i g_i* = sum_i g_i - (3 s - s_prev)/2 (sum_i g_eq_i =
  // phi, sum_i w_i k_i = -1), so g_0* - g_0 = sum_{i>0} (g_i - g_i*) - (3 s - s_prev)/2,
  // the value that relaxing g_0 by Eq. weq45 gives in exact arithmetic, added to hi + lo
  // without rounding error.  The moving populations enter as stored (with FP16 storage,
  // rounded), so phi's total over the lattice changes by the source alone.
  float gpre = 0.0f, gmov = 0.0f;
  const bool inner = x > 0 && x + 1 < k.nx && y > 0 && y + 1 < k.ny;
#pragma unroll
  for (int i0 = 1; i0 < 10; ++i0) {
    const int i = i0 == 9 ? 0 : i0;  // the moving populations first, the rest one last
    const bool axis = i >= 1 && i <= 4;
    // c_i.v of the direction (compile-time signs)
    auto dot = [&](float vx, float vy, float vpp, float vpm) {
      if (i == 0) return 0.0f;
      if (axis) return cx(i) != 0 ? (cx(i) > 0 ? vx : -vx) : (cy(i) > 0 ? vy : -vy);
      if (cx(i) == cy(i)) return cx(i) > 0 ? vpp : -vpp;
      return cx(i) > 0 ? vpm : -vpm;
    };
    const float cu = dot(ux, uy, upp, upm);
    // away from every edge a population lands at a fixed offset; at an edge the wrap, wall
    // or cut rule of push_target applies
    int dir = i;
    const int t = inner ? idx + cx(i) + cy(i) * k.nx : push_target(k, x, y, i, dir);
    // a6: Cahn-Hilliard, g_eq of Eq. weq46
    if (i != 0) {
      const float gn = __fadd_rn(__fmaf_rn(om_g, __fsub_rn(axis ? wmu_a : wmu_d, g[i]), g[i]),
                                 axis ? wks_a : wks_d);
      gpre = __fadd_rn(gpre, g[i]);
      gmov = __fadd_rn(gmov, st_pop_read<HALF>(k, pout, 0, dir, t, gn));
    } else {
      float hi = g[0], lo = src.g0_lo();
      two_float_add(hi, lo, __fsub_rn(__fsub_rn(gpre, gmov), gsrc));
      st_pop<HALF>(k, pout, 0, 0, t, hi);
      st_g0_lo<HALF>(k, pout, t, lo);
    }
    // a7: Nernst-Planck, l_eq of Eq. weq61, S_i + T_i of Eqs. weq59, weq60
    const float leq = i == 0 ? wq_0 : __fmaf_rn(axis ? wq3_a : wq3_d, cu, axis ? wq_a : wq_d);
    const float lsrc = i == 0 ? plwR_0
                              : __fmaf_rn(axis ? plw_a : plw_d, dot(djx, djy, jpp, jpm),
                                          axis ? plwR_a : plwR_d);
    const float ln = __fadd_rn(__fmaf_rn(om_l, __fsub_rn(leq, l[i]), l[i]), lsrc);
    // a8: hydrodynamics, f_eq of Eq. weq40, forcing of Eq. weq39 written as
    // w_i [c_i.F + (c_i.u)(c_i.grad rho)] / c_s^2 (the u.grad rho terms cancel)
    const float core = i == 0 ? m15uu : __fmaf_rn(cu, __fmaf_rn(4.5f, cu, 3.0f), m15uu);
    const float feq = __fmaf_rn(i == 0 ? rw_0 : (axis ? rw_a : rw_d), core,
                                i == 0 ? w3p_0 : (axis ? w3p_a : w3p_d));
    float fn = __fmaf_rn(om_f, __fsub_rn(feq, f[i]), f[i]);
    if (i != 0)
      fn = __fmaf_rn(axis ? pf3w_a : pf3w_d,
                     __fmaf_rn(cu, dot(grx, gry, gpp, gpm), dot(Fx, Fy, Fpp, Fpm)), fn);
    st_pop<HALF>(k, pout, 1, dir, t, ln);
    st_pop<HALF>(k, pout, 2, dir, t, fn);
  }
  idx = (int)EHD_IDX(k, idx, k.N);
  __stcs(hist + idx, s_adv);
  __stcs(hist + (size_t)N + idx, Jx);
  __stcs(hist + 2 * (size_t)N + idx, Jy);
  hist[3 * (size_t)N + idx] = R;  // read by the next moments pass
  __stcs(hist + 4 * (size_t)N + idx, Fx);
  __stcs(hist + 5 * (size_t)N + idx, Fy);
}

// The FP64 sums of phi and q of this step's moments pass from its np per-CTA partials (the
// whole block, a fixed order: thread t adds partials t, t + blockDim, ..., then a fixed
// tree), for the statistics and the loop control.
__device__ __forceinline__ void coupled_reduce_moments(const KParams& k,
                                                       const double2* __restrict__ partials,
                                                       int np, Ctl* ctl) {
  __shared__ double2 s_red[128];
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < np; j += blockDim.x) {
    const double2 v = __ldcg(partials + j);
    a += v.x;
    b += v.y;
  }
  s_red[threadIdx.x] = make_double2(a, b);
  __syncthreads();
  for (int o = (int)blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const double2 u = s_red[threadIdx.x + o];
      s_red[threadIdx.x].x += u.x;
      s_red[threadIdx.x].y += u.y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ctl->sum_phi = s_red[0].x;
    ctl->sum_q = s_red[0].y;
    ctl->mean_q = (float)(s_red[0].y / (double)k.nint);
    ctl->mpart_n = 0;
  }
  __syncthreads();
}

// Block `bid` of blocks of 128 threads over one simulation, one node per thread, loads
// straight from device memory.
template <bool HALF>
__device__ __forceinline__ void coupled_body(const KParams& k, StepState* ss, int cur,
                                             const Pops& pin, const Pops& pout,
                                             const float* __restrict__ phi_f,
                                             const float* __restrict__ hbuf,
                                             float* __restrict__ hist, Ctl* ctl,
                                             const double2* __restrict__ partials,
                                             DevStats* stats, int bid) {
  // the control words and this step's state are read by every thread and written by no
  // CTA of the pass (it writes the other state slot): the read-only path, one request
  // per SM
  const int parity = __ldg(&ctl->parity);
  StepState sa;
  {
    const StepState* p = ss + cur;
    sa.n = __ldg(&p->n);
    sa.first = __ldg(&p->first);
    sa.pad = 0;
    sa.cos_b = __ldg(&p->cos_b);
    sa.cos_t = __ldg(&p->cos_t);
    sa.vw_b = __ldg(&p->vw_b);
    sa.vw_t = __ldg(&p->vw_t);
  }
  if (bid == 0) {
    const int np = ld_cg(&ctl->mpart_n);
    if (np > 0) coupled_reduce_moments(k, partials, np, ctl);
    if (threadIdx.x == 0) coupled_record(k, ss, cur, sa, ctl, stats);
  }
  const int i0 = bid * blockDim.x + threadIdx.x;  // interior node
  if (i0 >= k.nint) return;
  const int y = i0 / k.nx, x = i0 - y * k.nx;
  const int idx = i0 + k.row0 * k.nx;              // its stored index
  const float* hs = hbuf + (size_t)parity * NH * k.N;
  const GlobalSrc<HALF> src{k, pin, hs, hist, idx};
  coupled_node<HALF>(k, sa, pout, phi_f, hs, hist, ctl, x, y, idx, src);
}

// 128 threads.  The FP32 form (specialised below): at least 7 CTAs per SM (at most
// 72 registers); the pass is bound by memory latency, and 7 resident CTAs run it 2.5 %
// faster than the 6 that 80 registers allow (8 CTAs at 64 registers spill more and run
// slower).  The FP16-storage form: at least 6 CTAs per SM (80 registers, no spills),
// 1.6 us faster at 512 x 1024 than the 5 its 96 registers allowed; 7 and 8 spill.
template <bool HALF>
__global__ void __launch_bounds__(128) k_coupled(KParams k, StepState* ss, int cur, Pops pin,
                                                 Pops pout,
                                                 const float* __restrict__ phi_f,
                                                 const float* __restrict__ hbuf,
                                                 float* __restrict__ hist, Ctl* ctl,
                                                 const double2* __restrict__ partials,
                                                 DevStats* stats) {
  coupled_body<HALF>(k, ss, cur, pin, pout, phi_f, hbuf, hist, ctl, partials, stats, blockIdx.x);
}
#ifndef EHD_COUPLED_MIN_CTAS
#define EHD_COUPLED_MIN_CTAS 7
#endif
template <>
__global__ void __launch_bounds__(128, EHD_COUPLED_MIN_CTAS) k_coupled<false>(KParams k, StepState* ss, int cur,
                                                           Pops pin, Pops pout,
                                                           const float* __restrict__ phi_f,
                                                           const float* __restrict__ hbuf,
                                                           float* __restrict__ hist,
                                                           Ctl* ctl,
                                                           const double2* __restrict__ partials,
                                                           DevStats* stats) {
  coupled_body<false>(k, ss, cur, pin, pout, phi_f, hbuf, hist, ctl, partials, stats, blockIdx.x);
}
#ifndef EHD_COUPLED16_MIN_CTAS
#define EHD_COUPLED16_MIN_CTAS 6
#endif
template <>
__global__ void __launch_bounds__(128, EHD_COUPLED16_MIN_CTAS) k_coupled<true>(KParams k, StepState* ss, int cur,
                                                            Pops pin, Pops pout,
                                                            const float* __restrict__ phi_f,
                                                            const float* __restrict__ hbuf,
                                                            float* __restrict__ hist,
                                                            Ctl* ctl,
                                                            const double2* __restrict__ partials,
                                                            DevStats* stats) {
  coupled_body<true>(k, ss, cur, pin, pout, phi_f, hbuf, hist, ctl, partials, stats, blockIdx.x);
}

// ------------------------------------------------------------------------------------
// Batched forms: one launch over the blocks of several simulations.  work[b] = (slot,
// block of that slot); every simulation gets exactly the blocks and arithmetic of its own
// launch, so its results do not depend on the others.
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_moments_batch(const StepSlot* __restrict__ slots,
                                                       const int2* __restrict__ work, int cur) {
  const int2 w = work[blockIdx.x];
  const StepSlot& S = slots[w.x];
  const Pops P = pops_copy(S.k, S.b, cur);
  if (S.quad && S.k.half)  // the blocks and arithmetic of the slot's own k_moments4 launch
    moments4_body<true, true>(S.k, S.b.ss + cur, P, S.b.hist, S.b.phi, S.b.aq, S.b.partials,
                              S.b.ctl, S.tol, S.min_iter, S.max_iter, S.fixed_iter, w.y,
                              S.mblocks);
  else if (S.quad)
    moments4_body<true, false>(S.k, S.b.ss + cur, P, S.b.hist, S.b.phi, S.b.aq, S.b.partials,
                               S.b.ctl, S.tol, S.min_iter, S.max_iter, S.fixed_iter, w.y,
                               S.mblocks);
  else if (S.k.half)
    moments_body<true>(S.k, S.b.ss + cur, P, S.b.hist, S.b.phi, S.b.aq, S.b.partials, S.b.ctl,
                       S.tol, S.min_iter, S.max_iter, S.fixed_iter, w.y, S.mblocks);
  else
    moments_body<false>(S.k, S.b.ss + cur, P, S.b.hist, S.b.phi, S.b.aq, S.b.partials, S.b.ctl,
                        S.tol, S.min_iter, S.max_iter, S.fixed_iter, w.y, S.mblocks);
}

// One form per storage precision, each over the work items of its slots: the FP32 form
// has the register budget of the single-simulation FP32 pass (7 CTAs per SM), which a
// kernel holding both forms could not have.
template <bool HALF>
__global__ void __launch_bounds__(128, HALF ? 1 : EHD_COUPLED_MIN_CTAS)
    k_coupled_batch(const StepSlot* __restrict__ slots, const int2* __restrict__ work,
                    int cur) {
  const int2 w = work[blockIdx.x];
  const StepSlot& S = slots[w.x];
  const Pops Pi = pops_copy(S.k, S.b, cur), Po = pops_copy(S.k, S.b, cur ^ 1);
  coupled_body<HALF>(S.k, S.b.ss, cur, Pi, Po, S.b.phi, S.b.h, S.b.hist, S.b.ctl, S.b.partials,
                     S.b.stats, w.y);
}

// Diagnostics: puts the grid barrier's arrival count half the counter range behind every
// target, so the next on-chip solve's waits run out (bounded) instead of completing.
__global__ void k_expire_barrier(Ctl* ctl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ctl->bar_count = 0x80000000u;
}

__global__ void k_stats_reset(DevStats* s) {
  s->iters_total = 0;
  s->iters_min = 0x7fffffff;
  s->iters_max = 0;
  s->not_converged = 0;
  s->nonfinite = 0;
  s->steps = 0;
  s->barrier_error = 0;
  s->last_rel = 0.0;
  s->sum_phi = 0.0;
  s->sum_q = 0.0;
}

// ------------------------------------------------------------------------------------
// Output fields.  k_phi_now: phi of the current populations; k_fields: the requested
// fields (order of the mask bits) into io[slot][N].
// ------------------------------------------------------------------------------------
// The contact line of a drop sitting on the bottom wall (the contact-radius histories of
// Sec. 7.2, Fig. 11): on each of the first two lattice rows, the nodes with phi >= level
// (current populations, phi as every pass forms it) span [a, b]; the crossings are placed
// by linear interpolation with the outside neighbours, a - (phi_a - level) / (phi_a -
// phi_{a-1}) and b + (phi_b - level) / (phi_b - phi_{b+1}), and each is extrapolated
// linearly from rows 0 and 1 to the wall at y = -1/2.  One CTA; out[0] = (left, right),
// out[1] = (radius = (right - left) / 2, 1), or NaNs and 0 when a row has no such node or
// the span reaches an end of the row (a drop across the periodic seam).
template <bool HALF>
__global__ void __launch_bounds__(256) k_contact_line(KParams k, Pops pops, float level,
                                                      double2* __restrict__ out) {
  __shared__ int s_lo[2], s_hi[2];
  if (threadIdx.x < 2) {
    s_lo[threadIdx.x] = 0x7fffffff;
    s_hi[threadIdx.x] = -1;
  }
  __syncthreads();
  for (int r = 0; r < 2; ++r)
    for (int x = threadIdx.x; x < k.nx; x += blockDim.x)
      if (phi_of<HALF>(k, pops, (size_t)r * k.nx + x) >= level) {
        atomicMin(&s_lo[r], x);
        atomicMax(&s_hi[r], x);
      }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  double left[2], right[2];
  bool ok = true;
  for (int r = 0; r < 2 && ok; ++r) {
    const int a = s_lo[r], b = s_hi[r];
    if (b < 0 || a == 0 || b == k.nx - 1) {
      ok = false;
      break;
    }
    const size_t row = (size_t)r * k.nx;
    const double pa = phi_of<HALF>(k, pops, row + a), pam = phi_of<HALF>(k, pops, row + a - 1);
    const double pb = phi_of<HALF>(k, pops, row + b), pbp = phi_of<HALF>(k, pops, row + b + 1);
    left[r] = (double)a - (pa - (double)level) / (pa - pam);
    right[r] = (double)b + (pb - (double)level) / (pb - pbp);
  }
  if (!ok) {
    out[0] = make_double2(nan, nan);
    out[1] = make_double2(nan, 0.0);
    return;
  }
  const double l = left[0] + 0.5 * (left[0] - left[1]);
  const double rr = right[0] + 0.5 * (right[0] - right[1]);
  out[0] = make_double2(l, rr);
  out[1] = make_double2(0.5 * (rr - l), 1.0);
}

cudaError_t launch_contact_line(const KParams& kp, const Buffers& b, int cur, float level,
                                cudaStream_t st) {
  const Pops P = pops_copy(kp, b, cur);
  if (kp.half)
    k_contact_line<true><<<1, 256, 0, st>>>(kp, P, level, b.partials);
  else
    k_contact_line<false><<<1, 256, 0, st>>>(kp, P, level, b.partials);
  return cudaGetLastError();
}

template <bool HALF>
__global__ void k_phi_now(KParams k, Pops pops, float* __restrict__ out) {
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (i0 >= k.nint) return;
  const int idx = i0 + k.row0 * k.nx;
  out[idx] = phi_of<HALF>(k, pops, idx);
}

template <bool HALF>
__global__ void k_fields(KParams k, const StepState* __restrict__ ss, Pops pops,
                         const float* __restrict__ phi_now, const float* __restrict__ phi_solve,
                         const float* __restrict__ hbuf, const float* __restrict__ hist,
                         const Ctl* ctl, unsigned mask, float* __restrict__ io) {
  const int N = k.N;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (i0 >= k.nint) return;
  const int y = i0 / k.nx, x = i0 - y * k.nx;
  const int idx = i0 + k.row0 * k.nx;
  const int parity = __ldg(&ctl->parity);  // not written in this pass: one request per SM
  const float* hs = hbuf + (size_t)parity * NH * N;
  const StepState sa = *ss;
  const Stencil st = load_stencil(k, sa, phi_now, x, y);
  float gphx, gphy, lap;
  grad_lap(st, gphx, gphy, lap);
  const float phi = st.c;
  float lsum = 0.0f, mx = 0.0f, my = 0.0f, fsum_nr = 0.0f;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float fi = ld_pop<HALF>(k, pops, 2, i, idx);
    lsum += ld_pop<HALF>(k, pops, 1, i, idx);
    mx += cx(i) * fi;
    my += cy(i) * fi;
    if (i) fsum_nr += fi;
  }
  const float q = lsum + 0.5f * hist[3 * (size_t)N + idx];
  const float rho = k.rho_v + k.drho * phi;
  const float ux = (mx + 0.5f * hist[4 * (size_t)N + idx]) / rho;
  const float uy = (my + 0.5f * hist[5 * (size_t)N + idx]) / rho;
  const float uu = ux * ux + uy * uy;
  const float p = 0.6f * (fsum_nr + 0.5f * k.drho * (ux * gphx + uy * gphy) -
                          (2.0f / 3.0f) * rho * uu);
  float hv[8];
  float hsum = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    hv[i] = __ldg(hs + i * (size_t)N + idx);
    hsum += hv[i];
  }
  const float varphi = hsum * (9.0f / 5.0f);
  float Ex, Ey;
  if (k.field_fd) {
    const Stencil sv = load_varphi_stencil(k, hs, x, y, __ldg(&ctl->vw_b), __ldg(&ctl->vw_t));
    float gvx, gvy, lv;
    grad_lap(sv, gvx, gvy, lv);
    Ex = -gvx;
    Ey = -gvy;
  } else {
    const float m1x = hv[0] - hv[2] + hv[4] - hv[5] - hv[6] + hv[7];
    const float m1y = hv[1] - hv[3] + hv[4] + hv[5] - hv[6] - hv[7];
    const float inv_den = 1.0f / potential_den(k, __ldg(phi_solve + idx));
    Ex = m1x * inv_den;
    Ey = m1y * inv_den;
  }
  // chemical potential (Eq. weq31) of the current phi with the last solve's field
  const float mu = k.beta4 * phi * (phi - 0.5f) * (phi - 1.0f) - k.kappa * lap -
                   0.5f * deps_of(k, phi) * (Ex * Ex + Ey * Ey);
  const float vals[NIO] = {phi, q, varphi, Ex, Ey, ux, uy, p, mu};
  int slot = 0;
#pragma unroll
  for (int b = 0; b < NIO; ++b) {
    if (mask & (1u << b)) {
      io[slot * (size_t)N + idx] = vals[b];
      ++slot;
    }
  }
}

// ------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------
static inline int blocks_for(int n, int t) { return (n + t - 1) / t; }

cudaError_t launch_step_set(const KParams& kp, const Buffers& b, int slot, long long n,
                            int first, cudaStream_t st) {
  k_step_set<<<1, 32, 0, st>>>(kp, b.ss + slot, n, first);
  return cudaGetLastError();
}

cudaError_t launch_init(const KParams& kp, const Buffers& b, int cur, bool have_p,
                        cudaStream_t st) {
  const Pops P = pops_copy(kp, b, cur);
  if (kp.half)
    k_init<true><<<blocks_for(kp.nint, 256), 256, 0, st>>>(kp, b.ss + cur, b.io, have_p ? 1 : 0, P,
                                                       b.h, b.hist);
  else
    k_init<false><<<blocks_for(kp.nint, 256), 256, 0, st>>>(kp, b.ss + cur, b.io, have_p ? 1 : 0,
                                                        P, b.h, b.hist);
  return cudaGetLastError();
}

cudaError_t launch_moments(const KParams& kp, const Buffers& b, int cur, double tol,
                           int min_iter, int max_iter, int fixed_iter, cudaStream_t st,
                           bool sums_in_coupled) {
  const int nb = moments_blocks(kp.nint);
  const Pops P = pops_copy(kp, b, cur);
  if (moments4_ok(kp)) {
    const bool tail = !(sums_in_coupled && !kp.neutralize);
    KParams k = kp;
    const StepState* ss = b.ss + cur;
    Pops pops = P;
    const float* hist = b.hist;
    float* phi = b.phi;
    float2* aq = b.aq;
    double2* partials = b.partials;
    Ctl* ctl = b.ctl;
    void* args[] = {&k, &ss, &pops, &hist, &phi, &aq, &partials, &ctl, &tol, &min_iter,
                    &max_iter, &fixed_iter};
    return cudaLaunchKernel(moments4_kernel(kp, tail), dim3(moments4_blocks(kp)), dim3(256), args,
                            0, st);
  }
  if (kp.half)
    k_moments<true><<<nb, 256, 0, st>>>(kp, b.ss + cur, P, b.hist, b.phi, b.aq, b.partials,
                                        b.ctl, tol, min_iter, max_iter, fixed_iter);
  else
    k_moments<false><<<nb, 256, 0, st>>>(kp, b.ss + cur, P, b.hist, b.phi, b.aq, b.partials,
                                         b.ctl, tol, min_iter, max_iter, fixed_iter);
  return cudaGetLastError();
}

cudaError_t launch_coupled(const KParams& kp, const Buffers& b, int cur, cudaStream_t st) {
  const Pops Pi = pops_copy(kp, b, cur), Po = pops_copy(kp, b, cur ^ 1);
  if (kp.half)
    k_coupled<true><<<blocks_for(kp.nint, 128), 128, 0, st>>>(kp, b.ss, cur, Pi, Po, b.phi, b.h,
                                                           b.hist, b.ctl, b.partials, b.stats);
  else
    k_coupled<false><<<blocks_for(kp.nint, 128), 128, 0, st>>>(kp, b.ss, cur, Pi, Po, b.phi, b.h,
                                                            b.hist, b.ctl, b.partials, b.stats);
  return cudaGetLastError();
}

cudaError_t launch_expire_barrier(const Buffers& b, cudaStream_t st) {
  k_expire_barrier<<<1, 32, 0, st>>>(b.ctl);
  return cudaGetLastError();
}

cudaError_t launch_stats_reset(const Buffers& b, cudaStream_t st) {
  k_stats_reset<<<1, 1, 0, st>>>(b.stats);
  return cudaGetLastError();
}

cudaError_t launch_fields(const KParams& kp, const Buffers& b, int cur, unsigned mask,
                          cudaStream_t st) {
  const Pops P = pops_copy(kp, b, cur);
  if (kp.half) {
    k_phi_now<true><<<blocks_for(kp.nint, 256), 256, 0, st>>>(kp, P, b.tmp);
    k_fields<true><<<blocks_for(kp.nint, 256), 256, 0, st>>>(kp, b.ss + cur, P, b.tmp, b.phi, b.h,
                                                          b.hist, b.ctl, mask, b.io);
  } else {
    k_phi_now<false><<<blocks_for(kp.nint, 256), 256, 0, st>>>(kp, P, b.tmp);
    k_fields<false><<<blocks_for(kp.nint, 256), 256, 0, st>>>(kp, b.ss + cur, P, b.tmp, b.phi,
                                                           b.h, b.hist, b.ctl, mask, b.io);
  }
  return cudaGetLastError();
}

// The two halves of launch_fields, for slabs (whose phi ghost rows are exchanged in
// between): phi of the current populations into tmp, then the requested fields into io.
cudaError_t launch_phi_now(const KParams& kp, const Buffers& b, int cur, cudaStream_t st) {
  const Pops P = pops_copy(kp, b, cur);
  if (kp.half)
    k_phi_now<true><<<blocks_for(kp.nint, 256), 256, 0, st>>>(kp, P, b.tmp);
  else
    k_phi_now<false><<<blocks_for(kp.nint, 256), 256, 0, st>>>(kp, P, b.tmp);
  return cudaGetLastError();
}
cudaError_t launch_fields_from_phi(const KParams& kp, const Buffers& b, int cur, unsigned mask,
                                   cudaStream_t st) {
  const Pops P = pops_copy(kp, b, cur);
  if (kp.half)
    k_fields<true><<<blocks_for(kp.nint, 256), 256, 0, st>>>(kp, b.ss + cur, P, b.tmp, b.phi, b.h,
                                                             b.hist, b.ctl, mask, b.io);
  else
    k_fields<false><<<blocks_for(kp.nint, 256), 256, 0, st>>>(kp, b.ss + cur, P, b.tmp, b.phi,
                                                              b.h, b.hist, b.ctl, mask, b.io);
  return cudaGetLastError();
}

// Graph nodes (the argument values are copied by cudaGraphAddKernelNode).
cudaError_t add_moments_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                             cudaGraphNode_t* out, const KParams& kp, const Buffers& b, int cur,
                             double tol, int min_iter, int max_iter, int fixed_iter,
                             bool sums_in_coupled) {
  KParams k = kp;
  const StepState* ss = b.ss + cur;
  Pops pops = pops_copy(kp, b, cur);
  const float* hist = b.hist;
  float* phi = b.phi;
  float2* aq = b.aq;
  double2* partials = b.partials;
  Ctl* ctl = b.ctl;
  void* args[] = {&k, &ss, &pops, &hist, &phi, &aq, &partials, &ctl, &tol, &min_iter, &max_iter,
                  &fixed_iter};
  cudaKernelNodeParams p = {};
  p.func = moments4_ok(kp)
               ? const_cast<void*>(moments4_kernel(kp, !(sums_in_coupled && !kp.neutralize)))
               : (kp.half ? (void*)k_moments<true> : (void*)k_moments<false>);
  p.gridDim = dim3(moments4_ok(kp) ? moments4_blocks(kp) : moments_blocks(kp.nint));
  p.blockDim = dim3(256);
  p.kernelParams = args;
  return cudaGraphAddKernelNode(out, g, deps, nd, &p);
}

cudaError_t add_coupled_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                             cudaGraphNode_t* out, const KParams& kp, const Buffers& b, int cur) {
  KParams k = kp;
  StepState* ss = b.ss;
  Pops pin = pops_copy(kp, b, cur);
  Pops pout = pops_copy(kp, b, cur ^ 1);
  const float* phi = b.phi;
  const float* h = b.h;
  float* hist = b.hist;
  Ctl* ctl = b.ctl;
  const double2* partials = b.partials;
  DevStats* stats = b.stats;
  void* args[] = {&k, &ss, &cur, &pin, &pout, &phi, &h, &hist, &ctl, &partials, &stats};
  cudaKernelNodeParams p = {};
  p.func = kp.half ? (void*)k_coupled<true> : (void*)k_coupled<false>;
  p.gridDim = dim3(blocks_for(kp.nint, 128));
  p.blockDim = dim3(128);
  p.kernelParams = args;
  return cudaGraphAddKernelNode(out, g, deps, nd, &p);
}

static cudaError_t add_batch_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                                  cudaGraphNode_t* out, void* func, int threads,
                                  const StepSlot* slots, const int2* work, int nwork, int cur) {
  void* args[] = {&slots, &work, &cur};
  cudaKernelNodeParams p = {};
  p.func = func;
  p.gridDim = dim3(nwork);
  p.blockDim = dim3(threads);
  p.kernelParams = args;
  return cudaGraphAddKernelNode(out, g, deps, nd, &p);
}

cudaError_t add_moments_batch_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                                   cudaGraphNode_t* out, const StepSlot* slots, const int2* work,
                                   int nwork, int cur) {
  return add_batch_node(g, deps, nd, out, (void*)k_moments_batch, 256, slots, work, nwork, cur);
}

cudaError_t add_coupled_batch_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                                   cudaGraphNode_t* out, const StepSlot* slots, const int2* work,
                                   int nwork, int cur, bool half) {
  return add_batch_node(g, deps, nd, out,
                        half ? (void*)k_coupled_batch<true> : (void*)k_coupled_batch<false>, 128,
                        slots, work, nwork, cur);
}

cudaError_t add_poisson_node(cudaGraph_t g, cudaGraphNode_t* out, const KParams& kp,
                             const Buffers& b, cudaGraphConditionalHandle cond);

cudaError_t build_step_graph(const KParams& kp, const Buffers& b, int cur, double tol,
                             int min_iter, int max_iter, int fixed_iter, const ResidentGeom* rg,
                             int rthreads, size_t rsmem, cudaGraph_t* out,
                             const cudaEvent_t* ev, int nsteps) {
  if (nsteps < 1 || (ev && nsteps != 1)) return cudaErrorInvalidValue;
  cudaGraph_t g;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  // the nodes in order, each depending on the previous one; with events, a record node
  // before the moments pass and after each of the three parts of the step
  cudaGraphNode_t last = nullptr;
  bool have = false;
  auto record = [&](int j) -> cudaError_t {
    if (!ev) return cudaSuccess;
    cudaGraphNode_t n;
    const cudaError_t r = cudaGraphAddEventRecordNode(&n, g, have ? &last : nullptr, have ? 1 : 0,
                                                      ev[j]);
    if (r == cudaSuccess) {
      last = n;
      have = true;
    }
    return r;
  };
  auto done = [&](cudaError_t r) {
    if (r != cudaSuccess) {
      cudaGraphDestroy(g);
      return r;
    }
    *out = g;
    return cudaSuccess;
  };
  for (int j = 0; j < nsteps; ++j) {
    const int c = (cur + j) & 1;
    cudaGraphNode_t mn, wn, pn, cn;
    if ((e = record(0)) != cudaSuccess ||
        (e = add_moments_node(g, have ? &last : nullptr, have ? 1 : 0, &mn, kp, b, c, tol,
                              min_iter, max_iter, fixed_iter, rg != nullptr)) != cudaSuccess)
      return done(e);
    last = mn;
    have = true;
    if ((e = record(1)) != cudaSuccess) return done(e);
    if (rg) {
      if ((e = add_poisson_resident_node(g, &last, 1, &pn, kp, *rg, rthreads, rsmem, b)) !=
          cudaSuccess)
        return done(e);
      last = pn;
    } else {
      // each step's WHILE node has its own handle, reset to 1 at every launch of the graph
      cudaGraphConditionalHandle h;
      if ((e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) !=
          cudaSuccess)
        return done(e);
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      if ((e = cudaGraphAddNode(&wn, g, &last, nullptr, 1, &cp)) != cudaSuccess ||
          (e = add_poisson_node(cp.conditional.phGraph_out[0], &pn, kp, b, h)) != cudaSuccess)
        return done(e);
      last = wn;
    }
    if ((e = record(2)) != cudaSuccess ||
        (e = add_coupled_node(g, &last, 1, &cn, kp, b, c)) != cudaSuccess)
      return done(e);
    last = cn;
    if ((e = record(3)) != cudaSuccess) return done(e);
  }
  return done(cudaSuccess);
}

}  // namespace ehd
