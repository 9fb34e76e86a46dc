// Internal definitions shared by the CUDA kernels and the host side of the library.
//
// Lattice: D2Q9 (Sec. 3, Eq. weq37).  Direction i = 0 rest; 1..4 axis directions
// (1,0), (0,1), (-1,0), (0,-1); 5..8 diagonals (1,1), (-1,1), (-1,-1), (1,-1).
// Weights 4/9, 1/9, 1/36; c_s^2 = 1/3.
//
// Device layout of one simulation (N = nx * ny nodes, x fastest):
//   pops[2][28][N]  post-stream populations g (0..8), l (9..17), f (18..26) and the low
//                   part of g_0 (27), two copies used alternately (ping-pong).  g_0 (about
//                   phi) is held as hi + lo so that the small per-step changes of a near
//                   steady state survive the FP32 spacing of an O(1) value, and phi's
//                   total is conserved to far below FP32 resolution;
//   h[2][8][N]      post-stream potential populations h_1..h_8, two copies.  h_0 is not
//                   stored: it never enters varphi (Eq. weq55), grad varphi (Eq. eqA.16)
//                   or any other population, so it cannot influence any result;
//   hist[8][N]      lagged quantities s = u.grad phi, J = q u (x, y), R, F (x, y), and
//                   E (x, y) of the previous step (used by the lagged-field variant);
//   phi[N]          phi of the current step (input of the stencils and of the
//                   potential coefficient);
//   aq[N]           float2 per node: (a, q) with a = eps_hat / (c_s^2 tau_h (eps_hat +
//                   c_s^2 tau_h)), the coefficient of the potential forcing once
//                   grad varphi is written with the local first moment (Eq. eqA.16);
//   io[9][N]        staging area for field input / output;
//   partials[]      per-CTA FP64 partial sums;
//   ctl, stats      loop control and statistics (device structs below).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ehd {

constexpr int Q9 = 9;
constexpr int NPOP = 27;   // g, l, f
// FP32 planes of one population copy: the 27 populations and the low part of g_0 (the
// Cahn-Hilliard rest population is kept as an unevaluated sum hi + lo of two floats)
constexpr int NP32 = NPOP + 1;
// FP32 planes of one copy with FP16-deviation storage: the rest populations of g, l, f
// and the low part of g_0
constexpr int NP32_HALF = 4;
constexpr int NH = 8;      // h_1..h_8
constexpr int NHIST = 8;
constexpr int NIO = 9;   // field staging slots: one per ehd_read_fields bit
constexpr int MAX_PARTIALS = 1 << 16;
// Tiles of the streaming potential kernel (one CTA and one FP64 partial pair each).
constexpr int STREAM_TX = 64;
constexpr int STREAM_TY = 16;
__host__ __device__ constexpr long long stream_tiles(int nx, int ny) {
  return (long long)((nx + STREAM_TX - 1) / STREAM_TX) * ((ny + STREAM_TY - 1) / STREAM_TY);
}
// The moments pass runs at most this many CTAs of 256 threads (one wave on the GPU), each
// thread striding over the lattice, so the per-CTA reduction tails overlap.
constexpr int MOMENTS_MAX_BLOCKS = 1216;
__host__ __device__ constexpr int moments_blocks(int n) {
  return (n + 255) / 256 < MOMENTS_MAX_BLOCKS ? (n + 255) / 256 : MOMENTS_MAX_BLOCKS;
}

__host__ __device__ constexpr int cx(int i) {
  return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
  return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}
__host__ __device__ constexpr float wgt(int i) {
  return i == 0 ? 4.0f / 9.0f : (i <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
// CH source shape factor -1 + (|c_i|^2 - 2 c_s^2) / (2 c_s^2) of Eq. weq47:
// -2 (rest), -1/2 (axis), +1 (diagonal).
__host__ __device__ constexpr float ch_k(int i) {
  return i == 0 ? -2.0f : (i <= 4 ? -0.5f : 1.0f);
}

// Coefficients of one simulation, single precision, computed on the host from the
// double-precision parameters.
struct KParams {
  int nx, ny, N, walls;     // N: nodes per stored field (interior rows, plus ghost rows in a
                            // slab); walls applies to the sides without a ghost row
  int nint;                 // interior nodes nx * ny (= N outside slabs)
  int row0;                 // stored row of interior row 0: 1 in a slab (a ghost row below)
  int halo_lo, halo_hi;     // 1: the row below interior row 0 / above row ny-1 is a ghost row
                            // holding the neighbouring slab's values (slab decomposition)
  int slab;                 // 1: one slab of a decomposed lattice (reductions are combined
                            // across slabs by separate kernels)
  int y_global0, ny_global; // the slab's first row and the height of the whole lattice
  int neutralize;
  float rho_v, drho;        // rho = rho_v + drho phi
  float mu_v, dmu;          // mu = mu_v + dmu phi
  float sig_v, dsig;        // sigma = sig_v + dsig phi
  float eps_v, deps;        // eps_hat = phi^2 (2 phi - 3) deps, deps = eps_v - eps_l
  float beta4;              // 4 beta
  float kappa;
  float wet_a;              // sqrt(2 beta / kappa) = 4 / W
  float omega_g;            // 1 / tau_g
  float omega_l;            // 1 / tau_l
  float pref_l;             // 1 - 1 / (2 tau_l)
  float omega_h;            // 1 / tau_h
  float cs2tauh;            // c_s^2 tau_h
  int scheme;               // potential LBE: 0 the paper's (Eq. weq53), 1 conventional
  int field_fd;             // E outside the forcing: 0 local first moment, 1 stencil on varphi
  int lagged;               // 1: hbar of step n uses E of step n-1
  float inv_chi;            // conventional: 1 / chi
  float inv_chi_cs2;        // conventional: 1 / (chi c_s^2)
  float gbx, gby;           // body acceleration
  // ramped wall values (double: evaluated once per step by one thread)
  double cos_yb, cos_yt;    // cosines of the Young angles
  double ew_signed;         // ew_sign * eta/d of the bottom wall
  double varphi_b, varphi_t;
  int ramp_steps;
  // population storage: 0 FP32; 1 FP16 moving populations, stored as half(S_f p_i / w_i)
  // per field f (g, l, f) with power-of-two scales S_f, rest populations FP32
  int half;
  float psc[3];             // S_f
  float ipsc[3];            // 1 / S_f
  unsigned* oob;            // checked build: where out-of-range indices are counted
};

// Checked build (-DEHD_CHECKED; no counterpart in the paper): the indices the per-node
// helpers, the stencil loads, the coupled pass's stores and the two-step loop's state
// loads and stores form from lattice coordinates are tested against their field's size;
// one out of range is counted at k.oob and replaced by 0, so the run goes on without
// touching memory outside the field (no trap: a failing device assert is not an option on
// a shared GPU).  Other builds compile EHD_IDX to the index itself.
#ifdef EHD_CHECKED
__device__ __forceinline__ size_t checked_index(const KParams& k, size_t i, size_t n) {
  if (i < n) return i;
  if (k.oob) atomicAdd(k.oob, 1u);
  return 0;
}
#define EHD_IDX(k, i, n) ::ehd::checked_index((k), (size_t)(i), (size_t)(n))
#else
#define EHD_IDX(k, i, n) ((size_t)(i))
#endif

// One copy of the g, l, f populations.  FP32: p32 = [28][N] (the 27 populations, then the
// low part of g_0).  FP16: p32 = rest populations [3][N] and the low part of g_0, p16 =
// moving populations [24][N].
struct Pops {
  float* p32;
  __half* p16;
};

__host__ __device__ constexpr float inv_wgt(int i) {
  return i == 0 ? 9.0f / 4.0f : (i <= 4 ? 9.0f : 36.0f);
}

template <bool HALF>
__device__ __forceinline__ float ld_pop(const KParams& k, const Pops& P, int field, int i,
                                        size_t idx) {
  const size_t N = (size_t)k.N;
  idx = EHD_IDX(k, idx, N);
  if (!HALF) return __ldg(P.p32 + (size_t)(field * 9 + i) * N + idx);
  if (i == 0) return __ldg(P.p32 + (size_t)field * N + idx);
  const __half v = P.p16[(size_t)(field * 8 + i - 1) * N + idx];
  return __half2float(v) * (k.ipsc[field] * wgt(i));
}

template <bool HALF>
__device__ __forceinline__ void st_pop(const KParams& k, const Pops& P, int field, int i,
                                       size_t idx, float v) {
  idx = EHD_IDX(k, idx, k.N);
  const size_t N = (size_t)k.N;
  if (!HALF) {
    // the hydrodynamic populations are read only by the next coupled pass: stored
    // evict-first (st.global.cs); g and l stay in L2 for the next moments pass
    if (field == 2)
      __stcs(P.p32 + (size_t)(field * 9 + i) * N + idx, v);
    else
      P.p32[(size_t)(field * 9 + i) * N + idx] = v;
  } else if (i == 0) {
    if (field == 2)  // as above: the hydrodynamic populations evict-first
      __stcs(P.p32 + (size_t)field * N + idx, v);
    else
      P.p32[(size_t)field * N + idx] = v;
  } else {
    const __half hv = __float2half_rn(v * (k.psc[field] * inv_wgt(i)));
    if (field == 2)
      __stcs(P.p16 + (size_t)(field * 8 + i - 1) * N + idx, hv);
    else
      P.p16[(size_t)(field * 8 + i - 1) * N + idx] = hv;
  }
}

// The low part of the rest Cahn-Hilliard population g_0 = hi + lo (hi is population (0, 0)).
template <bool HALF>
__device__ __forceinline__ float ld_g0_lo(const KParams& k, const Pops& P, size_t idx) {
  idx = EHD_IDX(k, idx, k.N);
  return __ldg(P.p32 + (size_t)(HALF ? 3 : NPOP) * k.N + idx);
}
template <bool HALF>
__device__ __forceinline__ void st_g0_lo(const KParams& k, const Pops& P, size_t idx, float v) {
  idx = EHD_IDX(k, idx, k.N);
  P.p32[(size_t)(HALF ? 3 : NPOP) * k.N + idx] = v;
}
// Stores a population and returns the value a later ld_pop of it reads (with FP16 storage
// the rounded value).
template <bool HALF>
__device__ __forceinline__ float st_pop_read(const KParams& k, const Pops& P, int field, int i,
                                             size_t idx, float v) {
  idx = EHD_IDX(k, idx, k.N);
  const size_t N = (size_t)k.N;
  if (!HALF || i == 0) {
    st_pop<HALF>(k, P, field, i, idx, v);
    return v;
  }
  const __half hv = __float2half_rn(v * (k.psc[field] * inv_wgt(i)));
  if (field == 2)
    __stcs(P.p16 + (size_t)(field * 8 + i - 1) * N + idx, hv);
  else
    P.p16[(size_t)(field * 8 + i - 1) * N + idx] = hv;
  return __half2float(hv) * (k.ipsc[field] * wgt(i));
}
// phi = sum_i g_i of a node (Eq. weq49) with g_0 = hi + lo: the moving populations in
// direction order, the low part, then the high part.  Every kernel forms phi this way.
template <bool HALF>
__device__ __forceinline__ float phi_of(const KParams& k, const Pops& P, size_t idx) {
  float m = 0.0f;
#pragma unroll
  for (int i = 1; i < 9; ++i) m = __fadd_rn(m, ld_pop<HALF>(k, P, 0, i, idx));
  return __fadd_rn(ld_pop<HALF>(k, P, 0, 0, idx), __fadd_rn(m, ld_g0_lo<HALF>(k, P, idx)));
}
// The moments of one node from its post-stream populations (Algorithm 1, first step):
// phi = sum_i g_i with g_0 = hi + lo (the moving populations summed in order, then lo,
// then hi, as phi_of does) and q = sum_i l_i + R/2 (the Nernst-Planck source's half-step
// correction).  Every rounding is explicit: the same bits in every translation unit.
__device__ __forceinline__ void moments_of(const float (&g)[9], float lo, const float (&l)[9],
                                           float R, float& phi, float& q) {
  float m = 0.0f;
#pragma unroll
  for (int i = 1; i < 9; ++i) m = __fadd_rn(m, g[i]);
  phi = __fadd_rn(g[0], __fadd_rn(m, lo));
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 9; ++i) s = __fadd_rn(s, l[i]);
  q = __fadd_rn(s, __fmul_rn(0.5f, R));
}

// (hi, lo) + d as two floats again: Knuth's two-sum of hi and d (exact), the rounding
// error folded into lo, then one fast two-sum to renormalise.
__device__ __forceinline__ void two_float_add(float& hi, float& lo, float d) {
  const float s = __fadd_rn(hi, d);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(d, bp));
  const float l2 = __fadd_rn(lo, e);
  hi = __fadd_rn(s, l2);
  lo = __fsub_rn(l2, __fsub_rn(hi, s));
}

// Values that change from step to step, kept on the device so that a step needs no
// host input: written for the next step by the coupled kernel (one thread), for the
// first step by k_step_set.  Two slots, indexed like the population copies.
struct StepState {
  long long n;              // step index
  int first;                // 1: no history yet, backward differences are zero
  int pad;
  float cos_b, cos_t;       // effective contact-angle cosines of the bottom / top walls
  float vw_b, vw_t;         // wall potentials
};

// Ramp fraction r = min(1, n / ramp_steps); wall potentials r varphi_w; the bottom
// wall's electrowetting term scales with r^2 (Eq. weq69: eta/d is quadratic in the
// voltage); cosines clamped to [-1, 1].  Explicit roundings keep it free of fused
// multiply-adds.
__device__ __forceinline__ StepState make_step(const KParams& k, long long n, int first) {
  StepState s;
  double r = 1.0;
  if (k.ramp_steps > 0) {
    r = __ddiv_rn((double)n, (double)k.ramp_steps);
    r = r < 1.0 ? r : 1.0;
  }
  double cb = __dadd_rn(k.cos_yb, __dmul_rn(__dmul_rn(k.ew_signed, r), r));
  double ct = k.cos_yt;
  cb = cb < -1.0 ? -1.0 : (cb > 1.0 ? 1.0 : cb);
  ct = ct < -1.0 ? -1.0 : (ct > 1.0 ? 1.0 : ct);
  s.n = n;
  s.first = first;
  s.pad = 0;
  s.cos_b = (float)cb;
  s.cos_t = (float)ct;
  s.vw_b = (float)__dmul_rn(r, k.varphi_b);
  s.vw_t = (float)__dmul_rn(r, k.varphi_t);
  return s;
}

// Potential loop control; written by the reduction of the moments kernel (reset) and of
// the potential kernel (advance), read at the start of each potential launch.
struct Ctl {
  int iter;                 // sub-iterations made in the current solve
  int done;                 // loop finished: later potential launches do nothing
  int converged;            // finished by the stopping rule (or a fixed count)
  int parity;               // which h copy holds the current state
  double rel;               // relative change of the last sub-iteration
  double tol;
  int min_iter, max_iter, fixed_iter;
  int nonfinite;            // phi or q held NaN / Inf
  double sum_phi, sum_q;    // FP64 sums of phi and q of the last moments pass
  float mean_q;             // sum_q / N (source shift when neutralising)
  unsigned ticket_m;        // CTA arrival counters of the two reductions
  unsigned ticket_p;
  float vw_b, vw_t;         // wall potentials of the current solve
  unsigned bar_count;       // grid barrier of the resident potential loop: arrivals in
                            // the current solve (reset with the loop control)
  int bar_error;            // a barrier wait timed out (sticky)
  double slab_num, slab_den;// one slab's stopping sums of its last sub-iteration
  int mpart_n;              // > 0: the moments pass left its FP64 sums as this many
                            // per-CTA partials, reduced by the coupled pass
  unsigned oob;             // checked build: out-of-range indices met (see EHD_IDX)
};

// Tiling of the resident potential loop: ntx x nty tiles of TX x TY nodes (the last
// column / row may be smaller), pmax perimeter slots per tile.
struct ResidentGeom {
  int TX, TY, ntx, nty, pmax;
  int depth;  // 0: one sub-iteration per exchange; 2, 3: that many (ring and band as wide)
};

struct DevStats {
  int iters_total, iters_min, iters_max, not_converged, nonfinite, steps;
  int barrier_error, pad;
  double last_rel, sum_phi, sum_q;
};

// Property laws (Remark II, Eq. weq36).
__device__ __forceinline__ float eps_hat_of(const KParams& k, float phi) {
  return __fmul_rn(__fmul_rn(__fmul_rn(phi, phi), __fsub_rn(__fmul_rn(2.0f, phi), 3.0f)), k.deps);
}

// Per-node coefficient of the potential collision, kept in aq[].x: the paper's scheme
// a = eps_hat / (c_s^2 tau_h (eps_hat + c_s^2 tau_h)) (forcing through the local first
// moment, Eq. eqA.16); the conventional scheme its relaxation rate 1 / tau_varphi with
// tau_varphi = 1/2 + eps(phi) / (chi c_s^2) (Sec. 3.3).
// Every rounding is explicit, so each translation unit computes the same bits whatever its
// multiply-add contraction.
__device__ __forceinline__ float potential_coef(const KParams& k, float phi) {
  const float eh = eps_hat_of(k, phi);
  if (k.scheme == 1)
    return __fdiv_rn(1.0f, __fadd_rn(0.5f, __fmul_rn(__fadd_rn(k.eps_v, eh), k.inv_chi_cs2)));
  return __fdiv_rn(eh, __fmul_rn(k.cs2tauh, __fadd_rn(eh, k.cs2tauh)));
}
// The denominator d of grad varphi = -sum_i c_i h_i / d: eps_hat + c_s^2 tau_h
// (Eq. eqA.16), or c_s^2 tau_varphi for the conventional scheme.
__device__ __forceinline__ float potential_den(const KParams& k, float phi) {
  const float eh = eps_hat_of(k, phi);
  if (k.scheme == 1) return (1.0f / 3.0f) * (0.5f + (k.eps_v + eh) * k.inv_chi_cs2);
  return eh + k.cs2tauh;
}
__device__ __forceinline__ float deps_of(const KParams& k, float phi) {
  return 6.0f * phi * (phi - 1.0f) * k.deps;
}

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

template <typename T>
__device__ __forceinline__ T ld_cg(const T* p) { return __ldcg(p); }

// Potential sub-iteration arithmetic (Eq. weq53 with the forcing of Eq. eqA.16 written
// through the local first moment), shared by every kernel that runs the potential loop.
// Each rounding is explicit (no multiply-add contraction by the compiler), so the
// streaming, resident and batched loops compute the same bits for the same state.
//
// varphi = (sum_{i>0} h_i) / (1 - w_0) = 9/5 sum h_i (Eq. weq55); m1 = sum c_i h_i.
__device__ __forceinline__ float h_sum8(const float (&h)[8]) {
  float s = h[0];
#pragma unroll
  for (int i = 1; i < 8; ++i) s = __fadd_rn(s, h[i]);
  return s;
}
__device__ __forceinline__ float h_varphi(float hsum) { return __fmul_rn(hsum, 9.0f / 5.0f); }
__device__ __forceinline__ void h_moment1(const float (&h)[8], float& m1x, float& m1y) {
  m1x = __fadd_rn(__fsub_rn(__fsub_rn(__fadd_rn(__fsub_rn(h[0], h[2]), h[4]), h[5]), h[6]),
                  h[7]);
  m1y = __fsub_rn(__fsub_rn(__fadd_rn(__fadd_rn(__fsub_rn(h[1], h[3]), h[4]), h[5]), h[6]),
                  h[7]);
}
// Post-collision h_i* (i = 1..8): h_i - (h_i - w_i varphi)/tau_h + a w_i c_i.m1 + q/8, with
// a = eps_hat / (c_s^2 tau_h (eps_hat + c_s^2 tau_h)) and q/8 the source share.
__device__ __forceinline__ float h_star(int i, float hi, float om, float varphi, float a,
                                        float m1x, float m1y, float qs) {
  const float w = wgt(i);
  const float cm = (cx(i) != 0 && cy(i) != 0) ? __fadd_rn(cx(i) * m1x, cy(i) * m1y)
                                               : (cx(i) != 0 ? cx(i) * m1x : cy(i) * m1y);
  float v = __fmaf_rn(-w, varphi, hi);
  v = __fmaf_rn(-om, v, hi);
  v = __fmaf_rn(__fmul_rn(a, w), cm, v);
  return __fadd_rn(v, qs);
}
// Conventional scheme (Sec. 3.3): h_i - (h_i - w_i varphi) / tau_varphi + q / (8 chi),
// om_x = 1 / tau_varphi of the node, qs = q / (8 chi).
__device__ __forceinline__ float h_star_conv(int i, float hi, float om_x, float varphi,
                                             float qs) {
  float v = __fmaf_rn(-wgt(i), varphi, hi);
  v = __fmaf_rn(-om_x, v, hi);
  return __fadd_rn(v, qs);
}
// Anti-bounce-back at a Dirichlet wall of potential vw: -h_opp* + 2 w_i vw.
__device__ __forceinline__ float h_wall(int i, float h_opp_star, float vw) {
  return __fmaf_rn(2.0f * wgt(i), vw, -h_opp_star);
}
// The same arithmetic on two nodes at once (packed FP32 pairs; each component rounds as
// the scalar form above, so the results are bit-identical to it).
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 h_sum8x2(const float2 (&h)[8]) {
  float2 s = h[0];
#pragma unroll
  for (int i = 1; i < 8; ++i) s = __fadd2_rn(s, h[i]);
  return s;
}
__device__ __forceinline__ float2 h_varphi2(float2 hsum) { return __fmul2_rn(hsum, f2(9.0f / 5.0f)); }
__device__ __forceinline__ void h_moment1x2(const float2 (&h)[8], float2& m1x, float2& m1y) {
  m1x = __fadd2_rn(__fadd2_rn(__fadd2_rn(__fadd2_rn(__fadd2_rn(h[0], neg2(h[2])), h[4]),
                                         neg2(h[5])), neg2(h[6])), h[7]);
  m1y = __fadd2_rn(__fadd2_rn(__fadd2_rn(__fadd2_rn(__fadd2_rn(h[1], neg2(h[3])), h[4]), h[5]),
                              neg2(h[6])), neg2(h[7]));
}
// Post-collision h_1*..h_8* of two nodes.  c_i.m1 is +-m1x, +-m1y, +-(m1x + m1y) or
// +-(m1x - m1y); its sign is moved onto a w_i (exact), which the scalar form rounds alike.
__device__ __forceinline__ void h_star8x2(const float2 (&h)[8], float om, float2 varphi, float2 a,
                                          float2 m1x, float2 m1y, float2 qs, float2 (&out)[8]) {
  const float2 aw1 = __fmul2_rn(a, f2(wgt(1))), aw2 = __fmul2_rn(a, f2(wgt(5)));
  const float2 dp = __fadd2_rn(m1x, m1y), dm = __fadd2_rn(m1x, neg2(m1y));
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const float w = wgt(i);
    float2 coef, m;
    if (i <= 4) {
      coef = (cx(i) + cy(i)) > 0 ? aw1 : neg2(aw1);
      m = cx(i) != 0 ? m1x : m1y;
    } else {
      coef = cx(i) > 0 ? aw2 : neg2(aw2);
      m = cx(i) == cy(i) ? dp : dm;
    }
    float2 v = __ffma2_rn(f2(-w), varphi, h[i - 1]);
    v = __ffma2_rn(f2(-om), v, h[i - 1]);
    v = __ffma2_rn(coef, m, v);
    out[i - 1] = __fadd2_rn(v, qs);
  }
}
// h_star_conv on two nodes at once: om_x their 1 / tau_varphi, qs their q / (8 chi).
__device__ __forceinline__ void h_star_conv8x2(const float2 (&h)[8], float2 om_x, float2 varphi,
                                               float2 qs, float2 (&out)[8]) {
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    float2 v = __ffma2_rn(f2(-wgt(i)), varphi, h[i - 1]);
    v = __ffma2_rn(neg2(om_x), v, h[i - 1]);
    out[i - 1] = __fadd2_rn(v, qs);
  }
}

// Stopping sums: (varphi^{k+1} - varphi^k)^2 and (varphi^k)^2 added to num, den.
__device__ __forceinline__ void h_change(float vnew, float vold, float& num, float& den) {
  const float d = __fsub_rn(vnew, vold);
  num = __fmaf_rn(d, d, num);
  den = __fmaf_rn(vold, vold, den);
}

}  // namespace ehd

// Launch functions implemented in the .cu files (host side).
namespace ehd {
struct Buffers {
  StepState* ss;     // [2]
  float* pops;       // FP32: [2][28][N]; FP16: [2][4][N] rest populations and g_0's low part
  __half* pops16;    // FP16: [2][24][N] moving populations
  float* h;          // [2][8][N]
  float* hist;       // [6][N]
  float* phi;        // [N]
  float2* aq;        // [N]
  float* io;         // [9][N]
  float* tmp;        // [N]
  double2* partials; // [MAX_PARTIALS]
  Ctl* ctl;
  DevStats* stats;
  float* exports;    // resident loop: [2][tiles][8][pmax]
  float2* rpartials; // resident loop: [2][tiles] float2; D-step loop: [2][tiles][D / 2 + D % 2] float4
};

__host__ __device__ inline Pops pops_copy(const KParams& k, const Buffers& b, int c) {
  Pops P;
  if (k.half) {
    P.p32 = b.pops + (size_t)c * NP32_HALF * k.N;
    P.p16 = b.pops16 + (size_t)c * 24 * k.N;
  } else {
    P.p32 = b.pops + (size_t)c * NP32 * k.N;
    P.p16 = nullptr;
  }
  return P;
}

// Everything the resident loop of one simulation needs (batch launches keep a table).
struct ResidentSlot {
  KParams k;
  ResidentGeom rg;
  float* h;
  const float2* aq;
  float* exports;
  float2* rpartials;
  Ctl* ctl;
};

// Tile height of every simulation in a batch (tiles of 64 x rows nodes): the default, and
// the heights a batch may be set to (all slots of a batch share one).
constexpr int BATCH_ROWS = 32;
constexpr int BATCH_ROW_CHOICES[3] = {16, 32, 64};

// One simulation of a batch as the batched moments and coupled kernels see it.
struct StepSlot {
  KParams k;
  Buffers b;
  double tol;
  int min_iter, max_iter, fixed_iter;
  int mblocks;       // moments blocks of this simulation (its own moments launch's grid)
  int quad;          // 1: moments four nodes per thread, as k_moments4 (moments4_ok)
};

// Whether a lattice's moments pass takes four nodes per thread with vector loads
// (k_moments4): no slab, N a multiple of 4 (either storage precision).
__host__ __device__ inline bool moments4_ok(const KParams& kp) {
  return !kp.slab && kp.N % 4 == 0 && kp.N == kp.nint;
}

// Batched moments / coupled passes: one launch over work[] = (slot, block of that slot).
cudaError_t add_moments_batch_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                                   cudaGraphNode_t* out, const StepSlot* slots, const int2* work,
                                   int nwork, int cur);
// half: the work items are of FP16-storage slots (the pass's FP16 form), else FP32.
cudaError_t add_coupled_batch_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                                   cudaGraphNode_t* out, const StepSlot* slots, const int2* work,
                                   int nwork, int cur, bool half);

// Resident potential loop (poisson_resident.cu).  fixed_ty > 0: tiles of 64 x fixed_ty
// (a multiple of 8 up to 64).
bool resident_geometry(const KParams& kp, int num_sms, ResidentGeom* g, int* threads,
                       size_t* smem, int fixed_ty = 0, int depth = 0);
// The single-simulation kernel of a tile height (nullptr if none): heights 8..64 in
// steps of 8; with two sub-iterations per exchange, 24..64.
const void* resident_kernel(int tile_rows, int depth = 0, bool conv = false);
const void* resident_batch_kernel(int tile_rows);  // 16, 32 or 64; else nullptr
// Tensor-memory columns (of the SM's 512) one CTA of that loop allocates: 0 for the
// one-step loop, -1 for a shape with no kernel.
int resident_tmem_columns(int tile_rows, int depth);
cudaError_t launch_poisson_resident(const KParams& kp, const ResidentGeom& g, int threads,
                                    size_t smem, const Buffers& b, cudaStream_t st);
cudaError_t add_poisson_resident_node(cudaGraph_t graph, const cudaGraphNode_t* deps, size_t nd,
                                      cudaGraphNode_t* out, const KParams& kp,
                                      const ResidentGeom& g, int threads, size_t smem,
                                      const Buffers& b);

cudaError_t launch_step_set(const KParams& kp, const Buffers& b, int slot, long long n,
                            int first, cudaStream_t st);
cudaError_t launch_init(const KParams& kp, const Buffers& b, int cur, bool have_p,
                        cudaStream_t st);
// sums_in_coupled: the potential loop that follows runs on chip, so (without a neutralised
// source) the moments pass may leave its FP64 sums as per-CTA partials for the coupled pass.
cudaError_t launch_moments(const KParams& kp, const Buffers& b, int cur, double tol,
                           int min_iter, int max_iter, int fixed_iter, cudaStream_t st,
                           bool sums_in_coupled = false);
cudaError_t launch_poisson(const KParams& kp, const Buffers& b, cudaStream_t st);
cudaError_t launch_coupled(const KParams& kp, const Buffers& b, int cur, cudaStream_t st);
cudaError_t launch_stats_reset(const Buffers& b, cudaStream_t st);
cudaError_t launch_expire_barrier(const Buffers& b, cudaStream_t st);
cudaError_t launch_fields(const KParams& kp, const Buffers& b, int cur, unsigned mask,
                          cudaStream_t st);
cudaError_t launch_phi_now(const KParams& kp, const Buffers& b, int cur, cudaStream_t st);
// The contact line on the bottom wall into b.partials[0..1] (see k_contact_line).
cudaError_t launch_contact_line(const KParams& kp, const Buffers& b, int cur, float level,
                                cudaStream_t st);
cudaError_t launch_fields_from_phi(const KParams& kp, const Buffers& b, int cur, unsigned mask,
                                   cudaStream_t st);
cudaError_t add_poisson_node_nocond(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                                    cudaGraphNode_t* out, const KParams& kp, const Buffers& b);

// Graph nodes of the per-step kernels (argument values are copied into the node).
cudaError_t add_moments_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                             cudaGraphNode_t* out, const KParams& kp, const Buffers& b, int cur,
                             double tol, int min_iter, int max_iter, int fixed_iter,
                             bool sums_in_coupled = false);
cudaError_t add_coupled_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                             cudaGraphNode_t* out, const KParams& kp, const Buffers& b, int cur);

// Graph of one time step for population copy `cur`: moments -> while(loop not done)
// { potential sub-iteration } -> coupled pass.  All arguments live on the device, so the
// graph is launched unchanged every step.
// With `rg` non-null the potential loop is the single resident cooperative kernel instead
// of the WHILE node.
// With `ev` (4 events) the graph records ev[0] before the moments pass, ev[1] after it,
// ev[2] after the potential loop and ev[3] after the coupled pass (per-kernel timing).
// With nsteps > 1 (and no events) the graph holds that many consecutive steps, the first
// on population copy `cur`, the copies alternating: one launch runs them all.
cudaError_t build_step_graph(const KParams& kp, const Buffers& b, int cur, double tol,
                             int min_iter, int max_iter, int fixed_iter, const ResidentGeom* rg,
                             int rthreads, size_t rsmem, cudaGraph_t* out,
                             const cudaEvent_t* ev = nullptr, int nsteps = 1);
}  // namespace ehd
