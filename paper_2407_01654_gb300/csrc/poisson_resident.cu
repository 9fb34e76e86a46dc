// The whole potential loop of one solve (Algorithm 1 step 3) in one cooperative launch,
// with the potential populations held on chip.
//
// The lattice is cut into 64 x TY tiles (TY a multiple of 8, a compile-time constant of
// the kernel), one CTA of 16 TY threads per tile.  Thread t owns the four nodes of column
// t mod 64 in rows t/64 + s TY/4 (s = 0..3) and keeps their post-stream populations
// h_1..h_8 in registers for the whole loop, so every shared-memory address is a
// per-thread base plus a constant.  A sub-iteration (Eq. weq53, the same arithmetic as k_poisson):
//   1. collide the tile's nodes; post-collision populations go to shared memory, and
//      those of perimeter nodes also to a per-tile export area in global memory;
//   2. grid barrier;
//   3. decide: one lane reduces the previous sub-iteration's per-tile partial sums in a
//      fixed order and applies the stopping rule, so every CTA takes the same decision;
//      if the loop is done the registers hold exactly the paper's final state, which is
//      written back;
//   4. stream: gather h_i(x) = h*_i(x - c_i) from shared memory, from a neighbour tile's
//      export area, or from the anti-bounce-back wall rule; form varphi^{k+1} and the
//      partial sums of sum (varphi^{k+1} - varphi^k)^2 and sum (varphi^k)^2.
// Export areas and partials are double-buffered by sub-iteration parity, so one grid
// barrier per sub-iteration suffices.  The collision made just before the loop stops
// never leaves the chip.
//
// The stopping sums are FP32 throughout (per node, per warp, per tile, across tiles, each
// in a fixed order).  varphi^{k+1} - varphi^k is itself an FP32 difference of two nearly
// equal FP32 values, so the summand carries a relative error near 1e-7 / (relative
// change); FP32 accumulation (relative error below 1e-6 for these tree depths) adds
// nothing visible to the decision, and the FP64 units of this part are slow enough that
// FP64 sums here cost more than the rest of a sub-iteration.
//
// The grid barrier counts arrivals in the loop control (reset for each solve by the
// moments kernel): a CTA adds one with release semantics and waits, with acquire loads
// and a time limit, until the count reaches its target; on timeout it sets an error flag
// and the kernel returns (with a cooperative launch all CTAs are co-resident, so the
// limit is never reached in normal operation).
#include "ehd_internal.cuh"

#include <type_traits>

namespace ehd {

namespace {

constexpr int NPT = 4;              // nodes per thread
constexpr int TXR = 64;             // tile width
constexpr int RX = TXR + 2;         // shared ring row: the tile row plus one node each side
constexpr unsigned long long BARRIER_TIMEOUT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// The grid barriers of the loops below (co-resident CTAs): after a CTA barrier, thread 0
// adds one arrival with release semantics and polls the count with acquire loads until
// it reaches `target` (the arrivals it waits for), within BARRIER_TIMEOUT_NS; a timeout
// sets Ctl::bar_error and the CTA leaves its loop.

__device__ __forceinline__ int perim_slot(int lx, int ly, int w, int h) {
  if (ly == 0) return lx;
  if (ly == h - 1) return w + lx;
  if (lx == 0) return 2 * w + ly;
  return 2 * w + h + ly;  // lx == w - 1
}

// One of the 3 x 3 tiles around (and including) this one.
struct Nb {
  int id;      // tile index, -1 beyond a wall
  int w, h;    // its size
};

// Compile-time shape of a 64 x TY tile.
template <int TY>
struct Tile {
  static_assert(TY % 8 == 0 && TY >= 8 && TY <= 64, "tile height: a multiple of 8 up to 64");
  static constexpr int RY = TY + 2;
  static constexpr int PLANE = RY * RX;            // one direction's shared populations
  static constexpr int THREADS = TXR * TY / NPT;   // 16 TY
  static constexpr int ROWS = TY / NPT;            // rows between a thread's nodes
  static constexpr int PMAX = 2 * TXR + 2 * TY;    // perimeter slots
  static constexpr int MIN_BLOCKS = THREADS >= 1024 ? 1 : (1024 / THREADS);
};

}  // namespace

// The loop for one tile of one simulation; `tile` of `ntiles` tiles of that simulation.
// CONV: the conventional potential collision (Sec. 3.3; per-node 1 / tau_varphi in the
// coefficient array, q / chi as the source) instead of the paper's.
template <int TY, bool CONV>
__device__ __forceinline__ void resident_loop(const KParams& k, const ResidentGeom& rg,
                                              float* __restrict__ hbuf,
                                              const float2* __restrict__ aq,
                                              float* __restrict__ exports,
                                              float2* __restrict__ rpartials, Ctl* ctl,
                                              const int tile, const int ntiles) {
  using T = Tile<TY>;
  extern __shared__ float sm[];  // [8][RY][RX] populations, then [TY*64] a, [TY*64] q
  __shared__ float2 s_w[T::THREADS / 32];
  __shared__ int s_done, s_ok;
  __shared__ Nb s_nb[3][3];

  const int nx = k.nx, ny = k.ny;
  const size_t N = (size_t)k.N;
  const int tcol = tile % rg.ntx, trow = tile / rg.ntx;
  const int tx0 = tcol * TXR, ty0 = trow * TY;
  const int tw = min(TXR, nx - tx0), th = min(TY, ny - ty0);
  float* ca = sm + 8 * T::PLANE;
  float* cq = ca + TY * TXR;
  // the loop control's fields this solve reads but no CTA of it writes come through the
  // read-only path: every warp of every CTA asks for the same few words at once, which
  // L1 merges per SM instead of sending each request to one L2 slice
  const int parity = __ldg(&ctl->parity);
  float* __restrict__ hsrc = hbuf + (size_t)parity * NH * N;
  const float qshift = k.neutralize ? __ldg(&ctl->mean_q) : 0.0f;
  const float vw_b = __ldg(&ctl->vw_b), vw_t = __ldg(&ctl->vw_t);
  const double tol = ctl->tol;
  // a non-finite phi or q (flagged by the moments pass) stops the loop after one
  // sub-iteration, not converged
  const bool bad_state = __ldg(&ctl->nonfinite) != 0;
  const int min_iter = bad_state ? 1 : ctl->min_iter, max_iter = bad_state ? 1 : ctl->max_iter,
            fixed = bad_state ? 0 : ctl->fixed_iter;
  const float om = k.omega_h;
  constexpr int pstride = 8 * T::PMAX;
  // this thread's nodes: column lx, rows ly0 + s ROWS
  const int lx = threadIdx.x & (TXR - 1);
  const int ly0 = threadIdx.x >> 6;
  const int at0 = (ly0 + 1) * RX + lx + 1;   // shared index of node 0 (direction 1's plane)
  const int j0 = ly0 * TXR + lx;             // coefficient index of node 0
  const int nrows = lx < tw ? th : 0;        // my nodes are the rows ly0 + s ROWS < nrows

  if (threadIdx.x < 9) {
    const int dx = (int)threadIdx.x % 3 - 1, dy = (int)threadIdx.x / 3 - 1;
    const int c = (tcol + dx + rg.ntx) % rg.ntx;
    int r = trow + dy;
    Nb nb;
    if (r < 0 || r >= rg.nty) {
      if (k.walls) {
        nb.id = -1;
        nb.w = nb.h = 0;
        s_nb[dy + 1][dx + 1] = nb;
        r = -1;
      } else {
        r = (r + rg.nty) % rg.nty;
      }
    }
    if (r >= 0) {
      nb.id = r * rg.ntx + c;
      nb.w = min(TXR, nx - c * TXR);
      nb.h = min(TY, ny - r * TY);
      s_nb[dy + 1][dx + 1] = nb;
    }
  }

  // state of my nodes: registers, as two pairs (nodes 0, 1 and 2, 3) for packed FP32
  // arithmetic; coefficients: shared memory.  Nodes outside the lattice (partial tiles)
  // compute along with their pair but never enter a sum, an export or the result, and
  // every shared-memory cell they write lies inside the tile's array and is either never
  // read by a lattice node or rewritten by the ring fill before it is.
  float2 h[2][8];
  bool valid[NPT];
  float2 c4[NPT];
  // every load is issued before any is used (a node outside the lattice loads node 0 of
  // the lattice and then starts from zero)
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    valid[s] = ly0 + s * T::ROWS < nrows;
    const int g = valid[s] ? (ty0 + ly0 + s * T::ROWS) * nx + tx0 + lx : 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (s & 1)
        h[s >> 1][i].y = hsrc[i * N + g];
      else
        h[s >> 1][i].x = hsrc[i * N + g];
    }
    c4[s] = aq[g];
  }
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    ca[j0 + s * T::ROWS * TXR] = valid[s] ? c4[s].x : 0.0f;
    const float qn = __fsub_rn(c4[s].y, qshift);
    cq[j0 + s * T::ROWS * TXR] = valid[s] ? (CONV ? __fmul_rn(qn, k.inv_chi) : qn) : 0.0f;
    if (!valid[s]) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (s & 1)
          h[s >> 1][i].y = 0.0f;
        else
          h[s >> 1][i].x = 0.0f;
      }
    }
  }
  __syncthreads();

  unsigned target = 0;
  int it = 0;
  float rel = 0.0f;
  int conv = 0;
  constexpr int dwarp = T::THREADS / 32 - 1;  // the warp that reduces the tiles' sums
  // One sub-iteration; returns 0 to go on, 1 when the rule stopped the loop at the previous
  // one, 2 when the grid barrier timed out.  Sub-iterations alternate between two layouts
  // of the shared populations (SW: sub-iteration it odd).  Own layout: direction i of the
  // node at x sits in slot i of its own cell and streams from slot i of the cell x - c_i.
  // Swapped layout: it goes to slot opp(i) of the cell x + c_i, and streams from slot
  // opp(i) of the node's own cell.  A slot the collision of sub-iteration it + 1 writes was
  // read in the streaming of sub-iteration it only by the writing thread itself, so no CTA
  // barrier separates a streaming from the next collision.
  auto sub_iteration = [&](auto swc) -> int {
    constexpr bool SW = decltype(swc)::value;
    // where direction i of the node at shared index f lies after the collision
    auto slot = [](int i, int f) {
      return SW ? (opp(i) - 1) * T::PLANE + f + cy(i) * RX + cx(i) : (i - 1) * T::PLANE + f;
    };
    // 1. collide into the tile's shared populations; keep varphi^k per node
    float2 vold[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int o0 = 2 * p * T::ROWS, o1 = (2 * p + 1) * T::ROWS;  // row offsets of the pair
      const float2 varphi = h_varphi2(h_sum8x2(h[p]));
      vold[p] = varphi;
      float2 m1x, m1y;
      h_moment1x2(h[p], m1x, m1y);
      const float2 a = make_float2(ca[j0 + o0 * TXR], ca[j0 + o1 * TXR]);
      const float2 qs = __fmul2_rn(f2(0.125f), make_float2(cq[j0 + o0 * TXR], cq[j0 + o1 * TXR]));
      float2 hs[8];
      if constexpr (CONV)
        h_star_conv8x2(h[p], a, varphi, qs, hs);
      else
        h_star8x2(h[p], om, varphi, a, m1x, m1y, qs, hs);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        sm[slot(i + 1, at0) + o0 * RX] = hs[i].x;
        sm[slot(i + 1, at0) + o1 * RX] = hs[i].y;
      }
    }
    __syncthreads();
    // perimeter nodes export their post-collision populations for the neighbour tiles
    {
      float* exp_cur = exports + (size_t)(it & 1) * ntiles * pstride + (size_t)tile * pstride;
      const int np = 2 * tw + 2 * th;
      for (int sl = threadIdx.x; sl < np; sl += T::THREADS) {
        int ex, ey;
        if (sl < tw) { ex = sl; ey = 0; }
        else if (sl < 2 * tw) { ex = sl - tw; ey = th - 1; }
        else if (sl < 2 * tw + th) { ex = 0; ey = sl - 2 * tw; }
        else { ex = tw - 1; ey = sl - 2 * tw - th; }
        const int at = (ey + 1) * RX + ex + 1;
#pragma unroll
        for (int i = 1; i < 9; ++i) exp_cur[(i - 1) * T::PMAX + sl] = sm[slot(i, at)];
      }
    }
    // 2. grid barrier: warp 0 reduces the previous sub-iteration's warp sums (warps in a
    // fixed order) and its lane 0 publishes them, then releases the CTA's exports (ordered
    // before it by the CTA barrier) and waits, within a time limit, for every tile
    __syncthreads();
    target += ntiles;
    if (threadIdx.x < 32) {
      if (it > 0) {
        constexpr int nwarps = T::THREADS / 32;
        float2 v = (int)threadIdx.x < nwarps ? s_w[threadIdx.x] : make_float2(0.0f, 0.0f);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
          v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
        }
        if (threadIdx.x == 0) rpartials[(size_t)((it - 1) & 1) * ntiles + tile] = v;
      }
      if (threadIdx.x == 0) {
        int ok = 1;
        red_release_add(&ctl->bar_count, 1u);
        const unsigned long long t0 = global_ns();
        while ((int)(ld_acquire(&ctl->bar_count) - target) < 0) {
          if (global_ns() - t0 > BARRIER_TIMEOUT_NS) {
            atomicOr(&ctl->bar_error, 1);
            ok = 0;
            break;
          }
        }
        s_ok = ok;
      }
    }
    __syncthreads();  // every tile's exports and sums visible (or the wait gave up)
    if (!s_ok) return 2;
    // 3. the deciding warp reduces the previous sub-iteration's sums (tiles in a fixed
    // order) and one lane applies the stopping rule, while the other warps fill the ring
    if (it > 0 && (int)(threadIdx.x >> 5) == dwarp) {
      const int lane = threadIdx.x & 31;
      const float2* pp = rpartials + (size_t)((it - 1) & 1) * ntiles;
      float sa = 0.0f, sb = 0.0f;
      for (int t = lane; t < ntiles; t += 32) {
        const float2 v = __ldcg(pp + t);
        sa += v.x;
        sb += v.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
      }
      if (lane == 0) {
        if (sa == 0.0f && sb == 0.0f)
          rel = 0.0f;
        else if (sb == 0.0f)
          rel = __int_as_float(0x7f800000);
        else
          rel = sqrtf(sa / sb);
        bool done;
        if (fixed > 0) {
          done = it >= fixed;
          conv = 1;
        } else {
          conv = (it >= min_iter) && ((double)rel < tol);
          done = conv || it >= max_iter;
        }
        s_done = done;
      }
    }
    // 4a. ring: for every boundary node and direction whose source lies outside the tile,
    // put the source value where the streaming will read it
    {
      const float* exp_all = exports + (size_t)(it & 1) * ntiles * pstride;
      const int nring = 6 * (tw + th);
      for (int e = threadIdx.x; e < nring; e += T::THREADS) {
        int bx, by, i;
        if (e < 3 * th) {                 // west boundary, directions with cx = +1
          by = e / 3; bx = 0;
          const int kk = e - 3 * by;
          i = kk == 0 ? 1 : (kk == 1 ? 5 : 8);
        } else if (e < 6 * th) {          // east boundary, cx = -1
          const int f = e - 3 * th;
          by = f / 3; bx = tw - 1;
          const int kk = f - 3 * by;
          i = kk == 0 ? 3 : (kk == 1 ? 6 : 7);
        } else if (e < 6 * th + 3 * tw) { // south boundary, cy = +1
          const int f = e - 6 * th;
          bx = f / 3; by = 0;
          const int kk = f - 3 * bx;
          i = kk == 0 ? 2 : (kk == 1 ? 5 : 6);
        } else {                          // north boundary, cy = -1
          const int f = e - 6 * th - 3 * tw;
          bx = f / 3; by = th - 1;
          const int kk = f - 3 * bx;
          i = kk == 0 ? 4 : (kk == 1 ? 7 : 8);
        }
        const int sxl = bx - cx(i), syl = by - cy(i);
        if (sxl >= 0 && sxl < tw && syl >= 0 && syl < th) continue;  // inside the tile
        const int nbx = sxl < 0 ? 0 : (sxl >= tw ? 2 : 1);
        const int nby = syl < 0 ? 0 : (syl >= th ? 2 : 1);
        const Nb nb = s_nb[nby][nbx];
        const int bf = (by + 1) * RX + bx + 1;  // the consuming node's cell
        float v;
        if (nb.id < 0) {
          // beyond a wall: anti-bounce-back on the consuming node's own population opp(i)
          const float vw = nby == 0 ? vw_b : vw_t;
          v = h_wall(i, sm[slot(opp(i), bf)], vw);
        } else {
          const int olx = nbx == 0 ? nb.w - 1 : (nbx == 2 ? 0 : sxl);
          const int oly = nby == 0 ? nb.h - 1 : (nby == 2 ? 0 : syl);
          v = __ldcg(exp_all + (size_t)nb.id * pstride + (i - 1) * T::PMAX +
                     perim_slot(olx, oly, nb.w, nb.h));
        }
        // where the streaming of the consuming node reads direction i
        sm[SW ? (opp(i) - 1) * T::PLANE + bf : (i - 1) * T::PLANE + (syl + 1) * RX + sxl + 1] = v;
      }
    }
    __syncthreads();
    // the registers still hold the state the decision was about
    if (it > 0 && s_done) return 1;
    // 4b. stream: every source is now in shared memory
    float num = 0.0f, den = 0.0f;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int o0 = 2 * p * T::ROWS, o1 = (2 * p + 1) * T::ROWS;
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        const int off = SW ? (opp(i) - 1) * T::PLANE + at0 : (i - 1) * T::PLANE + at0 - cy(i) * RX - cx(i);
        h[p][i - 1] = make_float2(sm[off + o0 * RX], sm[off + o1 * RX]);
      }
      const float2 d = __fadd2_rn(h_varphi2(h_sum8x2(h[p])), neg2(vold[p]));
      if (valid[2 * p]) {
        num = __fmaf_rn(d.x, d.x, num);
        den = __fmaf_rn(vold[p].x, vold[p].x, den);
      }
      if (valid[2 * p + 1]) {
        num = __fmaf_rn(d.y, d.y, num);
        den = __fmaf_rn(vold[p].y, vold[p].y, den);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      num += __shfl_xor_sync(0xffffffffu, num, o);
      den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    // reduced by warp 0 inside the next grid barrier
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = make_float2(num, den);
    ++it;
    return 0;
  };
  for (;;) {
    int r = sub_iteration(std::false_type{});
    if (r == 2) return;
    if (r == 1) break;
    r = sub_iteration(std::true_type{});
    if (r == 2) return;
    if (r == 1) break;
  }

  // the registers hold the final state: write it back in place
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    if (!valid[s]) continue;
    const int g = (ty0 + ly0 + s * T::ROWS) * nx + tx0 + lx;
#pragma unroll
    for (int i = 0; i < 8; ++i) hsrc[i * N + g] = (s & 1) ? h[s >> 1][i].y : h[s >> 1][i].x;
  }
  if (tile == 0 && (int)threadIdx.x == dwarp * 32) {
    ctl->iter = it;
    ctl->rel = (double)rel;
    ctl->converged = conv;
    ctl->done = 1;
  }
}

template <int TY, bool CONV>
__global__ void __launch_bounds__(Tile<TY>::THREADS, Tile<TY>::MIN_BLOCKS)
    k_poisson_resident(KParams k, ResidentGeom rg, float* __restrict__ hbuf,
                       const float2* __restrict__ aq, float* __restrict__ exports,
                       float2* __restrict__ rpartials, Ctl* ctl) {
  resident_loop<TY, CONV>(k, rg, hbuf, aq, exports, rpartials, ctl, blockIdx.x, gridDim.x);
}

// Several simulations in one cooperative launch, all tiled 64 x TY: CTA b runs tile
// work[b].y of simulation work[b].x.  Simulations exchange nothing, so each synchronises
// only its own tiles (its own barrier counter and partial sums) and stops at its own
// sub-iteration count.
template <int TY>
__global__ void __launch_bounds__(Tile<TY>::THREADS, Tile<TY>::MIN_BLOCKS)
    k_poisson_resident_batch(const ResidentSlot* __restrict__ slots,
                             const int2* __restrict__ work) {
  const int2 w = work[blockIdx.x];
  const ResidentSlot& S = slots[w.x];
  resident_loop<TY, false>(S.k, S.rg, S.h, S.aq, S.exports, S.rpartials, S.ctl, w.y,
                    S.rg.ntx * S.rg.nty);
}

// ---------------------------------------------------------------------------------------
// Two sub-iterations per exchange.  The same arithmetic per node as resident_loop, but a
// CTA advances its tile by two sub-iterations between grid barriers: it imports a
// two-node-wide ring of its neighbours' post-stream state, collides tile and ring in the
// first sub-iteration (streaming into the tile and the ring's inner layer), collides tile
// and inner layer in the second (swapped layout, so no CTA barrier separates the first
// streaming from the second collision), then exports its own two-node-wide band.  The
// stopping rule is applied to both sub-iterations, in order, once every tile's sums are
// in (after the next cycle's first collision, which is dropped if the loop stops); when
// the first one already ends the loop, the state it produced is restored from tensor
// memory (TMEM), where every thread parks its four nodes' populations after the first
// sub-iteration.
// Every CTA reaches the same decisions and each state is the one resident_loop produces,
// bit for bit.  Half the grid barriers and halo round trips of resident_loop.
// ---------------------------------------------------------------------------------------
namespace {

constexpr int PXF = TXR + 4;  // frame row: the tile row plus two ring nodes each side

__host__ __device__ constexpr int pow2_at_least(int v) {
  return v <= 32 ? 32 : (v <= 64 ? 64 : (v <= 128 ? 128 : (v <= 256 ? 256 : 512)));
}

template <int TY>
struct Tile2 {
  static_assert(TY % 8 == 0 && TY >= 24 && TY <= 64, "two-step tiles: 24 to 64 rows");
  static constexpr int PY = TY + 4;
  static constexpr int PLANE = PY * PXF;           // one direction over tile and ring
  static constexpr int THREADS = TXR * TY / NPT;
  static constexpr int ROWS = TY / NPT;
  static constexpr int NR = 4 * PXF + 4 * TY;      // ring nodes of a full tile
  static constexpr int PMAX = 4 * TXR + 4 * TY;    // band slots (a full tile uses 16 fewer)
  static constexpr int TCOLS = pow2_at_least((THREADS / 128) * 32);  // TMEM columns
  static_assert(THREADS >= NR, "one ring node per thread at most");
  static_assert(THREADS % 128 == 0, "whole warp quarters for TMEM");
};

// 16-byte global -> shared copy that bypasses L1 (the source was written by another SM
// in this launch), completed by cp_async_wait_all in the issuing thread.  Both addresses
// 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src_gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  const size_t g = __cvta_generic_to_global(src_gmem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Slot of node (x, y) in the two-node-wide export band of a w x h tile (w, h >= 4): the
// two bottom rows, the two top rows, then the two left and two right columns between.
__device__ __forceinline__ int band_slot(int x, int y, int w, int h) {
  if (y < 2) return y * w + x;
  if (y >= h - 2) return 2 * w + (y - (h - 2)) * w + x;
  if (x < 2) return 4 * w + (y - 2) * 2 + x;
  return 4 * w + 2 * (h - 4) + (y - 2) * 2 + (x - (w - 2));
}

// Inverse of band_slot: the node of band slot sl of a w x h tile.
__device__ __forceinline__ void band_coords(int sl, int w, int h, int& x, int& y) {
  if (sl < 2 * w) {
    y = sl < w ? 0 : 1;
    x = sl - y * w;
    return;
  }
  sl -= 2 * w;
  if (sl < 2 * w) {
    y = h - 2 + (sl < w ? 0 : 1);
    x = sl - (sl < w ? 0 : w);
    return;
  }
  sl -= 2 * w;
  if (sl < 2 * (h - 4)) {
    y = 2 + (sl >> 1);
    x = sl & 1;
    return;
  }
  sl -= 2 * (h - 4);
  y = 2 + (sl >> 1);
  x = w - 2 + (sl & 1);
}

// Tile-relative coordinates of ring node r of a tw x th tile: two rows below, two rows
// above (each tw + 4 wide), then two columns left and two right (th high).
__device__ __forceinline__ void ring_coords(int r, int tw, int th, int& x, int& y) {
  const int w4 = tw + 4;
  if (r < 2 * w4) {
    y = r < w4 ? -2 : -1;
    x = r - (r < w4 ? 0 : w4) - 2;
    return;
  }
  r -= 2 * w4;
  if (r < 2 * w4) {
    y = r < w4 ? th : th + 1;
    x = r - (r < w4 ? 0 : w4) - 2;
    return;
  }
  r -= 2 * w4;
  if (r < 2 * th) {
    y = r >> 1;
    x = -2 + (r & 1);
    return;
  }
  r -= 2 * th;
  y = r >> 1;
  x = tw + (r & 1);
}

__device__ __forceinline__ void tmem_store32(uint32_t taddr, const float2 (&h)[2][8]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, "
      "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, "
      "%27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "f"(h[0][0].x), "f"(h[0][0].y), "f"(h[0][1].x), "f"(h[0][1].y), "f"(h[0][2].x),
      "f"(h[0][2].y), "f"(h[0][3].x), "f"(h[0][3].y), "f"(h[0][4].x), "f"(h[0][4].y),
      "f"(h[0][5].x), "f"(h[0][5].y), "f"(h[0][6].x), "f"(h[0][6].y), "f"(h[0][7].x),
      "f"(h[0][7].y), "f"(h[1][0].x), "f"(h[1][0].y), "f"(h[1][1].x), "f"(h[1][1].y),
      "f"(h[1][2].x), "f"(h[1][2].y), "f"(h[1][3].x), "f"(h[1][3].y), "f"(h[1][4].x),
      "f"(h[1][4].y), "f"(h[1][5].x), "f"(h[1][5].y), "f"(h[1][6].x), "f"(h[1][6].y),
      "f"(h[1][7].x), "f"(h[1][7].y)
      : "memory");
}

__device__ __forceinline__ void tmem_load32(uint32_t taddr, float2 (&h)[2][8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=f"(h[0][0].x), "=f"(h[0][0].y), "=f"(h[0][1].x), "=f"(h[0][1].y), "=f"(h[0][2].x),
        "=f"(h[0][2].y), "=f"(h[0][3].x), "=f"(h[0][3].y), "=f"(h[0][4].x), "=f"(h[0][4].y),
        "=f"(h[0][5].x), "=f"(h[0][5].y), "=f"(h[0][6].x), "=f"(h[0][6].y), "=f"(h[0][7].x),
        "=f"(h[0][7].y), "=f"(h[1][0].x), "=f"(h[1][0].y), "=f"(h[1][1].x), "=f"(h[1][1].y),
        "=f"(h[1][2].x), "=f"(h[1][2].y), "=f"(h[1][3].x), "=f"(h[1][3].y), "=f"(h[1][4].x),
        "=f"(h[1][4].y), "=f"(h[1][5].x), "=f"(h[1][5].y), "=f"(h[1][6].x), "=f"(h[1][6].y),
        "=f"(h[1][7].x), "=f"(h[1][7].y)
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Post-stream population i of the node at frame index f: the post-collision population
// of the node behind it, or the anti-bounce-back rule when that node lies beyond a wall
// (bw / tw_: the consuming node is on the bottom / top lattice row of a walled lattice).
template <int PLANE>
__device__ __forceinline__ float gather(const float* sm, int i, int f, bool bw, bool tw_,
                                        float vw_b, float vw_t) {
  if (cy(i) > 0 && bw) return h_wall(i, sm[(opp(i) - 1) * PLANE + f], vw_b);
  if (cy(i) < 0 && tw_) return h_wall(i, sm[(opp(i) - 1) * PLANE + f], vw_t);
  return sm[(i - 1) * PLANE + f - cy(i) * PXF - cx(i)];
}

// The same population when the post-collision populations were written in the swapped
// layout of a second sub-iteration (direction i of the node at f leaves in slot opp(i) of
// the cell at f + c_i): it is slot opp(i) of the consuming node's own cell, and a node
// next to a wall finds its own post-collision population opp(i) in slot i of the cell
// beyond the wall.
template <int PLANE>
__device__ __forceinline__ float gather_swapped(const float* sm, int i, int f, bool bw,
                                                bool tw_, float vw_b, float vw_t) {
  if (cy(i) > 0 && bw) return h_wall(i, sm[(i - 1) * PLANE + f - cy(i) * PXF - cx(i)], vw_b);
  if (cy(i) < 0 && tw_) return h_wall(i, sm[(i - 1) * PLANE + f - cy(i) * PXF - cx(i)], vw_t);
  return sm[(opp(i) - 1) * PLANE + f];
}

}  // namespace

template <int TY, bool CONV>
__device__ __forceinline__ void resident_loop2(const KParams& k, const ResidentGeom& rg,
                                               float* __restrict__ hbuf,
                                               const float2* __restrict__ aq,
                                               float* __restrict__ exports,
                                               float2* __restrict__ rpartials, Ctl* ctl,
                                               const int tile, const int ntiles) {
  using T = Tile2<TY>;
  // shared memory: [8][PY][PXF] post-collision populations over tile and ring, [PY][PXF]
  // a, [PY][PXF] q, then [8][NR] ring state (also the export staging area)
  extern __shared__ float sm[];
  __shared__ float2 s_w1[T::THREADS / 32], s_w2[T::THREADS / 32];  // warp sums per sub-iteration
  __shared__ int s_done, s_ok;
  __shared__ float4 s_pp[160];  // the deciding warp's copy of the tiles' sums
  __shared__ uint32_t s_taddr;
  __shared__ Nb s_nb[3][3];

  const int nx = k.nx, ny = k.ny;
  const size_t N = (size_t)k.N;
  const int tcol = tile % rg.ntx, trow = tile / rg.ntx;
  const int tx0 = tcol * TXR, ty0 = trow * TY;
  const int tw = min(TXR, nx - tx0), th = min(TY, ny - ty0);
  float* ca = sm + 8 * T::PLANE;
  float* cq = ca + T::PLANE;
  float* ring = cq + T::PLANE;
  // the loop control's fields this solve reads but no CTA of it writes come through the
  // read-only path: every warp of every CTA asks for the same few words at once, which
  // L1 merges per SM instead of sending each request to one L2 slice
  const int parity = __ldg(&ctl->parity);
  float* __restrict__ hsrc = hbuf + (size_t)parity * NH * N;
  // my tile nodes: column lx, rows ly0 + s ROWS
  const int lx = threadIdx.x & (TXR - 1);
  const int ly0 = threadIdx.x >> 6;
  const int at0 = (ly0 + 2) * PXF + lx + 2;   // frame index of node 0
  const int nrows = lx < tw ? th : 0;
  // per node: inside the lattice; on the bottom / top lattice row next to a wall
  auto valid = [&](int s) { return ly0 + s * T::ROWS < nrows; };
  auto bw = [&](int s) { return k.walls && ty0 + ly0 + s * T::ROWS == 0; };
  auto tw_ = [&](int s) { return k.walls && ty0 + ly0 + s * T::ROWS == ny - 1; };
  // every load of the thread's four nodes is issued at entry, before the tensor-memory
  // allocation, the neighbour table and the ring import, and before any value is used (a
  // node outside the lattice loads node 0 and then starts from zero): their round trip to
  // memory overlaps the rest of the set-up
  float2 h[2][8];
  float2 tc[NPT];
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    const int g = (int)EHD_IDX(k, valid(s) ? (ty0 + ly0 + s * T::ROWS) * nx + tx0 + lx : 0, N);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float v = hsrc[i * N + g];
      if (s & 1)
        h[s >> 1][i].y = v;
      else
        h[s >> 1][i].x = v;
    }
    tc[s] = aq[g];
  }
  const float qshift = k.neutralize ? __ldg(&ctl->mean_q) : 0.0f;
  const float vw_b = __ldg(&ctl->vw_b), vw_t = __ldg(&ctl->vw_t);
  const double tol = ctl->tol;
  // a non-finite phi or q (flagged by the moments pass) stops the loop after one
  // sub-iteration, not converged
  const bool bad_state = __ldg(&ctl->nonfinite) != 0;
  const int min_iter = bad_state ? 1 : ctl->min_iter, max_iter = bad_state ? 1 : ctl->max_iter,
            fixed = bad_state ? 0 : ctl->fixed_iter;
  const float om = k.omega_h;
  constexpr int pstride = 8 * T::PMAX;
  const int warp = threadIdx.x >> 5;
  constexpr int dwarp = T::THREADS / 32 - 1;

  // TMEM for the parked state: warp w uses lanes 32 (w mod 4) .. + 31, columns 32 (w / 4)
  if (warp == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_taddr);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
                 "n"(T::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }

  if (threadIdx.x < 9) {
    const int dx = (int)threadIdx.x % 3 - 1, dy = (int)threadIdx.x / 3 - 1;
    const int c = (tcol + dx + rg.ntx) % rg.ntx;
    int r = trow + dy;
    Nb nb;
    if (r < 0 || r >= rg.nty) {
      if (k.walls) {
        nb.id = -1;
        nb.w = nb.h = 0;
        s_nb[dy + 1][dx + 1] = nb;
        r = -1;
      } else {
        r = (r + rg.nty) % rg.nty;
      }
    }
    if (r >= 0) {
      nb.id = r * rg.ntx + c;
      nb.w = min(TXR, nx - c * TXR);
      nb.h = min(TY, ny - r * TY);
      s_nb[dy + 1][dx + 1] = nb;
    }
  }
  if (threadIdx.x == 0) s_done = 0;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = s_taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));

  // my ring node (thread r < number of ring nodes): frame index, flags, import source
  const int nring = 4 * (tw + 4) + 4 * th;
  int rf = 0, rsrc = 0;  // frame index; offset of my ring node in its tile's export band
  bool rexist = false, rlayer1 = false, rbw = false, rtw = false;
  if ((int)threadIdx.x < nring) {
    int x, y;
    ring_coords(threadIdx.x, tw, th, x, y);
    rf = (y + 2) * PXF + x + 2;
    const int nbx = x < 0 ? 0 : (x >= tw ? 2 : 1);
    const int nby = y < 0 ? 0 : (y >= th ? 2 : 1);
    const Nb nb = s_nb[nby][nbx];
    rexist = nb.id >= 0;
    if (rexist) {
      const int olx = x < 0 ? nb.w + x : (x >= tw ? x - tw : x);
      const int oly = y < 0 ? nb.h + y : (y >= th ? y - th : y);
      rsrc = nb.id * pstride + band_slot(olx, oly, nb.w, nb.h);
      rlayer1 = ((y == -1 || y == th) && x >= -1 && x <= tw) ||
                ((x == -1 || x == tw) && y >= 0 && y < th);
      const int gy = ty0 + y;
      rbw = k.walls && gy == 0;
      rtw = k.walls && gy == ny - 1;
      // first import: the lattice's own post-stream state; coefficients once per solve
      const int gx = (tx0 + x + nx) % nx;
      const int g = (int)EHD_IDX(k, ((gy + ny) % ny) * nx + gx, N);
#pragma unroll
      for (int i = 0; i < 8; ++i) ring[i * T::NR + threadIdx.x] = hsrc[i * N + g];
      const float2 c = aq[g];
      ca[rf] = c.x;
      const float qn = __fsub_rn(c.y, qshift);
      cq[rf] = CONV ? __fmul_rn(qn, k.inv_chi) : qn;
    }
  }

  // my tile nodes: the state loaded at entry sits in registers (two packed pairs), the
  // coefficients go to the frame.  Nodes outside the lattice (partial tiles) compute with
  // their pair but write nothing to shared memory: their cells may be ring nodes of this
  // tile.
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    if (valid(s)) {  // a node outside the lattice may sit on a ring node's cell
      float q = __fsub_rn(tc[s].y, qshift);
      if (CONV) q = __fmul_rn(q, k.inv_chi);
      ca[at0 + s * T::ROWS * PXF] = tc[s].x;
      cq[at0 + s * T::ROWS * PXF] = q;
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (s & 1)
          h[s >> 1][i].y = 0.0f;
        else
          h[s >> 1][i].x = 0.0f;
      }
    }
  }
  __syncthreads();

  unsigned target = 0;
  int cyc = 0, it = 0, conv = 0;
  float rel = 0.0f;
  int done = 0;
  for (;;) {
    // ---- after the previous cycle's grid barrier: the deciding warp starts copying that
    // cycle's per-tile sums and the ring threads import the ring for this one.  Every
    // thread then collides, and the deciding warp applies the rule to the previous
    // cycle's two sub-iterations; the collision is dropped if the rule stopped the loop
    // (it writes shared memory only). ----
    if (cyc > 0) {
      if (warp == dwarp) {
        // the previous cycle's sums of every tile (num and den of its two sub-iterations),
        // copied while the warp collides its nodes; lane l takes tiles l, l + 32, ...
        const float4* pp = reinterpret_cast<const float4*>(rpartials) + (size_t)((cyc - 1) & 1) * ntiles;
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int j = 0; j < 5; ++j)
          if (lane + 32 * j < ntiles) cp_async16(&s_pp[lane + 32 * j], pp + lane + 32 * j);
      }
      if (rexist) {  // the thread's own ring slot: no CTA barrier needed before its collision
        const float* src = exports + (size_t)((cyc - 1) & 1) * ntiles * pstride + rsrc;
#pragma unroll
        for (int i = 0; i < 8; ++i) ring[i * T::NR + threadIdx.x] = __ldcg(src + i * T::PMAX);
      }
    }
    // ---- sub-iteration 1: collide tile and ring, stream into tile and inner ring ----
    float2 vold[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int o0 = 2 * p * T::ROWS * PXF, o1 = (2 * p + 1) * T::ROWS * PXF;
      const float2 varphi = h_varphi2(h_sum8x2(h[p]));
      vold[p] = varphi;
      float2 m1x, m1y;
      h_moment1x2(h[p], m1x, m1y);
      const float2 a = make_float2(ca[at0 + o0], ca[at0 + o1]);
      const float2 qs = __fmul2_rn(f2(0.125f), make_float2(cq[at0 + o0], cq[at0 + o1]));
      float2 hs[8];
      if constexpr (CONV)
        h_star_conv8x2(h[p], a, varphi, qs, hs);
      else
        h_star8x2(h[p], om, varphi, a, m1x, m1y, qs, hs);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (valid(2 * p)) sm[i * T::PLANE + at0 + o0] = hs[i].x;
        if (valid(2 * p + 1)) sm[i * T::PLANE + at0 + o1] = hs[i].y;
      }
    }
    if (cyc > 0 && warp == dwarp) {
      // the rule, applied to the previous cycle's two sub-iterations in order
      cp_async_wait_all();
      const float4* pp = reinterpret_cast<const float4*>(rpartials) + (size_t)((cyc - 1) & 1) * ntiles;
      const int lane = threadIdx.x & 31;
      float a1 = 0.0f, b1 = 0.0f, a2 = 0.0f, b2 = 0.0f;
#pragma unroll
      for (int j = 0; j < 5; ++j) {  // absent tiles add +0: exact for these non-negative sums
        const float4 v = lane + 32 * j < ntiles ? s_pp[lane + 32 * j] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        a1 += v.x;
        b1 += v.y;
        a2 += v.z;
        b2 += v.w;
      }
      for (int t = lane + 160; t < ntiles; t += 32) {
        const float4 v = __ldcg(pp + t);
        a1 += v.x;
        b1 += v.y;
        a2 += v.z;
        b2 += v.w;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        b1 += __shfl_xor_sync(0xffffffffu, b1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        b2 += __shfl_xor_sync(0xffffffffu, b2, o);
      }
      if (lane == 0) {
        int d = 0;
        for (int u = 0; u < 2 && !d; ++u) {
          const int st = 2 * (cyc - 1) + 1 + u;
          const float sa = u ? a2 : a1, sb = u ? b2 : b1;
          float r;
          if (sa == 0.0f && sb == 0.0f)
            r = 0.0f;
          else if (sb == 0.0f)
            r = __int_as_float(0x7f800000);
          else
            r = sqrtf(sa / sb);
          bool dn;
          int cv;
          if (fixed > 0) {
            dn = st >= fixed;
            cv = 1;
          } else {
            cv = (st >= min_iter) && ((double)r < tol);
            dn = cv || st >= max_iter;
          }
          rel = r;
          conv = cv;
          it = st;
          if (dn) d = u + 1;
        }
        s_done = d;
      }
    }
    if (rexist) {
      float hr[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) hr[i] = ring[i * T::NR + threadIdx.x];
      const float varphi = h_varphi(h_sum8(hr));
      float m1x, m1y;
      h_moment1(hr, m1x, m1y);
      const float qs = 0.125f * cq[rf];
      const float a = ca[rf];
#pragma unroll
      for (int i = 1; i < 9; ++i)
        sm[(i - 1) * T::PLANE + rf] = CONV ? h_star_conv(i, hr[i - 1], a, varphi, qs)
                                           : h_star(i, hr[i - 1], om, varphi, a, m1x, m1y, qs);
    }
    __syncthreads();  // post-collision populations and the rule's verdict visible
    done = s_done;
    if (done) break;
    float num = 0.0f, den = 0.0f;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int f0 = at0 + 2 * p * T::ROWS * PXF, f1 = at0 + (2 * p + 1) * T::ROWS * PXF;
      if (bw(2 * p) || tw_(2 * p) || bw(2 * p + 1) || tw_(2 * p + 1)) {
#pragma unroll
        for (int i = 1; i < 9; ++i)
          h[p][i - 1] = make_float2(
              gather<T::PLANE>(sm, i, f0, bw(2 * p), tw_(2 * p), vw_b, vw_t),
              gather<T::PLANE>(sm, i, f1, bw(2 * p + 1), tw_(2 * p + 1), vw_b, vw_t));
      } else {
#pragma unroll
        for (int i = 1; i < 9; ++i) {
          const int off = (i - 1) * T::PLANE - cy(i) * PXF - cx(i);
          h[p][i - 1] = make_float2(sm[off + f0], sm[off + f1]);
        }
      }
      const float2 d = __fadd2_rn(h_varphi2(h_sum8x2(h[p])), neg2(vold[p]));
      if (valid(2 * p)) {
        num = __fmaf_rn(d.x, d.x, num);
        den = __fmaf_rn(vold[p].x, vold[p].x, den);
      }
      if (valid(2 * p + 1)) {
        num = __fmaf_rn(d.y, d.y, num);
        den = __fmaf_rn(vold[p].y, vold[p].y, den);
      }
    }
    if (rlayer1) {
#pragma unroll
      for (int i = 1; i < 9; ++i)
        ring[(i - 1) * T::NR + threadIdx.x] = gather<T::PLANE>(sm, i, rf, rbw, rtw, vw_b, vw_t);
    }
    // park the state after the first sub-iteration in TMEM (restored if the rule stops
    // the loop there)
    tmem_store32(taddr, h);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      num += __shfl_xor_sync(0xffffffffu, num, o);
      den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if ((threadIdx.x & 31) == 0) s_w1[warp] = make_float2(num, den);
    // ---- sub-iteration 2: collide tile and inner ring, stream into the tile.  Direction
    // i of the node at x goes to slot opp(i) of the cell at x + c_i, the one slot the
    // thread of node x itself read in the first streaming, so no thread can still be
    // reading a slot this collision overwrites and no CTA barrier is needed before it. ----
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int o0 = 2 * p * T::ROWS * PXF, o1 = (2 * p + 1) * T::ROWS * PXF;
      const float2 varphi = h_varphi2(h_sum8x2(h[p]));
      vold[p] = varphi;
      float2 m1x, m1y;
      h_moment1x2(h[p], m1x, m1y);
      const float2 a = make_float2(ca[at0 + o0], ca[at0 + o1]);
      const float2 qs = __fmul2_rn(f2(0.125f), make_float2(cq[at0 + o0], cq[at0 + o1]));
      float2 hs[8];
      if constexpr (CONV)
        h_star_conv8x2(h[p], a, varphi, qs, hs);
      else
        h_star8x2(h[p], om, varphi, a, m1x, m1y, qs, hs);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int sw = (opp(i + 1) - 1) * T::PLANE + cy(i + 1) * PXF + cx(i + 1);
        if (valid(2 * p)) sm[sw + at0 + o0] = hs[i].x;
        if (valid(2 * p + 1)) sm[sw + at0 + o1] = hs[i].y;
      }
    }
    if (rlayer1) {
      float hr[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) hr[i] = ring[i * T::NR + threadIdx.x];
      const float varphi = h_varphi(h_sum8(hr));
      float m1x, m1y;
      h_moment1(hr, m1x, m1y);
      const float qs = 0.125f * cq[rf];
      const float a = ca[rf];
#pragma unroll
      for (int i = 1; i < 9; ++i)
        sm[(opp(i) - 1) * T::PLANE + cy(i) * PXF + cx(i) + rf] =
            CONV ? h_star_conv(i, hr[i - 1], a, varphi, qs)
                 : h_star(i, hr[i - 1], om, varphi, a, m1x, m1y, qs);
    }
    __syncthreads();
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    num = 0.0f;
    den = 0.0f;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int f0 = at0 + 2 * p * T::ROWS * PXF, f1 = at0 + (2 * p + 1) * T::ROWS * PXF;
      if (bw(2 * p) || tw_(2 * p) || bw(2 * p + 1) || tw_(2 * p + 1)) {
#pragma unroll
        for (int i = 1; i < 9; ++i)
          h[p][i - 1] = make_float2(
              gather_swapped<T::PLANE>(sm, i, f0, bw(2 * p), tw_(2 * p), vw_b, vw_t),
              gather_swapped<T::PLANE>(sm, i, f1, bw(2 * p + 1), tw_(2 * p + 1), vw_b, vw_t));
      } else {
#pragma unroll
        for (int i = 1; i < 9; ++i) {
          const int off = (opp(i) - 1) * T::PLANE;
          h[p][i - 1] = make_float2(sm[off + f0], sm[off + f1]);
        }
      }
      const float2 d = __fadd2_rn(h_varphi2(h_sum8x2(h[p])), neg2(vold[p]));
      if (valid(2 * p)) {
        num = __fmaf_rn(d.x, d.x, num);
        den = __fmaf_rn(vold[p].x, vold[p].x, den);
      }
      if (valid(2 * p + 1)) {
        num = __fmaf_rn(d.y, d.y, num);
        den = __fmaf_rn(vold[p].y, vold[p].y, den);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      num += __shfl_xor_sync(0xffffffffu, num, o);
      den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if ((threadIdx.x & 31) == 0) s_w2[warp] = make_float2(num, den);
    {
      // export band: the new state of the tile's two outer rows and columns, gathered
      // again from the second sub-iteration's post-collision populations (still in
      // shared memory, swapped layout), one band slot per thread, coalesced
      float* exp_cur = exports + (size_t)(cyc & 1) * ntiles * pstride + (size_t)tile * pstride;
      const int nslots = 4 * tw + 4 * th - 16;
      for (int sl = threadIdx.x; sl < nslots; sl += T::THREADS) {
        int x, y;
        band_coords(sl, tw, th, x, y);
        const int f = (y + 2) * PXF + x + 2;
        const bool b = k.walls && ty0 + y == 0, t = k.walls && ty0 + y == ny - 1;
#pragma unroll
        for (int i = 1; i < 9; ++i)
          exp_cur[(i - 1) * T::PMAX + sl] = gather_swapped<T::PLANE>(sm, i, f, b, t, vw_b, vw_t);
      }
    }
    // ---- grid barrier.  Warp 0 reduces both sub-iterations' warp sums (warps in a fixed
    // order) and its lane 0 publishes them, then releases the CTA's band writes (ordered
    // before it by the CTA barrier) and waits, within a time limit, for every tile. ----
    __syncthreads();
    target += ntiles;
    if (threadIdx.x < 32) {
      constexpr int nwarps = T::THREADS / 32;
      const bool in = (int)threadIdx.x < nwarps;
      float2 v1 = in ? s_w1[threadIdx.x] : make_float2(0.0f, 0.0f);
      float2 v2 = in ? s_w2[threadIdx.x] : make_float2(0.0f, 0.0f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v1.x += __shfl_xor_sync(0xffffffffu, v1.x, o);
        v1.y += __shfl_xor_sync(0xffffffffu, v1.y, o);
        v2.x += __shfl_xor_sync(0xffffffffu, v2.x, o);
        v2.y += __shfl_xor_sync(0xffffffffu, v2.y, o);
      }
      if (threadIdx.x == 0) {
        reinterpret_cast<float4*>(rpartials)[(size_t)(cyc & 1) * ntiles + tile] =
            make_float4(v1.x, v1.y, v2.x, v2.y);
        int ok = 1;
        red_release_add(&ctl->bar_count, 1u);
        const unsigned long long t0 = global_ns();
        while ((int)(ld_acquire(&ctl->bar_count) - target) < 0) {
          if (global_ns() - t0 > BARRIER_TIMEOUT_NS) {
            atomicOr(&ctl->bar_error, 1);
            ok = 0;
            break;
          }
        }
        s_ok = ok;
      }
    }
    __syncthreads();  // every tile's band and sums visible (or the wait gave up)
    if (!s_ok) {
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_taddr),
                     "n"(T::TCOLS)
                     : "memory");
      }
      return;
    }
    ++cyc;
  }
  if (done == 1) tmem_load32(taddr, h);  // the loop stopped after the first sub-iteration

  // the registers hold the final state: write it back in place
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    if (!valid(s)) continue;
    const int g = (int)EHD_IDX(k, (ty0 + ly0 + s * T::ROWS) * nx + tx0 + lx, N);
#pragma unroll
    for (int i = 0; i < 8; ++i) hsrc[i * N + g] = (s & 1) ? h[s >> 1][i].y : h[s >> 1][i].x;
  }
  if (tile == 0 && (int)threadIdx.x == dwarp * 32) {
    ctl->iter = it;
    ctl->rel = (double)rel;
    ctl->converged = conv;
    ctl->done = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_taddr),
                 "n"(T::TCOLS)
                 : "memory");
  }
}

template <int TY, bool CONV>
__global__ void __launch_bounds__(Tile2<TY>::THREADS, 1)
    k_poisson_resident2(KParams k, ResidentGeom rg, float* __restrict__ hbuf,
                        const float2* __restrict__ aq, float* __restrict__ exports,
                        float2* __restrict__ rpartials, Ctl* ctl) {
  resident_loop2<TY, CONV>(k, rg, hbuf, aq, exports, rpartials, ctl, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------------------
// D sub-iterations per exchange, written for any D (used for D = 3: the loop above is a
// hand-scheduled D = 2 and measured 2 % faster than this form at D = 2, with the same
// bits).  Sub-iteration u (0-based) of a cycle collides the tile and the ring layers
// 1 .. D - u and streams into the tile and the layers 1 .. D - 1 - u, in the own layout
// for even u and the swapped layout for odd u; the states after sub-iterations 0 .. D - 2
// are parked in TMEM.  Every CTA reaches the same decisions and each state is the one
// resident_loop produces, bit for bit.
// ---------------------------------------------------------------------------------------
namespace {

// Compile-time shape of a 64 x TY tile with a D-node-wide ring.
template <int TY, int D>
struct TileD {
  static_assert(D == 2 || D == 3, "two or three sub-iterations per exchange");
  static_assert(TY % 8 == 0 && TY <= 64, "tile height: a multiple of 8 up to 64");
  static constexpr int PX = TXR + 2 * D;            // frame row: tile row and ring
  static constexpr int PY = TY + 2 * D;
  static constexpr int PLANE = PY * PX;             // one direction over tile and ring
  static constexpr int THREADS = TXR * TY / NPT;
  static constexpr int ROWS = TY / NPT;
  static constexpr int NR = 2 * D * PX + 2 * D * TY;     // ring nodes of a full tile
  static constexpr int PMAX = 2 * D * TXR + 2 * D * TY;  // band slots (a full tile: 4 D^2 fewer)
  static constexpr int SLOT_COLS = (THREADS / 128) * 32;  // TMEM columns of one parked state
  static constexpr int TCOLS = pow2_at_least((D - 1) * SLOT_COLS);
  static constexpr int SUMS4 = D == 2 ? 1 : 2;      // float4 of sums per tile and cycle
  static_assert(THREADS >= NR, "one ring node per thread at most");
  static_assert(THREADS % 128 == 0, "whole warp quarters for TMEM");
  static_assert((D - 1) * SLOT_COLS <= 512, "the parked states fit in tensor memory");
};

// Slot of node (x, y) in the D-node-wide export band of a w x h tile (w, h >= 2 D): the
// D bottom rows, the D top rows, then the D left and D right columns between.
template <int D>
__device__ __forceinline__ int band_slot_d(int x, int y, int w, int h) {
  if (y < D) return y * w + x;
  if (y >= h - D) return D * w + (y - (h - D)) * w + x;
  if (x < D) return 2 * D * w + (y - D) * D + x;
  return 2 * D * w + D * (h - 2 * D) + (y - D) * D + (x - (w - D));
}

// Inverse of band_slot: the node of band slot sl of a w x h tile.
template <int D>
__device__ __forceinline__ void band_coords_d(int sl, int w, int h, int& x, int& y) {
  if (sl < 2 * D * w) {
    int r = 0;
    while (sl >= w) {
      sl -= w;
      ++r;
    }
    y = r < D ? r : h - 2 * D + r;
    x = sl;
    return;
  }
  sl -= 2 * D * w;
  if (sl < D * (h - 2 * D)) {
    y = D + sl / D;
    x = sl % D;
    return;
  }
  sl -= D * (h - 2 * D);
  y = D + sl / D;
  x = w - D + sl % D;
}

// Tile-relative coordinates of ring node r of a tw x th tile: D rows below, D rows above
// (each tw + 2 D wide), then D columns left and D right (th high).
template <int D>
__device__ __forceinline__ void ring_coords_d(int r, int tw, int th, int& x, int& y) {
  const int wd = tw + 2 * D;
  if (r < 2 * D * wd) {
    int k = 0;
    while (r >= wd) {
      r -= wd;
      ++k;
    }
    y = k < D ? k - D : th + k - D;
    x = r - D;
    return;
  }
  r -= 2 * D * wd;
  if (r < D * th) {
    y = r / D;
    x = -D + r % D;
    return;
  }
  r -= D * th;
  y = r / D;
  x = tw + r % D;
}

// Post-stream population i of the node at frame index f of a frame PX wide.  Own layout
// (swapped = false): direction i of the node at x sits in slot i of its own cell, so the
// source is slot i of the cell at f - c_i; a node next to a wall (bw / tw_: on the bottom /
// top lattice row of a walled lattice) takes the anti-bounce-back rule on its own
// post-collision population opp(i).  Swapped layout: direction i of the node at x sits in
// slot opp(i) of the cell at x + c_i, so the source is slot opp(i) of the consuming node's
// own cell, and a node next to a wall finds its own population opp(i) in slot i of the cell
// beyond the wall.
template <int PLANE, int PX>
__device__ __forceinline__ float gather_d(const float* sm, int i, int f, bool bw, bool tw_,
                                          float vw_b, float vw_t, bool swapped) {
  const int own = (opp(i) - 1) * PLANE + f;                // own cell, slot opp(i)
  const int back = (i - 1) * PLANE + f - cy(i) * PX - cx(i);  // cell f - c_i, slot i
  if (cy(i) > 0 && bw) return h_wall(i, sm[swapped ? back : own], vw_b);
  if (cy(i) < 0 && tw_) return h_wall(i, sm[swapped ? back : own], vw_t);
  return sm[swapped ? own : back];
}

// Where direction i of the node at frame index f goes after its collision.
template <int PLANE, int PX>
__device__ __forceinline__ int scatter_at(int i, int f, bool swapped) {
  return swapped ? (opp(i) - 1) * PLANE + f + cy(i) * PX + cx(i) : (i - 1) * PLANE + f;
}

}  // namespace

template <int TY, int D>
__device__ __forceinline__ void resident_loopD(const KParams& k, const ResidentGeom& rg,
                                               float* __restrict__ hbuf,
                                               const float2* __restrict__ aq,
                                               float* __restrict__ exports,
                                               float2* __restrict__ rpartials, Ctl* ctl,
                                               const int tile, const int ntiles) {
  using T = TileD<TY, D>;
  constexpr int PX = T::PX;
  // shared memory: [8][PY][PX] post-collision populations over tile and ring, [PY][PX] a,
  // [PY][PX] q, then [8][NR] ring state (each ring node belongs to one thread)
  extern __shared__ __align__(16) float smd[];
  float* sm = smd;
  __shared__ float2 s_w[D][T::THREADS / 32];  // warp sums per sub-iteration
  __shared__ int s_done, s_ok;
  __shared__ float4 s_pp[160 * T::SUMS4];     // the deciding warp's copy of the tiles' sums
  __shared__ uint32_t s_taddr;
  __shared__ Nb s_nb[3][3];

  const int nx = k.nx, ny = k.ny;
  const size_t N = (size_t)k.N;
  const int tcol = tile % rg.ntx, trow = tile / rg.ntx;
  const int tx0 = tcol * TXR, ty0 = trow * TY;
  const int tw = min(TXR, nx - tx0), th = min(TY, ny - ty0);
  float* ca = sm + 8 * T::PLANE;
  float* cq = ca + T::PLANE;
  float* ring = cq + T::PLANE;
  // the loop control's fields this solve reads but no CTA of it writes come through the
  // read-only path: every warp of every CTA asks for the same few words at once, which
  // L1 merges per SM instead of sending each request to one L2 slice
  const int parity = __ldg(&ctl->parity);
  float* __restrict__ hsrc = hbuf + (size_t)parity * NH * N;
  const float qshift = k.neutralize ? __ldg(&ctl->mean_q) : 0.0f;
  const float vw_b = __ldg(&ctl->vw_b), vw_t = __ldg(&ctl->vw_t);
  const double tol = ctl->tol;
  // a non-finite phi or q (flagged by the moments pass) stops the loop after one
  // sub-iteration, not converged
  const bool bad_state = __ldg(&ctl->nonfinite) != 0;
  const int min_iter = bad_state ? 1 : ctl->min_iter, max_iter = bad_state ? 1 : ctl->max_iter,
            fixed = bad_state ? 0 : ctl->fixed_iter;
  const float om = k.omega_h;
  constexpr int pstride = 8 * T::PMAX;
  const int warp = threadIdx.x >> 5;
  constexpr int dwarp = T::THREADS / 32 - 1;

  // TMEM for the parked states: warp w uses lanes 32 (w mod 4) .. + 31 and, for the state
  // after sub-iteration u, columns u SLOT_COLS + 32 (w / 4) .. + 31
  if (warp == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_taddr);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
                 "n"(T::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }

  // my tile nodes: column lx, rows ly0 + s ROWS
  const int lx = threadIdx.x & (TXR - 1);
  const int ly0 = threadIdx.x >> 6;
  const int at0 = (ly0 + D) * PX + lx + D;  // frame index of node 0
  const int nrows = lx < tw ? th : 0;

  if (threadIdx.x < 9) {
    const int dx = (int)threadIdx.x % 3 - 1, dy = (int)threadIdx.x / 3 - 1;
    const int c = (tcol + dx + rg.ntx) % rg.ntx;
    int r = trow + dy;
    Nb nb;
    if (r < 0 || r >= rg.nty) {
      if (k.walls) {
        nb.id = -1;
        nb.w = nb.h = 0;
        s_nb[dy + 1][dx + 1] = nb;
        r = -1;
      } else {
        r = (r + rg.nty) % rg.nty;
      }
    }
    if (r >= 0) {
      nb.id = r * rg.ntx + c;
      nb.w = min(TXR, nx - c * TXR);
      nb.h = min(TY, ny - r * TY);
      s_nb[dy + 1][dx + 1] = nb;
    }
  }
  if (threadIdx.x == 0) s_done = 0;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = s_taddr + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));

  // my ring node (thread r < number of ring nodes): frame index, layer (1 next to the
  // tile .. D), wall rows, import source
  const int nring = 2 * D * (tw + 2 * D) + 2 * D * th;
  int rf = 0, rsrc = 0, rl = D + 1;  // rl > D: no ring node
  bool rbw = false, rtw = false;
  if ((int)threadIdx.x < nring) {
    int x, y;
    ring_coords_d<D>(threadIdx.x, tw, th, x, y);
    rf = (y + D) * PX + x + D;
    const int nbx = x < 0 ? 0 : (x >= tw ? 2 : 1);
    const int nby = y < 0 ? 0 : (y >= th ? 2 : 1);
    const Nb nb = s_nb[nby][nbx];
    if (nb.id >= 0) {
      const int olx = x < 0 ? nb.w + x : (x >= tw ? x - tw : x);
      const int oly = y < 0 ? nb.h + y : (y >= th ? y - th : y);
      rsrc = nb.id * pstride + band_slot_d<D>(olx, oly, nb.w, nb.h);
      const int lxd = x < 0 ? -x : (x >= tw ? x - tw + 1 : 0);
      const int lyd = y < 0 ? -y : (y >= th ? y - th + 1 : 0);
      rl = lxd > lyd ? lxd : lyd;
      const int gy = ty0 + y;
      rbw = k.walls && gy == 0;
      rtw = k.walls && gy == ny - 1;
      // first import: the lattice's own post-stream state; coefficients once per solve
      const int gx = (tx0 + x + nx) % nx;
      const int g = ((gy + ny) % ny) * nx + gx;
#pragma unroll
      for (int i = 0; i < 8; ++i) ring[i * T::NR + threadIdx.x] = hsrc[i * N + g];
      const float2 c = aq[g];
      ca[rf] = c.x;
      cq[rf] = c.y - qshift;
    }
  }

  // my tile nodes: state in registers (two packed pairs), coefficients in the frame.
  // Nodes outside the lattice (partial tiles) compute with their pair but write nothing
  // to shared memory: their cells may be ring nodes of this tile.
  float2 h[2][8];
  // per node: inside the lattice; on the bottom / top lattice row next to a wall
  auto valid = [&](int s) { return ly0 + s * T::ROWS < nrows; };
  auto bw = [&](int s) { return k.walls && ty0 + ly0 + s * T::ROWS == 0; };
  auto tw_ = [&](int s) { return k.walls && ty0 + ly0 + s * T::ROWS == ny - 1; };
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    const int ly = ly0 + s * T::ROWS;
    float v[8];
    float a = 0.0f, q = 0.0f;
    if (valid(s)) {
      const int g = (ty0 + ly) * nx + tx0 + lx;
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = hsrc[i * N + g];
      const float2 c = aq[g];
      a = c.x;
      q = c.y - qshift;
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = 0.0f;
    }
    if (valid(s)) {  // a node outside the lattice may sit on a ring node's cell
      ca[at0 + s * T::ROWS * PX] = a;
      cq[at0 + s * T::ROWS * PX] = q;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (s & 1)
        h[s >> 1][i].y = v[i];
      else
        h[s >> 1][i].x = v[i];
    }
  }
  __syncthreads();

  // collision of the tile nodes into the frame (own or swapped layout); varphi before it
  // kept in vold for the rule
  float2 vold[2];
  auto collide_tile = [&](bool swapped) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int o0 = 2 * p * T::ROWS * PX, o1 = (2 * p + 1) * T::ROWS * PX;
      const float2 varphi = h_varphi2(h_sum8x2(h[p]));
      vold[p] = varphi;
      float2 m1x, m1y;
      h_moment1x2(h[p], m1x, m1y);
      const float2 a = make_float2(ca[at0 + o0], ca[at0 + o1]);
      const float2 qs = __fmul2_rn(f2(0.125f), make_float2(cq[at0 + o0], cq[at0 + o1]));
      float2 hs[8];
      h_star8x2(h[p], om, varphi, a, m1x, m1y, qs, hs);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int d = scatter_at<T::PLANE, PX>(i + 1, at0, swapped);
        if (valid(2 * p)) sm[d + o0] = hs[i].x;
        if (valid(2 * p + 1)) sm[d + o1] = hs[i].y;
      }
    }
  };
  // collision of my ring node (its state in the ring array)
  auto collide_ring = [&](bool swapped) {
    float hr[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) hr[i] = ring[i * T::NR + threadIdx.x];
    const float varphi = h_varphi(h_sum8(hr));
    float m1x, m1y;
    h_moment1(hr, m1x, m1y);
    const float qs = 0.125f * cq[rf];
    const float a = ca[rf];
#pragma unroll
    for (int i = 1; i < 9; ++i)
      sm[scatter_at<T::PLANE, PX>(i, rf, swapped)] =
          h_star(i, hr[i - 1], om, varphi, a, m1x, m1y, qs);
  };
  // streaming into the tile nodes; returns the thread's (num, den) of the rule
  auto stream_tile = [&](bool swapped) {
    float num = 0.0f, den = 0.0f;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int f0 = at0 + 2 * p * T::ROWS * PX, f1 = at0 + (2 * p + 1) * T::ROWS * PX;
      if (bw(2 * p) || tw_(2 * p) || bw(2 * p + 1) || tw_(2 * p + 1)) {
#pragma unroll
        for (int i = 1; i < 9; ++i)
          h[p][i - 1] = make_float2(
              gather_d<T::PLANE, PX>(sm, i, f0, bw(2 * p), tw_(2 * p), vw_b, vw_t, swapped),
              gather_d<T::PLANE, PX>(sm, i, f1, bw(2 * p + 1), tw_(2 * p + 1), vw_b, vw_t,
                                   swapped));
      } else {
#pragma unroll
        for (int i = 1; i < 9; ++i) {
          const int off = swapped ? (opp(i) - 1) * T::PLANE : (i - 1) * T::PLANE - cy(i) * PX - cx(i);
          h[p][i - 1] = make_float2(sm[off + f0], sm[off + f1]);
        }
      }
      const float2 d = __fadd2_rn(h_varphi2(h_sum8x2(h[p])), neg2(vold[p]));
      if (valid(2 * p)) {
        num = __fmaf_rn(d.x, d.x, num);
        den = __fmaf_rn(vold[p].x, vold[p].x, den);
      }
      if (valid(2 * p + 1)) {
        num = __fmaf_rn(d.y, d.y, num);
        den = __fmaf_rn(vold[p].y, vold[p].y, den);
      }
    }
    return make_float2(num, den);
  };

  unsigned target = 0;
  int cyc = 0, it = 0, conv = 0;
  float rel = 0.0f;
  int done = 0;
  for (;;) {
    // ---- after the previous cycle's grid barrier: the deciding warp starts copying that
    // cycle's per-tile sums and the ring threads import the ring for this one.  Every
    // thread then collides, and the deciding warp applies the rule to the previous
    // cycle's D sub-iterations; the collision is dropped if the rule stopped the loop
    // (it writes shared memory only). ----
    if (cyc > 0) {
      if (warp == dwarp) {
        // the previous cycle's sums of every tile (num and den of its D sub-iterations),
        // copied while the warp collides its nodes; lane l takes tiles l, l + 32, ...
        const float4* pp = reinterpret_cast<const float4*>(rpartials) +
                           (size_t)((cyc - 1) & 1) * ntiles * T::SUMS4;
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int j = 0; j < 5; ++j) {
          const int t = lane + 32 * j;
          if (t < ntiles) {
#pragma unroll
            for (int e = 0; e < T::SUMS4; ++e)
              cp_async16(&s_pp[t * T::SUMS4 + e], pp + (size_t)t * T::SUMS4 + e);
          }
        }
      }
      if (rl <= D) {  // the thread's own ring slot: no CTA barrier needed before its collision
        const float* src = exports + (size_t)((cyc - 1) & 1) * ntiles * pstride + rsrc;
#pragma unroll
        for (int i = 0; i < 8; ++i) ring[i * T::NR + threadIdx.x] = __ldcg(src + i * T::PMAX);
      }
    }
    // ---- sub-iteration 0: own layout; collide tile and all ring layers ----
    collide_tile(false);
    if (cyc > 0 && warp == dwarp) {
      // the rule, applied to the previous cycle's sub-iterations in order
      cp_async_wait_all();
      const float4* pp = reinterpret_cast<const float4*>(rpartials) +
                         (size_t)((cyc - 1) & 1) * ntiles * T::SUMS4;
      const int lane = threadIdx.x & 31;
      float sa[D], sb[D];
#pragma unroll
      for (int u = 0; u < D; ++u) sa[u] = sb[u] = 0.0f;
      auto add = [&](int t, bool cached) {
        const float4 v0 = cached ? s_pp[t * T::SUMS4] : __ldcg(pp + (size_t)t * T::SUMS4);
        sa[0] += v0.x;
        sb[0] += v0.y;
        sa[1] += v0.z;
        sb[1] += v0.w;
        if constexpr (D == 3) {
          const float4 v1 = cached ? s_pp[t * T::SUMS4 + 1] : __ldcg(pp + (size_t)t * T::SUMS4 + 1);
          sa[2] += v1.x;
          sb[2] += v1.y;
        }
      };
      // lane l sums tiles l, l + 32, ... in that order
#pragma unroll
      for (int j = 0; j < 5; ++j)
        if (lane + 32 * j < ntiles) add(lane + 32 * j, true);
      for (int t = lane + 160; t < ntiles; t += 32) add(t, false);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int u = 0; u < D; ++u) {
          sa[u] += __shfl_xor_sync(0xffffffffu, sa[u], o);
          sb[u] += __shfl_xor_sync(0xffffffffu, sb[u], o);
        }
      }
      if (lane == 0) {
        int d = 0;
#pragma unroll
        for (int u = 0; u < D; ++u) {
          if (d) break;
          const int st = D * (cyc - 1) + 1 + u;
          float r;
          if (sa[u] == 0.0f && sb[u] == 0.0f)
            r = 0.0f;
          else if (sb[u] == 0.0f)
            r = __int_as_float(0x7f800000);
          else
            r = sqrtf(sa[u] / sb[u]);
          bool dn;
          int cv;
          if (fixed > 0) {
            dn = st >= fixed;
            cv = 1;
          } else {
            cv = (st >= min_iter) && ((double)r < tol);
            dn = cv || st >= max_iter;
          }
          rel = r;
          conv = cv;
          it = st;
          if (dn) d = u + 1;
        }
        s_done = d;
      }
    }
    if (rl <= D) collide_ring(false);
    __syncthreads();  // post-collision populations and the rule's verdict visible
    done = s_done;
    if (done) break;
    // ---- sub-iterations 0 .. D - 1: stream (layout of the collision), collide the next
    // with the other layout.  Sub-iteration u + 1 writes direction i of node x into a slot
    // that, in the streaming of sub-iteration u, only the thread of node x itself read, so
    // no CTA barrier is needed between a streaming and the next collision. ----
#pragma unroll
    for (int u = 0; u < D; ++u) {
      const bool sw = (u & 1) != 0;
      if (u > 0) {
        collide_tile(sw);
        if (rl <= D - u) collide_ring(sw);
        __syncthreads();  // post-collision populations visible
      }
      float2 ws = stream_tile(sw);
      if (rl <= D - 1 - u) {
#pragma unroll
        for (int i = 1; i < 9; ++i)
          ring[(i - 1) * T::NR + threadIdx.x] =
              gather_d<T::PLANE, PX>(sm, i, rf, rbw, rtw, vw_b, vw_t, sw);
      }
      // park the state after every sub-iteration but the last in TMEM (restored if the
      // rule stops the loop there)
      if (u < D - 1) tmem_store32(taddr + (uint32_t)(u * T::SLOT_COLS), h);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ws.x += __shfl_xor_sync(0xffffffffu, ws.x, o);
        ws.y += __shfl_xor_sync(0xffffffffu, ws.y, o);
      }
      if ((threadIdx.x & 31) == 0) s_w[u][warp] = ws;
    }
    {
      // export band: the new state of the tile's D outer rows and columns, gathered from
      // the last sub-iteration's post-collision populations (still in shared memory), one
      // band slot per thread, coalesced
      constexpr bool swl = ((D - 1) & 1) != 0;
      float* exp_cur = exports + (size_t)(cyc & 1) * ntiles * pstride + (size_t)tile * pstride;
      const int nslots = 2 * D * (tw + th) - 4 * D * D;
      for (int sl = threadIdx.x; sl < nslots; sl += T::THREADS) {
        int x, y;
        band_coords_d<D>(sl, tw, th, x, y);
        const int f = (y + D) * PX + x + D;
        const bool b = k.walls && ty0 + y == 0, t = k.walls && ty0 + y == ny - 1;
#pragma unroll
        for (int i = 1; i < 9; ++i)
          exp_cur[(i - 1) * T::PMAX + sl] = gather_d<T::PLANE, PX>(sm, i, f, b, t, vw_b, vw_t, swl);
      }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    // ---- grid barrier.  Warp 0 reduces the sub-iterations' warp sums (warps in a fixed
    // order) and its lane 0 publishes them, then releases the CTA's band writes (ordered
    // before it by the CTA barrier) and waits, within a time limit, for every tile. ----
    __syncthreads();
    target += ntiles;
    if (threadIdx.x < 32) {
      constexpr int nwarps = T::THREADS / 32;
      const bool in = (int)threadIdx.x < nwarps;
      float2 v[D];
#pragma unroll
      for (int u = 0; u < D; ++u) v[u] = in ? s_w[u][threadIdx.x] : make_float2(0.0f, 0.0f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int u = 0; u < D; ++u) {
          v[u].x += __shfl_xor_sync(0xffffffffu, v[u].x, o);
          v[u].y += __shfl_xor_sync(0xffffffffu, v[u].y, o);
        }
      }
      if (threadIdx.x == 0) {
        float4* pp = reinterpret_cast<float4*>(rpartials) +
                     ((size_t)(cyc & 1) * ntiles + tile) * T::SUMS4;
        pp[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        if constexpr (D == 3) pp[1] = make_float4(v[2].x, v[2].y, 0.0f, 0.0f);
        int ok = 1;
        red_release_add(&ctl->bar_count, 1u);
        const unsigned long long t0 = global_ns();
        while ((int)(ld_acquire(&ctl->bar_count) - target) < 0) {
          if (global_ns() - t0 > BARRIER_TIMEOUT_NS) {
            atomicOr(&ctl->bar_error, 1);
            ok = 0;
            break;
          }
        }
        s_ok = ok;
      }
    }
    __syncthreads();  // every tile's band and sums visible (or the wait gave up)
    if (!s_ok) {
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_taddr),
                     "n"(T::TCOLS)
                     : "memory");
      }
      return;
    }
    ++cyc;
  }
  // the loop stopped after sub-iteration done - 1 of the previous cycle: before the last
  // one, its state is in TMEM
  if (done < D) tmem_load32(taddr + (uint32_t)((done - 1) * T::SLOT_COLS), h);

  // the registers hold the final state: write it back in place
#pragma unroll
  for (int s = 0; s < NPT; ++s) {
    if (!valid(s)) continue;
    const int g = (ty0 + ly0 + s * T::ROWS) * nx + tx0 + lx;
#pragma unroll
    for (int i = 0; i < 8; ++i) hsrc[i * N + g] = (s & 1) ? h[s >> 1][i].y : h[s >> 1][i].x;
  }
  if (tile == 0 && (int)threadIdx.x == dwarp * 32) {
    ctl->iter = it;
    ctl->rel = (double)rel;
    ctl->converged = conv;
    ctl->done = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_taddr),
                 "n"(T::TCOLS)
                 : "memory");
  }
}

template <int TY>
__global__ void __launch_bounds__(TileD<TY, 3>::THREADS, 1)
    k_poisson_resident3(KParams k, ResidentGeom rg, float* __restrict__ hbuf,
                        const float2* __restrict__ aq, float* __restrict__ exports,
                        float2* __restrict__ rpartials, Ctl* ctl) {
  resident_loopD<TY, 3>(k, rg, hbuf, aq, exports, rpartials, ctl, blockIdx.x, gridDim.x);
}

// The kernel of a tile height, sub-iterations per exchange (0: the one-step loop;
// 2: heights 24 to 64; 3: heights 48 to 64) and potential scheme (conv: the conventional
// one, on the one- and two-step loops), or nullptr.
template <bool CONV>
const void* resident_kernel_of(int ty, int depth) {
  if (depth == 2) {
    switch (ty) {
      case 24: return (const void*)k_poisson_resident2<24, CONV>;
      case 32: return (const void*)k_poisson_resident2<32, CONV>;
      case 40: return (const void*)k_poisson_resident2<40, CONV>;
      case 48: return (const void*)k_poisson_resident2<48, CONV>;
      case 56: return (const void*)k_poisson_resident2<56, CONV>;
      case 64: return (const void*)k_poisson_resident2<64, CONV>;
      default: return nullptr;
    }
  }
  if (depth == 3) {
    if (CONV) return nullptr;
    switch (ty) {
      case 48: return (const void*)k_poisson_resident3<48>;
      case 56: return (const void*)k_poisson_resident3<56>;
      case 64: return (const void*)k_poisson_resident3<64>;
      default: return nullptr;
    }
  }
  if (depth != 0) return nullptr;
  switch (ty) {
    case 8: return (const void*)k_poisson_resident<8, CONV>;
    case 16: return (const void*)k_poisson_resident<16, CONV>;
    case 24: return (const void*)k_poisson_resident<24, CONV>;
    case 32: return (const void*)k_poisson_resident<32, CONV>;
    case 40: return (const void*)k_poisson_resident<40, CONV>;
    case 48: return (const void*)k_poisson_resident<48, CONV>;
    case 56: return (const void*)k_poisson_resident<56, CONV>;
    case 64: return (const void*)k_poisson_resident<64, CONV>;
    default: return nullptr;
  }
}
const void* resident_kernel(int ty, int depth, bool conv) {
  return conv ? resident_kernel_of<true>(ty, depth) : resident_kernel_of<false>(ty, depth);
}

// Tensor-memory columns one CTA of the multi-step loop allocates (tcgen05.alloc; 0 for
// the one-step loop, which parks nothing), or -1 for a shape with no kernel.
int resident_tmem_columns(int ty, int depth) {
  if (depth == 0) return 0;
  if (!resident_kernel(ty, depth, false)) return -1;
  switch (depth == 2 ? ty : 1000 + ty) {
    case 24: return Tile2<24>::TCOLS;
    case 32: return Tile2<32>::TCOLS;
    case 40: return Tile2<40>::TCOLS;
    case 48: return Tile2<48>::TCOLS;
    case 56: return Tile2<56>::TCOLS;
    case 64: return Tile2<64>::TCOLS;
    case 1048: return TileD<48, 3>::TCOLS;
    case 1056: return TileD<56, 3>::TCOLS;
    case 1064: return TileD<64, 3>::TCOLS;
    default: return -1;
  }
}
const void* resident_batch_kernel(int ty) {
  switch (ty) {
    case 16: return (const void*)k_poisson_resident_batch<16>;
    case 32: return (const void*)k_poisson_resident_batch<32>;
    case 64: return (const void*)k_poisson_resident_batch<64>;
    default: return nullptr;
  }
}

// Tile geometry for the resident loop, or false if the lattice does not fit on chip with
// one tile per SM.  Heights are rounded up to a multiple of 8.  depth: sub-iterations per
// exchange of the multi-step loop (0: the one-step loop), whose D-node-wide ring and band
// need every tile at least 2 D x 2 D and heights of at least 24 (D = 2) or 48 (D = 3).
bool resident_geometry(const KParams& kp, int num_sms, ResidentGeom* g, int* threads,
                       size_t* smem, int fixed_ty, int depth) {
  if (depth != 0 && depth != 2 && depth != 3) return false;
  const long long N = (long long)kp.nx * kp.ny;
  const int ntx = (kp.nx + TXR - 1) / TXR;
  const int min_ty = depth == 3 ? 48 : (depth == 2 ? 24 : 8);
  int TY, nty;
  if (fixed_ty > 0) {
    // fixed 64 x fixed_ty tiles (autotuned schedules; batches: a simulation tiles the
    // same way in any mix)
    if (fixed_ty % 8 != 0 || fixed_ty > 64) return false;
    TY = fixed_ty;
    nty = (kp.ny + TY - 1) / TY;
  } else {
    if (ntx > num_sms) return false;
    // about 2048 nodes per tile, never more tiles than SMs, tiles at most 64 x 64
    long long want = (N + 2047) / 2048;
    if (want > num_sms) want = num_sms;
    nty = (int)(want / ntx);
    if (nty < 1) nty = 1;
    if (nty > num_sms / ntx) nty = num_sms / ntx;
    TY = (kp.ny + nty - 1) / nty;
    TY = (TY + 7) / 8 * 8;
    if (TY < min_ty) TY = min_ty;
    if (TY > 64) {
      // a narrow, tall lattice: as many rows of tiles as 64-row tiles need
      nty = (kp.ny + 63) / 64;
      if (nty > num_sms / ntx) return false;
      TY = (kp.ny + nty - 1) / nty;
      TY = (TY + 7) / 8 * 8;
      if (TY < min_ty) TY = min_ty;
      if (TY > 64) return false;
    }
    nty = (kp.ny + TY - 1) / TY;
  }
  g->TX = TXR;
  g->TY = TY;
  g->ntx = ntx;
  g->nty = nty;
  g->depth = depth;
  *threads = TXR * TY / NPT;
  if (depth != 0) {
    const int D = depth, px = TXR + 2 * D;
    if (TY < min_ty || kp.nx < 2 * D || kp.ny < 2 * D || kp.nx - (ntx - 1) * TXR < 2 * D ||
        kp.ny - (nty - 1) * TY < 2 * D)
      return false;
    g->pmax = 2 * D * TXR + 2 * D * TY;
    *smem = sizeof(float) * (10 * (size_t)(TY + 2 * D) * px + 8 * (size_t)(2 * D * px + 2 * D * TY));
  } else {
    g->pmax = 2 * TXR + 2 * TY;
    *smem = sizeof(float) * (8 * (size_t)(TY + 2) * RX + 2 * (size_t)TY * TXR);
  }
  return true;
}

cudaError_t launch_poisson_resident(const KParams& kp, const ResidentGeom& g, int threads,
                                    size_t smem, const Buffers& b, cudaStream_t st) {
  const void* f = resident_kernel(g.TY, g.depth, kp.scheme == 1);
  if (!f) return cudaErrorInvalidValue;
  KParams k = kp;
  ResidentGeom gg = g;
  float* h = b.h;
  const float2* aq = b.aq;
  float* ex = b.exports;
  float2* rp = b.rpartials;
  Ctl* ctl = b.ctl;
  void* args[] = {&k, &gg, &h, &aq, &ex, &rp, &ctl};
  return cudaLaunchCooperativeKernel(f, dim3(g.ntx * g.nty), dim3(threads), args, smem, st);
}

cudaError_t add_poisson_resident_node(cudaGraph_t graph, const cudaGraphNode_t* deps, size_t nd,
                                      cudaGraphNode_t* out, const KParams& kp,
                                      const ResidentGeom& g, int threads, size_t smem,
                                      const Buffers& b) {
  const void* f = resident_kernel(g.TY, g.depth, kp.scheme == 1);
  if (!f) return cudaErrorInvalidValue;
  KParams k = kp;
  ResidentGeom gg = g;
  float* h = b.h;
  const float2* aq = b.aq;
  float* ex = b.exports;
  float2* rp = b.rpartials;
  Ctl* ctl = b.ctl;
  void* args[] = {&k, &gg, &h, &aq, &ex, &rp, &ctl};
  cudaKernelNodeParams p = {};
  p.func = const_cast<void*>(f);
  p.gridDim = dim3(g.ntx * g.nty);
  p.blockDim = dim3(threads);
  p.sharedMemBytes = (unsigned)smem;
  p.kernelParams = args;
  cudaError_t e = cudaGraphAddKernelNode(out, graph, deps, nd, &p);
  if (e != cudaSuccess) return e;
  cudaKernelNodeAttrValue v = {};
  v.cooperative = 1;
  return cudaGraphKernelNodeSetAttribute(*out, cudaLaunchAttributeCooperative, &v);
}

}  // namespace ehd
