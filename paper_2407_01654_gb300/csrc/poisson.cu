// One sub-iteration of the potential LBE (Eq. weq53) with the stopping quantity of
// Algorithm 1, sqrt(sum (varphi^{k+1} - varphi^k)^2 / sum (varphi^k)^2).
//
// Each CTA owns a TX x TY tile.  Phase 1 collides the tile and a one-node ring around it
// from the stored (post-stream) populations into shared memory; phase 2 gathers, for
// every tile node, the post-collision populations arriving from its neighbours (the
// stream), writes them as the next post-stream state and forms varphi^{k+1} from them.
// The ring is collided redundantly by the two CTAs that share it, so one launch yields
// both the new state and its potential without a second pass over memory.  The
// anti-bounce-back Dirichlet rule h_opp(i) = -h*_i + 2 w_i varphi_wall closes the walls.
//
// The collision, with M1 = sum_i c_i h_i and grad varphi = -M1 / (eps_hat + c_s^2 tau_h)
// (Eq. eqA.16), is  h*_i = h_i - (h_i - w_i varphi)/tau_h + a w_i c_i.M1 + q/8,
// a = eps_hat / (c_s^2 tau_h (eps_hat + c_s^2 tau_h)), varphi = sum_{i != 0} h_i / (1 - w_0)
// (Eq. weq55).  h_0 is not carried (it never feeds back).
//
// Per-CTA FP64 partials are reduced by the last CTA to finish, in a fixed order, which
// then advances the loop control: iteration count, copy parity, relative change and the
// stopping decision.  Once the loop is done, further launches return at once.
#include "ehd_internal.cuh"

namespace ehd {

namespace {
// 64 x 16 tiles, 128 threads: a tile row is two whole 128-byte lines, the recomputed ring
// adds 16 % to the tile, and each thread keeps about nine nodes' loads in flight.  On
// GB300 this ran 1.7x faster per sub-iteration than 32 x 16 tiles of 256 threads (the
// same bits; 128 x 16, 128 x 8, 64 x 32, 64 x 8 and 64 x 16 with 64 or 256 threads were
// all slower).
constexpr int TX = STREAM_TX;
constexpr int TY = STREAM_TY;
constexpr int THREADS = 128;
constexpr int RX = TX + 2;
constexpr int RY = TY + 2;
}  // namespace

__global__ void __launch_bounds__(THREADS, 8) k_poisson(KParams k, float* __restrict__ hbuf,
                                                     const float2* __restrict__ aq,
                                                     double2* __restrict__ partials, Ctl* ctl,
                                                     cudaGraphConditionalHandle cond,
                                                     int use_cond) {
  __shared__ float sm[8][RY][RX];
  __shared__ float sphi[TY][TX];
  __shared__ double s_w[THREADS / 32][2];
  __shared__ int s_last;

  // every thread reads the same few words of the loop control, which only the last CTA
  // of a launch writes (after every CTA has read them): through the read-only path, so
  // L1 merges them per SM instead of one L2 slice serving every warp
  if (__ldg(&ctl->done)) return;
  const int parity = __ldg(&ctl->parity);
  const float qshift = k.neutralize ? __ldg(&ctl->mean_q) : 0.0f;
  const float vw_b = __ldg(&ctl->vw_b), vw_t = __ldg(&ctl->vw_t);
  const int nx = k.nx, ny = k.ny;
  const size_t N = (size_t)k.N;
  const float* __restrict__ src = hbuf + (size_t)parity * NH * N;
  float* __restrict__ dst = hbuf + (size_t)(parity ^ 1) * NH * N;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const float om = k.omega_h;

  // phase 1: collide tile + ring (interior rows y0 - 1 .. y0 + TY; in a slab the rows
  // beyond a cut are the stored ghost rows, -1 and ny)
  for (int t = threadIdx.x; t < RX * RY; t += THREADS) {
    const int ly = t / RX, lx = t - ly * RX;
    int gy = y0 + ly - 1;
    if (gy < 0 || gy >= ny) {
      if (!(gy < 0 ? k.halo_lo : k.halo_hi)) {
        if (k.walls) continue;  // outside a wall: never gathered
        gy = wrap(gy, ny);
      }
    }
    const int gx = wrap(x0 + lx - 1, nx);
    const size_t idx = (size_t)(gy + k.row0) * nx + gx;
    float h[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = __ldg(src + i * N + idx);
    const float2 c = __ldg(aq + idx);
    const float varphi = h_varphi(h_sum8(h));
    float m1x, m1y;
    h_moment1(h, m1x, m1y);
    if (k.scheme == 1) {
      const float qs = 0.125f * ((c.y - qshift) * k.inv_chi);
#pragma unroll
      for (int i = 1; i < 9; ++i) sm[i - 1][ly][lx] = h_star_conv(i, h[i - 1], c.x, varphi, qs);
    } else {
      const float qs = 0.125f * (c.y - qshift);
#pragma unroll
      for (int i = 1; i < 9; ++i)
        sm[i - 1][ly][lx] = h_star(i, h[i - 1], om, varphi, c.x, m1x, m1y, qs);
    }
    if (lx >= 1 && lx <= TX && ly >= 1 && ly <= TY) sphi[ly - 1][lx - 1] = varphi;
  }
  __syncthreads();

  // phase 2: stream into the tile nodes, write the new state, accumulate the change
  float num = 0.0f, den = 0.0f;
  for (int t = threadIdx.x; t < TX * TY; t += THREADS) {
    const int ly = t / TX, lx = t - ly * TX;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx >= nx || gy >= ny) continue;
    const size_t idx = (size_t)(gy + k.row0) * nx + gx;
    float hn[8];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const int sy = gy - cy(i);
      float v;
      if (k.walls && ((sy < 0 && !k.halo_lo) || (sy >= ny && !k.halo_hi))) {
        // anti-bounce-back at the wall the population came from
        v = h_wall(i, sm[opp(i) - 1][ly + 1][lx + 1], sy < 0 ? vw_b : vw_t);
      } else {
        v = sm[i - 1][ly + 1 - cy(i)][lx + 1 - cx(i)];
      }
      dst[(i - 1) * N + idx] = v;
      hn[i - 1] = v;
    }
    h_change(h_varphi(h_sum8(hn)), sphi[ly][lx], num, den);
  }

  // reduction: FP32 in a warp, FP64 across warps and CTAs
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_w[warp][0] = (double)num;
    s_w[warp][1] = (double)den;
  }
  __syncthreads();
  const int nblocks = gridDim.x * gridDim.y;
  const int bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < THREADS / 32; ++w) {
      a += s_w[w][0];
      b += s_w[w][1];
    }
    partials[bid] = make_double2(a, b);
    __threadfence();
    const unsigned tk = atomicAdd(&ctl->ticket_p, 1u);
    s_last = (tk == (unsigned)nblocks - 1u);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  __shared__ double s_red[THREADS][2];
  // (in a slab this CTA only publishes the slab's sums; the decision combines every
  // slab's, see k_slab_decide)
  double a = 0.0, b = 0.0;
  for (int j = threadIdx.x; j < nblocks; j += THREADS) {
    const double2 v = __ldcg(partials + j);
    a += v.x;
    b += v.y;
  }
  s_red[threadIdx.x][0] = a;
  s_red[threadIdx.x][1] = b;
  __syncthreads();
  for (int o = THREADS / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s_red[threadIdx.x][0] += s_red[threadIdx.x + o][0];
      s_red[threadIdx.x][1] += s_red[threadIdx.x + o][1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && k.slab) {
    ctl->slab_num = s_red[0][0];
    ctl->slab_den = s_red[0][1];
    ctl->ticket_p = 0u;
    __threadfence();
    return;
  }
  if (threadIdx.x == 0) {
    const double nm = s_red[0][0], dn = s_red[0][1];
    double rel;
    if (nm == 0.0 && dn == 0.0)
      rel = 0.0;
    else if (dn == 0.0)
      rel = __longlong_as_double(0x7ff0000000000000ll);  // +inf
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
    // inside a step graph: the while node repeats this kernel until the loop is done
    if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
  }
}

cudaError_t launch_poisson(const KParams& kp, const Buffers& b, cudaStream_t st) {
  if (stream_tiles(kp.nx, kp.ny) > MAX_PARTIALS) return cudaErrorInvalidValue;
  dim3 grid((kp.nx + TX - 1) / TX, (kp.ny + TY - 1) / TY);  // interior rows
  k_poisson<<<grid, THREADS, 0, st>>>(kp, b.h, b.aq, b.partials, b.ctl,
                                      (cudaGraphConditionalHandle)0, 0);
  return cudaGetLastError();
}

// One sub-iteration as a graph node that leaves the loop's condition alone (slabs: the
// kernel that combines the slabs' sums decides).
cudaError_t add_poisson_node_nocond(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd,
                                    cudaGraphNode_t* out, const KParams& kp, const Buffers& b) {
  if (stream_tiles(kp.nx, kp.ny) > MAX_PARTIALS) return cudaErrorInvalidValue;
  KParams k = kp;
  float* h = b.h;
  const float2* aq = b.aq;
  double2* partials = b.partials;
  Ctl* ctl = b.ctl;
  cudaGraphConditionalHandle cond = 0;
  int use = 0;
  void* args[] = {&k, &h, &aq, &partials, &ctl, &cond, &use};
  cudaKernelNodeParams p = {};
  p.func = (void*)k_poisson;
  p.gridDim = dim3((kp.nx + TX - 1) / TX, (kp.ny + TY - 1) / TY);
  p.blockDim = dim3(THREADS);
  p.kernelParams = args;
  return cudaGraphAddKernelNode(out, g, deps, nd, &p);
}

cudaError_t add_poisson_node(cudaGraph_t g, cudaGraphNode_t* out, const KParams& kp,
                             const Buffers& b, cudaGraphConditionalHandle cond) {
  // one FP64 partial pair per CTA: the grid must fit the partials region
  if (stream_tiles(kp.nx, kp.ny) > MAX_PARTIALS) return cudaErrorInvalidValue;
  KParams k = kp;
  float* h = b.h;
  const float2* aq = b.aq;
  double2* partials = b.partials;
  Ctl* ctl = b.ctl;
  int use = 1;
  void* args[] = {&k, &h, &aq, &partials, &ctl, &cond, &use};
  cudaKernelNodeParams p = {};
  p.func = (void*)k_poisson;
  p.gridDim = dim3((kp.nx + TX - 1) / TX, (kp.ny + TY - 1) / TY);
  p.blockDim = dim3(THREADS);
  p.kernelParams = args;
  return cudaGraphAddKernelNode(out, g, nullptr, 0, &p);
}

}  // namespace ehd
