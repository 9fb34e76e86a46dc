// Measurement helper (no counterpart in the paper): the shared-memory bandwidth the GPU
// sustains, the ceiling of the on-chip potential loop, whose per-node work between its
// synchronisations is a store of the eight post-collision populations to shared memory
// and a load of the eight streamed ones.
//
// Every CTA fills a shared buffer, then each thread repeatedly loads one 16-byte vector
// and stores one 16-byte vector per step, consecutive lanes on consecutive vectors (no
// bank conflicts), with many warps per SM in flight so the shared-memory pipe, not the
// latency of one warp's chain, sets the rate.  Bytes counted: loads plus stores.
//
// A second helper measures the synchronisation floor of the two-step on-chip loop: one
// cooperative launch of 64 x 56 tiles (896 threads, one per SM), each cycle exporting the
// tile's two-node-wide band (464 nodes x 8 populations) to global memory, meeting the
// other tiles at a grid barrier (release add, acquire poll bounded by %globaltimer) and
// importing the two-node-wide ring (496 nodes x 8 populations) from its eight neighbours'
// bands, with no collision arithmetic.  What a cycle of the loop costs beyond this floor
// is its arithmetic and shared-memory work.
#include "../../include/ehd.h"
#include "ehd_internal.cuh"

namespace ehd {
namespace {

constexpr int SMEM_THREADS = 512;
constexpr int SMEM_SLOTS = 4;  // float4 slots per thread

// Written only if the (non-negative) running sum were -1, i.e. never; it keeps the
// accesses live without a buffer argument.
__device__ float4 g_smem_sink;

// 16-byte shared-memory accesses the compiler must issue as written (a plain C++ load of
// a value this thread stored itself could be forwarded from a register instead).
__device__ __forceinline__ float4 lds128(unsigned addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}
__device__ __forceinline__ void sts128(unsigned addr, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}

__global__ void __launch_bounds__(SMEM_THREADS) k_smem_bandwidth(int iters) {
  __shared__ float4 buf[SMEM_SLOTS * SMEM_THREADS];
  const int t = threadIdx.x;
  // slot u of this thread: buf[u * SMEM_THREADS + t], inside the array for every u, t
  const unsigned base = (unsigned)__cvta_generic_to_shared(buf + t);
  constexpr unsigned SLOT = SMEM_THREADS * sizeof(float4);
#pragma unroll
  for (int u = 0; u < SMEM_SLOTS; ++u)
    sts128(base + u * SLOT, make_float4((float)(t + u), 1.0f, 2.0f, 3.0f));
  __syncthreads();
  float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < SMEM_SLOTS; ++u) {
      const float4 v = lds128(base + u * SLOT);
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
      sts128(base + ((u + 1) % SMEM_SLOTS) * SLOT, make_float4(v.y, v.z, v.w, acc.x));
    }
  }
  // every value stored or added is a sum of non-negative numbers, so this never stores
  if (acc.x + acc.y + acc.z + acc.w == -1.0f) g_smem_sink = acc;
}

constexpr int GX_TW = 64, GX_TH = 56, GX_THREADS = 896;
constexpr int GX_BAND = GX_TW * GX_TH - (GX_TW - 4) * (GX_TH - 4);  // 464 band nodes
constexpr int GX_RING = (GX_TW + 4) * (GX_TH + 4) - GX_TW * GX_TH;  // 496 ring nodes
constexpr int GX_PLANES = 8;
constexpr unsigned long long GX_TIMEOUT_NS = 2000000000ull;  // 2 s per wait
// unused dynamic shared memory that keeps one CTA per SM, as the loop's 179 KB of shared
// populations and ring do
constexpr int GX_DYN_SMEM = 180 * 1024;

struct GxCtl {
  unsigned count;  // barrier arrivals since the launch started
  int error;       // set when a wait ran out of time
};

__device__ __forceinline__ unsigned long long gx_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void gx_arrive(unsigned* p) {
  asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ unsigned gx_poll(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Neighbour tile of ring node j (0..GX_RING-1): two rows above the tile (68 nodes each,
// corners included), two rows below, then two columns left and right of the tile's rows.
__device__ __forceinline__ int gx_neighbour(int j, int tx, int ty, int ntx, int nty) {
  int dx = 0, dy = 0;
  if (j < 272) {
    const int x = (j % 136) % (GX_TW + 4);
    dy = j < 136 ? 1 : -1;
    dx = x < 2 ? -1 : (x >= GX_TW + 2 ? 1 : 0);
  } else {
    dx = j < 384 ? -1 : 1;
  }
  const int nx = (tx + dx + ntx) % ntx, ny = (ty + dy + nty) % nty;
  return ny * ntx + nx;
}

// bands: 2 parities x tiles x 8 planes x GX_BAND floats.  Grid: ntx * nty CTAs, all
// co-resident (cooperative launch).  Every index below stays inside `bands` and the
// shared arrays: slots < GX_BAND, planes < 8, tiles < ntx * nty.
__global__ void __launch_bounds__(GX_THREADS, 1)
    k_grid_exchange(int ntx, int nty, int cycles, float* __restrict__ bands, GxCtl* ctl) {
  __shared__ float s_band[GX_PLANES * GX_BAND];
  __shared__ float s_ring[GX_PLANES * GX_RING];
  __shared__ int s_ok;
  const int ntiles = ntx * nty, tile = blockIdx.x;
  const int tx = tile % ntx, ty = tile / ntx;
  for (int i = threadIdx.x; i < GX_PLANES * GX_BAND; i += GX_THREADS)
    s_band[i] = 1.0f + (float)(i & 7);
  for (int i = threadIdx.x; i < GX_PLANES * GX_RING; i += GX_THREADS) s_ring[i] = 0.0f;
  __syncthreads();
  unsigned target = 0;
  for (int c = 0; c < cycles; ++c) {
    const size_t par = (size_t)(c & 1) * ntiles;
    float* mine = bands + (par + tile) * GX_PLANES * GX_BAND;
    for (int i = threadIdx.x; i < GX_PLANES * GX_BAND; i += GX_THREADS) mine[i] = s_band[i];
    __syncthreads();
    target += ntiles;
    if (threadIdx.x == 0) {
      int ok = 1;
      gx_arrive(&ctl->count);
      const unsigned long long t0 = gx_ns();
      while ((int)(gx_poll(&ctl->count) - target) < 0) {
        if (gx_ns() - t0 > GX_TIMEOUT_NS) {
          atomicOr(&ctl->error, 1);
          ok = 0;
          break;
        }
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    if (threadIdx.x < GX_RING) {
      const int j = threadIdx.x;
      const float* src = bands + (par + gx_neighbour(j, tx, ty, ntx, nty)) * GX_PLANES * GX_BAND +
                         j % GX_BAND;
#pragma unroll
      for (int i = 0; i < GX_PLANES; ++i) s_ring[i * GX_RING + j] = __ldcg(src + i * GX_BAND);
    }
    __syncthreads();
    // the next export depends on this import, as in the loop
    for (int i = threadIdx.x; i < GX_PLANES * GX_BAND; i += GX_THREADS)
      s_band[i] = 0.5f * s_band[i] + 0.25f * s_ring[i % (GX_PLANES * GX_RING)];
  }
}

}  // namespace
}  // namespace ehd

using namespace ehd;

extern "C" int ehd_diag_grid_exchange(void* stream, int nx, int ny, double* seconds_per_cycle) {
  if (!seconds_per_cycle || nx < 1 || ny < 1) return EHD_ERR_INVALID_ARG;
  const int ntx = (nx + GX_TW - 1) / GX_TW, nty = (ny + GX_TH - 1) / GX_TH;
  // the ring of one tile reaches its neighbours on both sides: at least 3 tiles a direction
  if (ntx < 3 || nty < 3) return EHD_ERR_INVALID_ARG;
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
      cudaFuncSetAttribute(k_grid_exchange, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           GX_DYN_SMEM) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_exchange, GX_THREADS,
                                                    GX_DYN_SMEM) != cudaSuccess) {
    cudaGetLastError();
    return EHD_ERR_CUDA;
  }
  const long long ntiles = (long long)ntx * nty;
  if (!coop || per_sm < 1 || ntiles > (long long)sms * per_sm) return EHD_ERR_TOO_LARGE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t band_bytes = sizeof(float) * 2 * (size_t)ntiles * GX_PLANES * GX_BAND;
  char* mem = nullptr;
  if (cudaMalloc(&mem, band_bytes + 256) != cudaSuccess) {
    cudaGetLastError();
    return EHD_ERR_CUDA;
  }
  float* bands = reinterpret_cast<float*>(mem);
  GxCtl* ctl = reinterpret_cast<GxCtl*>(mem + band_bytes);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int status = EHD_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMemsetAsync(mem, 0, band_bytes + 256, s) != cudaSuccess)
    status = EHD_ERR_CUDA;
  // best time of `cycles` cycles in one launch, for a short and a long launch; the
  // difference over the extra cycles leaves out the launch and the start-up
  const int counts[2] = {64, 1088};
  float best[2] = {0.0f, 0.0f};
  for (int rep = 0; rep < 4 && status == EHD_OK; ++rep) {
    for (int w = 0; w < 2 && status == EHD_OK; ++w) {
      int a0 = ntx, a1 = nty, a2 = counts[w];
      void* args[] = {&a0, &a1, &a2, &bands, &ctl};
      float ms = 0.0f;
      int err = 0;
      if (cudaMemsetAsync(ctl, 0, sizeof(GxCtl), s) != cudaSuccess ||
          cudaEventRecord(e0, s) != cudaSuccess ||
          cudaLaunchCooperativeKernel((const void*)k_grid_exchange, dim3((unsigned)ntiles),
                                      dim3(GX_THREADS), args, GX_DYN_SMEM, s) != cudaSuccess ||
          cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
          cudaMemcpy(&err, &ctl->error, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        status = EHD_ERR_CUDA;
        break;
      }
      if (err) {
        status = EHD_ERR_TIMEOUT;
        break;
      }
      if (rep > 0 && (best[w] == 0.0f || ms < best[w])) best[w] = ms;  // rep 0 warms up
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(mem);
  cudaGetLastError();
  if (status != EHD_OK) return status;
  if (!(best[1] > best[0])) return EHD_ERR_CUDA;
  *seconds_per_cycle = (double)(best[1] - best[0]) * 1e-3 / (counts[1] - counts[0]);
  return EHD_OK;
}

extern "C" int ehd_diag_smem_bandwidth(void* stream, double* bytes_per_second) {
  if (!bytes_per_second) return EHD_ERR_INVALID_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_smem_bandwidth, SMEM_THREADS,
                                                    0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return EHD_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = sms * per_sm;
  const int iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return EHD_ERR_CUDA;
  }
  float best_ms = 0.0f;
  int status = EHD_OK;
  for (int rep = 0; rep < 5 && status == EHD_OK; ++rep) {
    cudaEventRecord(e0, s);
    k_smem_bandwidth<<<blocks, SMEM_THREADS, 0, s>>>(iters);
    cudaEventRecord(e1, s);
    float ms = 0.0f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      status = EHD_ERR_CUDA;
      break;
    }
    if (rep > 0 && (best_ms == 0.0f || ms < best_ms)) best_ms = ms;  // rep 0 warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != EHD_OK || !(best_ms > 0.0f)) return EHD_ERR_CUDA;
  const double bytes = (double)blocks * SMEM_THREADS * iters * SMEM_SLOTS * 2.0 * 16.0;
  *bytes_per_second = bytes / (best_ms * 1e-3);
  return EHD_OK;
}
