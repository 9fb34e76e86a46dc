// Measurement helper (no counterpart in the paper): the shared-memory bandwidth the GPU
// sustains, the ceiling of the on-chip potential loop, whose per-node work between its
// synchronisations is a store of the eight post-collision populations to shared memory
// and a load of the eight streamed ones.
//
// Every CTA fills a shared buffer, then each thread repeatedly loads one 16-byte vector
// and stores one 16-byte vector per step, consecutive lanes on consecutive vectors (no
// bank conflicts), with many warps per SM in flight so the shared-memory pipe, not the
// latency of one warp's chain, sets the rate.  Bytes counted: loads plus stores.
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

}  // namespace
}  // namespace ehd

using namespace ehd;

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
