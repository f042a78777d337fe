// Shared device/host helpers of the GCG library (internal header, not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/gcge.h"

namespace gcge {

// --------------------------------------------------------------------------- errors
struct CudaError {
  cudaError_t err;
  const char *file;
  int line;
};

// Records the first CUDA error seen by a handle-less call so that
// gcge_last_error_message() can report it.
void record_cuda_error(cudaError_t e, const char *file, int line);

#define GCGE_CUDA(...)                                                       \
  do {                                                                       \
    cudaError_t _e = (__VA_ARGS__);                                                 \
    if (_e != cudaSuccess) {                                                 \
      ::gcge::record_cuda_error(_e, __FILE__, __LINE__);                     \
      return GCGE_ECUDA;                                                     \
    }                                                                        \
  } while (0)

#define GCGE_CHECK(...)                                                      \
  do {                                                                       \
    int _s = (__VA_ARGS__);                                                         \
    if (_s != GCGE_OK) return _s;                                            \
  } while (0)

#define GCGE_LAUNCH_CHECK() GCGE_CUDA(cudaGetLastError())

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int64_t round_up(int64_t a, int64_t b) { return ((a + b - 1) / b) * b; }

constexpr int kNumSMs = 152;   // GB300: 2 dies x 76 SMs; grids are sized in multiples of this

int device_sm_count();         // queried once, falls back to kNumSMs

// --------------------------------------------------------------------------- device helpers
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = v > w ? v : w;
  }
  return v;
}

// Block-wide sum; `sh` must hold blockDim.x/32 elements. Result valid in all threads.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T t = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  T r = sh[0];
  __syncthreads();
  return r;
}

// Deterministic cross-CTA finish of per-CTA partial rows part[b * k + j] (b < gridDim.x):
// every CTA calls this after writing its row; the last CTA to arrive (atomic ticket, left
// at zero afterwards) sums the rows in a fixed order with all of its threads and calls
// fin(j, sum) for each column.  `sh` needs blockDim.x doubles.  Returns true in the last CTA.
template <typename F>
__device__ __forceinline__ bool last_cta_reduce(int k, const double *part, unsigned *ticket,
                                                double *sh, F fin) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  const int nb = gridDim.x;
  for (int j0 = 0; j0 < k; j0 += blockDim.x) {
    const int kc = (k - j0) < (int)blockDim.x ? (k - j0) : (int)blockDim.x;
    const int slots = blockDim.x / kc;
    const int slot = threadIdx.x / kc, j = j0 + threadIdx.x % kc;
    double s = 0.0;
    if (slot < slots) {
      // four independent sums in flight (fixed order), then combined
      double s4[4] = {0.0, 0.0, 0.0, 0.0};
      int b = slot;
      for (; b + 3 * slots < nb; b += 4 * slots) {
#pragma unroll
        for (int u = 0; u < 4; ++u) s4[u] += __ldcg(part + (int64_t)(b + u * slots) * k + j);
      }
      for (; b < nb; b += slots) s4[0] += __ldcg(part + (int64_t)b * k + j);
      s = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < kc) {
      double t = 0.0;
      for (int q = 0; q < slots; ++q) t += sh[q * kc + threadIdx.x];
      fin(j0 + threadIdx.x, t);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

}  // namespace gcge
