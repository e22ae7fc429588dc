// Block-level reductions shared by the streaming kernels: warp shuffles,
// then one warp over the per-warp sums; the cross-block stage always adds
// the per-block partials in index order, so every sum is deterministic.
#pragma once
#include <cuda_runtime.h>

namespace sg {

template <int THREADS>
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Sum over the block; every thread receives the result.
template <int THREADS>
__device__ double block_sum_d(double v) {
  __shared__ double sh[THREADS / 32];
  __shared__ double total;
  v = warp_sum_d<THREADS>(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (l < THREADS / 32) ? sh[l] : 0.0;
    t = warp_sum_d<THREADS>(t);
    if (l == 0) total = t;
  }
  __syncthreads();
  return total;
}

// Sum over a large block with few FP64 instructions (the FP64 pipe is the
// scarce one on this chip: one warp instruction holds a scheduler's FP64
// unit for 64 cycles): every thread parks its value in shared memory, then
// four warps -- one per scheduler -- each add THREADS / 128 values per lane
// in index order and combine their lanes with shuffles, and one thread adds
// the four quarters in order.  Every thread receives the result.
template <int THREADS>
__device__ double block_sum_few_d(double v) {
  static_assert(THREADS % 128 == 0, "four warps share the values");
  __shared__ double park[THREADS];
  __shared__ double quarter[4];
  __shared__ double total;
  park[threadIdx.x] = v;
  __syncthreads();
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (w < 4) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < THREADS / 128; ++k) t += park[w * (THREADS / 4) + l + 32 * k];
    t = warp_sum_d<THREADS>(t);
    if (l == 0) quarter[w] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) total = ((quarter[0] + quarter[1]) + quarter[2]) + quarter[3];
  __syncthreads();
  return total;
}

// Fixed-order sum of G per-block partials by one warp (few FP64
// instructions); every thread receives it.  Lane l adds p[l], p[l + 32],
// ... in that order; for G <= 256 its (up to eight) loads are issued
// together, so the read costs one L2 round trip instead of one per term.
template <int THREADS>
__device__ double sum_partials_few_d(const double* __restrict__ p, int G) {
  __shared__ double total;
  __syncthreads();  // every thread has read the previous total
  if (threadIdx.x < 32) {
    double t = 0.0;
    if (G <= 256) {
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = threadIdx.x + 32 * k;
        v[k] = i < G ? p[i] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (threadIdx.x + 32 * k < G) t += v[k];
    } else {
      for (int i = threadIdx.x; i < G; i += 32) t += p[i];
    }
    t = warp_sum_d<THREADS>(t);
    if (threadIdx.x == 0) total = t;
  }
  __syncthreads();
  return total;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Fixed-order sum of G per-block partials; every thread receives it.
template <int THREADS>
__device__ double sum_partials_d(const double* __restrict__ p, int G) {
  double v = 0.0;
  for (int i = threadIdx.x; i < G; i += THREADS) v += p[i];
  return block_sum_d<THREADS>(v);
}

}  // namespace sg
