// Vector kernels: deterministic dot products and norms (warp shuffles,
// then a fixed-order sum of per-block partials), the solution update
// x += Q y (Alg. 4, last line) and precision conversions.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "sg_internal.h"

namespace sg {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Sum over the block; every thread receives the result.
__device__ double block_sum(double v) {
  __shared__ double sh[kThreads / 32];
  __shared__ double total;
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (l < kThreads / 32) ? sh[l] : 0.0;
    t = warp_sum(t);
    if (l == 0) total = t;
  }
  __syncthreads();
  return total;
}

// Fixed-order sum of the G partials of a previous reduction.
__device__ double sum_partials(const double* __restrict__ p, int G) {
  double v = 0.0;
  for (int i = threadIdx.x; i < G; i += kThreads) v += p[i];
  return block_sum(v);
}

// Per-thread partial sums run in the vectors' own precision (T): FP64
// vectors in FP64, FP32 vectors in FP32 (each thread adds ~n/155k terms);
// the block and cross-block stages are FP64.
template <typename T>
__global__ void __launch_bounds__(kThreads)
dot_kernel(int64_t n, const T* __restrict__ x, const T* __restrict__ y,
           double* __restrict__ part) {
  T acc = T(0);
  const int64_t stride = static_cast<int64_t>(gridDim.x) * kThreads;
  int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    T xv[4], yv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { xv[u] = x[i + u * stride]; yv[u] = y[i + u * stride]; }
#pragma unroll
    for (int u = 0; u < 4; ++u) acc = fma(xv[u], yv[u], acc);
  }
  for (; i < n; i += stride) acc = fma(x[i], y[i], acc);
  const double tot = block_sum(static_cast<double>(acc));
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void finish_kernel(const double* __restrict__ part, int G,
                              double* out, int sqrt_out) {
  const double s = sum_partials(part, G);
  if (threadIdx.x == 0) out[0] = sqrt_out ? sqrt(s) : s;
}

__global__ void scale_kernel(int64_t n, const double* __restrict__ x,
                             double* __restrict__ y, double a) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kThreads)
    y[i] = x[i] * a;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
gemv_kernel(int64_t n, int k, const T* __restrict__ Q, int64_t ldq,
            const double* __restrict__ y, double* __restrict__ x) {
  extern __shared__ double ys[];
  for (int j = threadIdx.x; j < k; j += kThreads) ys[j] = y[j];
  __syncthreads();
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kThreads) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc += static_cast<double>(Q[i + j * ldq]) * ys[j];
    x[i] += acc;
  }
}

// FP32 basis: the correction Q y is formed in FP32 (y rounded to FP32 once)
// and added to the FP64 x: one FP64 add per row instead of an FP64 FMA
// and a conversion per product, which made this HBM-sized pass FP64-bound.
// The correction only has to be as accurate as the FP32 inner solve.
__global__ void __launch_bounds__(kThreads)
gemv32_kernel(int64_t n, int k, const float* __restrict__ Q, int64_t ldq,
              const double* __restrict__ y, double* __restrict__ x) {
  extern __shared__ float yf[];
  for (int j = threadIdx.x; j < k; j += kThreads) yf[j] = static_cast<float>(y[j]);
  __syncthreads();
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kThreads) {
    float acc = 0.0f;
    for (int j = 0; j < k; ++j) acc = fmaf(Q[i + j * ldq], yf[j], acc);
    x[i] += static_cast<double>(acc);
  }
}

__global__ void to_f32_kernel(int64_t n, const double* __restrict__ x,
                              float* __restrict__ y, float s) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kThreads)
    y[i] = static_cast<float>(x[i]) * s;
}

__global__ void axpy_f32_kernel(int64_t n, double a, const float* __restrict__ d,
                                double* __restrict__ x) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kThreads)
    x[i] += a * static_cast<double>(d[i]);
}

int stream_grid(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  const int64_t cap = static_cast<int64_t>(device_sm_count()) * 16;
  if (b > cap) b = cap;
  return static_cast<int>(b < 1 ? 1 : b);
}

}  // namespace

namespace {
constexpr int kMaxDevices = 64;
}  // namespace

int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) d = 0;
  return d;
}

// per device: a process may drive several GPUs
int device_sm_count() {
  static int cached[kMaxDevices] = {};
  const int d = current_device();
  if (!cached[d]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v <= 0)
      v = 1;
    cached[d] = v;
  }
  return cached[d];
}

void ensure_dynamic_smem(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> set_to;  // (kernel, device) -> bytes
  const int d = current_device();
  std::lock_guard<std::mutex> lock(mu);
  int& cur = set_to[{fn, d}];
  if (cur < bytes) {
    SG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    cur = bytes;
  }
}

__global__ void gather_kernel(int64_t count, const int32_t* __restrict__ idx,
                              const double* __restrict__ src, double* __restrict__ dst) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < count;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[k] = __ldg(src + idx[k]);
}

void gather(const int32_t* idx, int64_t count, const double* src, double* dst,
            cudaStream_t st) {
  if (count <= 0) return;
  int64_t blocks = (count + kThreads - 1) / kThreads;
  const int64_t cap = static_cast<int64_t>(device_sm_count()) * 8;
  if (blocks > cap) blocks = cap;
  gather_kernel<<<static_cast<int>(blocks), kThreads, 0, st>>>(count, idx, src, dst);
  SG_LAUNCH_CHECK();
}

int reduction_blocks() {
  // two 256-thread CTAs per SM: enough loads in flight for a streaming
  // pass, and few partials for every consumer CTA to re-add
  const int b = device_sm_count() * 2;
  return b > 1024 ? 1024 : b;
}

void dot_partials(int64_t n, const double* x, const double* y,
                  double* partials, cudaStream_t st) {
  dot_kernel<double><<<reduction_blocks(), kThreads, 0, st>>>(n, x, y, partials);
  SG_LAUNCH_CHECK();
}

void finish_sum(const double* partials, double* out, bool sqrt_out,
                cudaStream_t st) {
  finish_kernel<<<1, kThreads, 0, st>>>(partials, reduction_blocks(), out,
                                        sqrt_out ? 1 : 0);
  SG_LAUNCH_CHECK();
}

void scale_copy(int64_t n, const double* x, double* y, double alpha,
                cudaStream_t st) {
  scale_kernel<<<stream_grid(n), kThreads, 0, st>>>(n, x, y, alpha);
  SG_LAUNCH_CHECK();
}

void gemv_n_add(int64_t n, int k, const double* Q, int64_t ldq,
                const double* y, double* x, cudaStream_t st) {
  if (k <= 0) return;
  gemv_kernel<double><<<stream_grid(n), kThreads, sizeof(double) * k, st>>>(
      n, k, Q, ldq, y, x);
  SG_LAUNCH_CHECK();
}

void gemv_n_add32(int64_t n, int k, const float* Q, int64_t ldq,
                  const double* y, double* x, cudaStream_t st) {
  if (k <= 0) return;
  gemv32_kernel<<<stream_grid(n), kThreads, sizeof(float) * k, st>>>(n, k, Q, ldq, y, x);
  SG_LAUNCH_CHECK();
}

void to_f32(int64_t n, const double* x, float* y, float scale,
            cudaStream_t st) {
  to_f32_kernel<<<stream_grid(n), kThreads, 0, st>>>(n, x, y, scale);
  SG_LAUNCH_CHECK();
}

void axpy_f32_to_f64(int64_t n, double alpha, const float* d, double* x,
                     cudaStream_t st) {
  axpy_f32_kernel<<<stream_grid(n), kThreads, 0, st>>>(n, alpha, d, x);
  SG_LAUNCH_CHECK();
}

// Checks of a square CSR matrix's structure, one thread per row: rowptr
// starts at 0 and ends at nnz (bit 1), rows have 0 <= rowptr[r] <=
// rowptr[r+1] <= nnz (bit 2; a row that fails it is not read further, so
// no index leaves the arrays), columns lie in [0, ncols) (bit 4) and
// increase strictly within a row (bit 8).  Bits are OR-ed into flags[0],
// the longest row is merged into flags[1].
__global__ void check_csr_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 int64_t n, int64_t nnz, int64_t ncols, int* __restrict__ flags) {
  int bad = 0, longest = 0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < n; r += stride) {
    const int64_t a = rp[r], b = rp[r + 1];
    if (r == 0 && a != 0) bad |= 1;
    if (r == n - 1 && b != nnz) bad |= 1;
    if (a < 0 || b < a || b > nnz) {
      bad |= 2;
      continue;
    }
    longest = max(longest, static_cast<int>(b - a));
    int64_t prev = -1;
    for (int64_t k = a; k < b; ++k) {
      const int64_t c = ci[k];
      if (c < 0 || c >= ncols) bad |= 4;
      if (c <= prev) bad |= 8;
      prev = c;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    bad |= __shfl_xor_sync(0xffffffffu, bad, off);
    longest = max(longest, __shfl_xor_sync(0xffffffffu, longest, off));
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(flags, bad);
    atomicMax(flags + 1, longest);
  }
}

int check_csr(const int32_t* rowptr, const int32_t* colind, int64_t n, int64_t nnz,
              int64_t ncols, int* flags, int* longest, cudaStream_t st) {
  int* d = nullptr;
  SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&d), 2 * sizeof(int)));
  SG_CUDA(cudaMemsetAsync(d, 0, 2 * sizeof(int), st));
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 8 * static_cast<int64_t>(device_sm_count()));
  check_csr_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(rowptr, colind, n, nnz, ncols, d);
  SG_LAUNCH_CHECK();
  int h[2] = {0, 0};
  SG_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  SG_CUDA(cudaFree(d));
  *flags = h[0];
  *longest = h[1];
  return h[0];
}

void fill_zero(int64_t n, double* x, cudaStream_t st) {
  SG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
}

}  // namespace sg
