// CSR sparse kernels: the Newton-step SpMV of the matrix powers kernel
// (Sec. 2, Eq. newtonrecurrence), the residual, the sampled outer product
// of the adjoint gradient and the CSR transpose.
//
// SpMV layout: one thread per row.  One thread per row matters on this
// chip: FP64 warp instructions are expensive (the FP64 pipe is ~1/64 of the
// FP32 rate), so the per-row reduction must not spend shuffles and adds on
// idle lanes; the epilogue multiplies by 1/gamma instead of dividing.
//
// Preferred storage is SELL-32, built at ingest: rows are cut into slices
// of 32 (one warp), and slice q stores entry j of its row l at
// sptr[q] + 32 j + l, padded to the slice's longest row with column -1.
// Lane l of a warp then walks row 32q + l while the warp reads each entry
// index j as one coalesced 256-byte (values) and 128-byte (indices) line,
// with no staging and no barriers; x is gathered through the read-only
// path (stencil locality gives cache hits).  Up to eight entries per row
// are loaded before the FMAs, so their gathers are in flight together, and
// the chunks follow the slice width exactly (no predicated-off FP64 work).
//
// When the padding would be large, CSR is used as is: a CTA owns a
// contiguous block of rows and first stages that block's values and
// column indices in shared memory with coalesced streaming loads, then
// each thread walks its own row from shared memory.
#include <map>
#include <mutex>
#include <vector>

#include "k_reduce.cuh"
#include "sg_internal.h"

namespace sg {

namespace {

constexpr int kThreads = 256;
constexpr int kStage = 2048;   // staged nonzeros per CTA

__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ int ld_stream(const int* p) { return __ldcs(p); }

// MODE 0: y = (A x - theta x + c z) * inv_gamma   (HAS_Z: c z present)
// MODE 1: y = z - A x                              (residual, z = b)
template <int MODE, bool HAS_Z, typename T>
__global__ void __launch_bounds__(kThreads)
spmv_kernel(int n, int rows_per_cta, const int* __restrict__ rowptr,
            const int* __restrict__ colind, const T* __restrict__ val,
            const T* __restrict__ x, const T* __restrict__ z,
            T* __restrict__ y, T theta, T c, T inv_gamma) {
  __shared__ T sval[kStage];
  __shared__ int scol[kStage];
  const int t = threadIdx.x;
  for (int64_t r0 = static_cast<int64_t>(blockIdx.x) * rows_per_cta; r0 < n;
       r0 += static_cast<int64_t>(gridDim.x) * rows_per_cta) {
    const int64_t r1 = (r0 + rows_per_cta < n) ? r0 + rows_per_cta : n;
    const int k0 = rowptr[r0];
    const int len = rowptr[r1] - k0;
    const bool staged = len <= kStage;
    if (staged) {
      for (int e = t; e < len; e += kThreads) {
        sval[e] = ld_stream(val + k0 + e);
        scol[e] = ld_stream(colind + k0 + e);
      }
    }
    __syncthreads();
    for (int64_t row = r0 + t; row < r1; row += kThreads) {
      const int a = rowptr[row], b = rowptr[row + 1];
      T sum = T(0);
      if (staged) {
        for (int k = a - k0; k < b - k0; ++k) sum = fma(sval[k], __ldg(x + scol[k]), sum);
      } else {
        for (int k = a; k < b; ++k) sum = fma(ld_stream(val + k), __ldg(x + ld_stream(colind + k)), sum);
      }
      if (MODE == 1) {
        y[row] = z[row] - sum;
      } else {
        T v = fma(-theta, x[row], sum);
        if (HAS_Z) v = fma(c, z[row], v);
        y[row] = v * inv_gamma;
      }
    }
    __syncthreads();
  }
}

// U consecutive entries (j .. j+U-1) of a SELL-32 row starting at k: the
// indices and values are loaded first, then the gathers, then the FMAs, so
// all of the chunk's loads are in flight together.  Padding (column -1)
// is skipped per lane.
template <int U, typename T>
__device__ __forceinline__ void sell_chunk(const int* __restrict__ scol,
                                           const T* __restrict__ sval,
                                           const T* __restrict__ x, int k, T& sum) {
  int c[U];
  T v[U], xv[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    c[u] = ld_stream(scol + k + 32 * u);
    v[u] = ld_stream(sval + k + 32 * u);
  }
#pragma unroll
  for (int u = 0; u < U; ++u) xv[u] = c[u] >= 0 ? __ldg(x + c[u]) : T(0);
#pragma unroll
  for (int u = 0; u < U; ++u)
    if (c[u] >= 0) sum = fma(v[u], xv[u], sum);
}

// Sum over the SELL-32 row `row` (entries in column order, padding
// skipped), the same FMA sequence as the CSR walk of that row.  The slice
// width is the same for the whole warp, so the chunking below is uniform
// and issues exactly one FMA instruction per stored entry index.
template <typename T>
__device__ __forceinline__ T sell_row(const int* __restrict__ sptr,
                                      const int* __restrict__ scol,
                                      const T* __restrict__ sval,
                                      const T* __restrict__ x, int64_t row) {
  const int64_t q = row >> 5;
  const int a = sptr[q], e = sptr[q + 1];
  const int w = (e - a) >> 5;
  int k = a + static_cast<int>(row & 31);
  T sum = T(0);
  int j = 0;
  for (; j + 8 <= w; j += 8, k += 256) sell_chunk<8>(scol, sval, x, k, sum);
  switch (w - j) {
    case 7: sell_chunk<7>(scol, sval, x, k, sum); break;
    case 6: sell_chunk<6>(scol, sval, x, k, sum); break;
    case 5: sell_chunk<5>(scol, sval, x, k, sum); break;
    case 4: sell_chunk<4>(scol, sval, x, k, sum); break;
    case 3: sell_chunk<3>(scol, sval, x, k, sum); break;
    case 2: sell_chunk<2>(scol, sval, x, k, sum); break;
    case 1: sell_chunk<1>(scol, sval, x, k, sum); break;
    default: break;
  }
  return sum;
}

// The same chunk with the columns as 16-bit offsets from the slice's base
// (0xFFFF: padding).
template <int U, typename T>
__device__ __forceinline__ void sell_chunk16(int base, const uint16_t* __restrict__ soff,
                                             const T* __restrict__ sval,
                                             const T* __restrict__ x, int k, T& sum) {
  unsigned o[U];
  T v[U], xv[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    o[u] = __ldcs(soff + k + 32 * u);
    v[u] = ld_stream(sval + k + 32 * u);
  }
#pragma unroll
  for (int u = 0; u < U; ++u) xv[u] = o[u] != 0xFFFFu ? __ldg(x + base + static_cast<int>(o[u])) : T(0);
#pragma unroll
  for (int u = 0; u < U; ++u)
    if (o[u] != 0xFFFFu) sum = fma(v[u], xv[u], sum);
}

template <typename T>
__device__ __forceinline__ T sell_row16(const int* __restrict__ sptr, const int* __restrict__ sbase,
                                        const uint16_t* __restrict__ soff,
                                        const T* __restrict__ sval, const T* __restrict__ x,
                                        int64_t row) {
  const int64_t q = row >> 5;
  const int a = sptr[q], e = sptr[q + 1];
  const int w = (e - a) >> 5;
  const int base = sbase[q];
  int k = a + static_cast<int>(row & 31);
  T sum = T(0);
  int j = 0;
  for (; j + 8 <= w; j += 8, k += 256) sell_chunk16<8>(base, soff, sval, x, k, sum);
  switch (w - j) {
    case 7: sell_chunk16<7>(base, soff, sval, x, k, sum); break;
    case 6: sell_chunk16<6>(base, soff, sval, x, k, sum); break;
    case 5: sell_chunk16<5>(base, soff, sval, x, k, sum); break;
    case 4: sell_chunk16<4>(base, soff, sval, x, k, sum); break;
    case 3: sell_chunk16<3>(base, soff, sval, x, k, sum); break;
    case 2: sell_chunk16<2>(base, soff, sval, x, k, sum); break;
    case 1: sell_chunk16<1>(base, soff, sval, x, k, sum); break;
    default: break;
  }
  return sum;
}

// OFF16: columns from (sbase, soff) instead of scol.
template <int MODE, bool HAS_Z, bool OFF16, typename T>
__global__ void __launch_bounds__(kThreads)
sell_kernel(int n, int64_t rows32, const int* __restrict__ sptr,
            const int* __restrict__ scol, const int* __restrict__ sbase,
            const uint16_t* __restrict__ soff, const T* __restrict__ sval,
            const T* __restrict__ x, const T* __restrict__ z,
            T* __restrict__ y, T theta, T c, T inv_gamma) {
  for (int64_t row = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; row < rows32;
       row += static_cast<int64_t>(gridDim.x) * kThreads) {
    const T sum = OFF16 ? sell_row16(sptr, sbase, soff, sval, x, row)
                        : sell_row(sptr, scol, sval, x, row);
    if (row < n) {
      if (MODE == 1) {
        y[row] = z[row] - sum;
      } else {
        T v = fma(-theta, x[row], sum);
        if (HAS_Z) v = fma(c, z[row], v);
        y[row] = v * inv_gamma;
      }
    }
  }
}

int rows_per_cta(const DevCsr& A) {
  // as many rows as keep the CTA's nonzeros within the staging buffer,
  // with 25% slack for row-length variation; at most one row per thread
  const double per = A.mean_row > 0 ? A.mean_row * 1.25 : 1.0;
  int r = static_cast<int>(kStage / per);
  if (r > kThreads) r = kThreads;
  if (r < 32) r = 32;
  return r;
}

int grid_for(const DevCsr& A, int rpc) {
  int64_t blocks = (static_cast<int64_t>(A.n) + rpc - 1) / rpc;
  const int64_t cap = static_cast<int64_t>(device_sm_count()) * 16;
  if (blocks > cap) blocks = cap;
  return static_cast<int>(blocks < 1 ? 1 : blocks);
}

template <int MODE, bool HAS_Z, typename T>
void dispatch(const DevCsr& A, const T* val, const T* sval, const T* x, const T* z, T* y,
              T theta, T c, T gamma, cudaStream_t st) {
  if (A.sptr && sval) {
    const int64_t rows32 = static_cast<int64_t>(A.nslices) * 32;
    int64_t blocks = (rows32 + kThreads - 1) / kThreads;
    const int64_t cap = static_cast<int64_t>(device_sm_count()) * 64;
    if (blocks > cap) blocks = cap;
    const int g = static_cast<int>(blocks < 1 ? 1 : blocks);
    if (A.soff)
      sell_kernel<MODE, HAS_Z, true, T><<<g, kThreads, 0, st>>>(
          A.n, rows32, A.sptr, A.scol, A.sbase, A.soff, sval, x, z, y, theta, c, T(1) / gamma);
    else
      sell_kernel<MODE, HAS_Z, false, T><<<g, kThreads, 0, st>>>(
          A.n, rows32, A.sptr, A.scol, A.sbase, A.soff, sval, x, z, y, theta, c, T(1) / gamma);
    SG_LAUNCH_CHECK();
    return;
  }
  const int rpc = rows_per_cta(A);
  spmv_kernel<MODE, HAS_Z, T><<<grid_for(A, rpc), kThreads, 0, st>>>(
      A.n, rpc, A.rowptr, A.colind, val, x, z, y, theta, c, T(1) / gamma);
  SG_LAUNCH_CHECK();
}

// ------------------------------------------------------------------------
// One Arnoldi step of the Ritz pre-pass (Sec. 3.4) in a single cooperative
// launch: w = A v_j with the partial sums of w.w and v_0.w fused into the
// SpMV, then the j+1 modified Gram-Schmidt phases (h_l = v_l.w from the
// previous phase's partials, w -= h_l v_l, partials of v_{l+1}.w), then
// w /= ||w||.  Phases are separated by a grid barrier on a global arrival
// counter and generation word; every block is resident (cooperative
// launch), and each wait is time-bounded: on timeout the kernel records
// an error and runs to completion with whatever it has.  bar: 64 zeroed
// words (arrival counter and generation on separate 128-byte lines).
constexpr uint64_t kBarrierNs = 2000000000ull;

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bar[0]: arrivals; bar[32]: generation (a separate 128-byte line, so the
// pollers do not contend with the arrivals)
__device__ void grid_barrier(unsigned* bar, unsigned nblocks, int* err,
                             uint64_t limit_ns = kBarrierNs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 32;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 32, 1u);
    } else if (*reinterpret_cast<volatile int*>(err) == 0) {
      // (after an earlier timeout every barrier is skipped, so a broken
      // barrier costs one time limit, not one per phase)
      const uint64_t t0 = now_ns();
      unsigned spins = 0;
      while (*gen == g) {
        __nanosleep(32);
        if ((++spins & 255u) == 0 && now_ns() - t0 > limit_ns) {
          atomicExch(err, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Grid barrier on a counter that only grows: every CTA adds one per
// barrier, and barrier number k of the launch (counting from 0) is passed
// once the counter reaches base + G (k + 1), base being the counter's value
// when the launch started (known to the host, which zeroes the counter at
// the start of a pre-pass).  No reset and no generation word: the last
// arrival releases the waiters directly, one L2 round trip sooner than
// grid_barrier.  The wait is time-bounded like grid_barrier's.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ void grid_barrier_count(unsigned* ctr, unsigned target, int* err,
                                   uint64_t limit_ns = kBarrierNs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    if (*reinterpret_cast<volatile int*>(err) == 0) {
      const uint64_t t0 = now_ns();
      unsigned spins = 0;
      while (static_cast<int>(ld_acquire_u32(ctr) - target) < 0) {
        if ((++spins & 255u) == 0 && now_ns() - t0 > limit_ns) {
          atomicExch(err, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

constexpr int kCoopThreads = 1024;  // one CTA per SM, 32 warps in flight
constexpr int kCoopStage = 8192;    // staged nonzeros per CTA tile

// SELL: the SpMV phase walks the SELL-32 arrays (rowptr = sptr, colind =
// scol, val = sval, rows_per_cta unused) instead of staging CSR tiles.
template <typename T, bool SELL>
__global__ void __launch_bounds__(kCoopThreads, 1)
arnoldi_step_kernel(int n, int rows_per_cta, const int* __restrict__ rowptr,
                    const int* __restrict__ colind, const T* __restrict__ val,
                    T* __restrict__ V, int64_t ld, int j, double* __restrict__ H,
                    int ldh, double* __restrict__ wn, double* __restrict__ red,
                    unsigned* bar, int* err, int64_t rows32) {
  extern __shared__ __align__(16) unsigned char coop_smem[];
  T* sval = reinterpret_cast<T*>(coop_smem);
  int* scol = reinterpret_cast<int*>(coop_smem + sizeof(T) * kCoopStage);
  const int G = gridDim.x;
  const int t = threadIdx.x;
  const T* vj = V + static_cast<int64_t>(j) * ld;
  const T* v0 = V;
  T* w = V + static_cast<int64_t>(j + 1) * ld;
  double* pWW = red;
  double* pA = red + G;
  double* pB = red + 2 * G;
  // phase 0: w = A v_j, partials of w.w and v_0.w
  T accw = T(0), accv = T(0);
  if (SELL) {
    for (int64_t row = blockIdx.x * static_cast<int64_t>(kCoopThreads) + t; row < rows32;
         row += static_cast<int64_t>(G) * kCoopThreads) {
      const T sum = sell_row(rowptr, colind, val, vj, row);
      if (row < n) {
        w[row] = sum;
        accw = fma(sum, sum, accw);
        accv = fma(v0[row], sum, accv);
      }
    }
  } else
  for (int64_t r0 = static_cast<int64_t>(blockIdx.x) * rows_per_cta; r0 < n;
       r0 += static_cast<int64_t>(G) * rows_per_cta) {
    const int64_t r1 = (r0 + rows_per_cta < n) ? r0 + rows_per_cta : n;
    const int k0 = rowptr[r0];
    const int len = rowptr[r1] - k0;
    const bool staged = len <= kCoopStage;
    if (staged) {
      for (int e = t; e < len; e += kCoopThreads) {
        sval[e] = ld_stream(val + k0 + e);
        scol[e] = ld_stream(colind + k0 + e);
      }
    }
    __syncthreads();
    for (int64_t row = r0 + t; row < r1; row += kCoopThreads) {
      const int a = rowptr[row], b = rowptr[row + 1];
      T sum = T(0);
      if (staged) {
        for (int k = a - k0; k < b - k0; ++k) sum = fma(sval[k], __ldg(vj + scol[k]), sum);
      } else {
        for (int k = a; k < b; ++k) sum = fma(ld_stream(val + k), __ldg(vj + ld_stream(colind + k)), sum);
      }
      w[row] = sum;
      accw = fma(sum, sum, accw);
      accv = fma(v0[row], sum, accv);
    }
    __syncthreads();
  }
  {
    const double sw = block_sum_few_d<kCoopThreads>(static_cast<double>(accw));
    const double sv = block_sum_few_d<kCoopThreads>(static_cast<double>(accv));
    if (t == 0) { pWW[blockIdx.x] = sw; pA[blockIdx.x] = sv; }
  }
  grid_barrier(bar, G, err);
  if (blockIdx.x == 0) {
    const double ww = sum_partials_few_d<kCoopThreads>(pWW, G);
    if (t == 0) wn[j] = sqrt(ww);
  }
  // MGS phases l = 0..j (four independent element streams per thread)
  const int64_t stride = static_cast<int64_t>(G) * kCoopThreads;
  const int64_t i0 = blockIdx.x * static_cast<int64_t>(kCoopThreads) + t;
  double* pin = pA;
  double* pout = pB;
  for (int l = 0; l <= j; ++l) {
    const double h = sum_partials_few_d<kCoopThreads>(pin, G);
    if (blockIdx.x == 0 && t == 0) H[l + static_cast<int64_t>(j) * ldh] = h;
    const T ht = static_cast<T>(h);
    const T* vl = V + static_cast<int64_t>(l) * ld;
    const T* vn = (l < j) ? V + static_cast<int64_t>(l + 1) * ld : w;
    T acc = T(0);
    int64_t i = i0;
    for (; i + 3 * stride < n; i += 4 * stride) {
      T wv[4], vv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { wv[u] = w[i + u * stride]; vv[u] = vl[i + u * stride]; }
      T nv[4];
      if (l < j) {
#pragma unroll
        for (int u = 0; u < 4; ++u) nv[u] = vn[i + u * stride];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const T wi = fma(-ht, vv[u], wv[u]);
        w[i + u * stride] = wi;
        acc = fma(l < j ? nv[u] : wi, wi, acc);
      }
    }
    for (; i < n; i += stride) {
      const T wi = fma(-ht, vl[i], w[i]);
      w[i] = wi;
      acc = fma(l < j ? vn[i] : wi, wi, acc);
    }
    const double tot = block_sum_few_d<kCoopThreads>(static_cast<double>(acc));
    if (t == 0) pout[blockIdx.x] = tot;
    grid_barrier(bar, G, err);
    double* tmp = pin; pin = pout; pout = tmp;
  }
  // normalise
  const double nrm = sqrt(sum_partials_few_d<kCoopThreads>(pin, G));
  if (blockIdx.x == 0 && t == 0) H[(j + 1) + static_cast<int64_t>(j) * ldh] = nrm;
  const double inv = 1.0 / nrm;
  for (int64_t i = i0; i < n; i += stride)
    w[i] = static_cast<T>(static_cast<double>(w[i]) * inv);
}

// The same FP64 step with w resident on chip.  w = A v_j is first formed in
// V's column j+1 by the SELL SpMV kernel (full occupancy, and the whole L1
// for the gathers of v_j); then CTA b of this cooperative kernel loads its
// rows [b R, (b+1) R) of w into shared memory and keeps them there through
// the MGS phases to the final normalisation.  A thread always touches the
// same rows, so w needs no barrier of its own; each phase streams only v_l
// (just read as the previous phase's v_{l+1}, an L2 hit) and v_{l+1},
// instead of reading and writing w through HBM as well.  Phase order, fused
// next-vector dot and per-CTA partials are those of arnoldi_step_kernel;
// only the rows a CTA owns differ.
__global__ void __launch_bounds__(kCoopThreads, 1)
arnoldi_mgs_resident_kernel(int n, int rows_cta, double* __restrict__ V, int64_t ld, int j,
                            double* __restrict__ H, int ldh, double* __restrict__ wn,
                            double* __restrict__ red, unsigned* ctr, unsigned base, int* err) {
  extern __shared__ __align__(16) unsigned char coop_smem[];
  double* ws = reinterpret_cast<double*>(coop_smem);
  const int G = gridDim.x;
  const int t = threadIdx.x;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rows_cta;
  const int64_t r1 = (r0 + rows_cta < n) ? r0 + rows_cta : n;
  const int nr = r1 > r0 ? static_cast<int>(r1 - r0) : 0;
  const double* v0 = V + r0;
  double* w = V + static_cast<int64_t>(j + 1) * ld + r0;
  double* pWW = red;
  double* pA = red + G;
  double* pB = red + 2 * G;
  // this CTA's rows of w = A v_j, partials of w.w and v_0.w
  double accw = 0.0, accv = 0.0;
  for (int i = t; i < nr; i += kCoopThreads) {
    const double wi = w[i];
    ws[i] = wi;
    accw = fma(wi, wi, accw);
    accv = fma(v0[i], wi, accv);
  }
  {
    const double sw = block_sum_few_d<kCoopThreads>(accw);
    const double sv = block_sum_few_d<kCoopThreads>(accv);
    if (t == 0) { pWW[blockIdx.x] = sw; pA[blockIdx.x] = sv; }
  }
  unsigned target = base + static_cast<unsigned>(G);
  grid_barrier_count(ctr, target, err);
  if (blockIdx.x == 0) {
    const double ww = sum_partials_few_d<kCoopThreads>(pWW, G);
    if (t == 0) wn[j] = sqrt(ww);
  }
  // MGS phases l = 0..j: h_l from the previous phase's partials, w -= h_l
  // v_l, partials of v_{l+1}.w (of w.w in the last phase)
  double* pin = pA;
  double* pout = pB;
  for (int l = 0; l <= j; ++l) {
    const double h = sum_partials_few_d<kCoopThreads>(pin, G);
    if (blockIdx.x == 0 && t == 0) H[l + static_cast<int64_t>(j) * ldh] = h;
    const double* vl = V + static_cast<int64_t>(l) * ld + r0;
    const double* vn = V + static_cast<int64_t>(l + 1) * ld + r0;
    double acc = 0.0;
    int i = t;
    if (l < j) {
      for (; i + 3 * kCoopThreads < nr; i += 4 * kCoopThreads) {
        double wv[4], vv[4], nv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          wv[u] = ws[i + u * kCoopThreads];
          vv[u] = vl[i + u * kCoopThreads];
          nv[u] = vn[i + u * kCoopThreads];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const double wi = fma(-h, vv[u], wv[u]);
          ws[i + u * kCoopThreads] = wi;
          acc = fma(nv[u], wi, acc);
        }
      }
      for (; i < nr; i += kCoopThreads) {
        const double wi = fma(-h, vl[i], ws[i]);
        ws[i] = wi;
        acc = fma(vn[i], wi, acc);
      }
    } else {
      for (; i < nr; i += kCoopThreads) {
        const double wi = fma(-h, vl[i], ws[i]);
        ws[i] = wi;
        acc = fma(wi, wi, acc);
      }
    }
    const double tot = block_sum_few_d<kCoopThreads>(acc);
    if (t == 0) pout[blockIdx.x] = tot;
    target += static_cast<unsigned>(G);
    grid_barrier_count(ctr, target, err);
    double* tmp = pin; pin = pout; pout = tmp;
  }
  // normalise into V's column j+1
  const double nrm = sqrt(sum_partials_few_d<kCoopThreads>(pin, G));
  if (blockIdx.x == 0 && t == 0) H[(j + 1) + static_cast<int64_t>(j) * ldh] = nrm;
  const double inv = 1.0 / nrm;
  for (int i = t; i < nr; i += kCoopThreads) w[i] = ws[i] * inv;
}

// FP32 form of the same step with grouped lookahead (used for the steps
// past the two-barrier step's basis limit, kIcMaxCols vectors): the MGS
// projections are taken kGrp basis vectors per grid barrier.  With d_k = v_k.w and the
// group's Gram entries G_kq = v_k.v_q (q < k), all summed in the pass that
// precedes the group, the MGS coefficients follow exactly by forward
// substitution, h_k = d_k - sum_{q<k} G_kq h_q (what MGS computes, in
// another rounding order); w then loses the group in MGS order,
// w -= h_0 v_0, w -= h_1 v_1, ...  One barrier per group instead of one
// per vector: the FP32 step is barrier-bound, not bandwidth-bound, and
// reads every basis vector twice either way.
constexpr int kGrp = 4;
// per block, kNP sums: d_k = v_k.w at k (k < kGrp), then the Gram entry
// v_k.v_q (q < k) at kGrp + k(k-1)/2 + q; the norm pass uses slot 0
constexpr int kNP = kGrp + kGrp * (kGrp - 1) / 2;

__device__ __forceinline__ void group_sums(const float* __restrict__ V, int64_t ld, int64_t row,
                                           int l, int g, float wi, float* acc) {
  float v[kGrp];
#pragma unroll
  for (int k = 0; k < kGrp; ++k) v[k] = k < g ? V[row + static_cast<int64_t>(l + k) * ld] : 0.0f;
#pragma unroll
  for (int k = 0; k < kGrp; ++k) {
    acc[k] = fmaf(v[k], wi, acc[k]);
#pragma unroll
    for (int q = 0; q < k; ++q) acc[kGrp + k * (k - 1) / 2 + q] = fmaf(v[k], v[q], acc[kGrp + k * (k - 1) / 2 + q]);
  }
}

template <bool SELL>
__global__ void __launch_bounds__(kCoopThreads, 1)
arnoldi_step_grouped_kernel(int n, int rows_per_cta, const int* __restrict__ rowptr,
                            const int* __restrict__ colind, const float* __restrict__ val,
                            float* __restrict__ V, int64_t ld, int j,
                            double* __restrict__ H, int ldh, double* __restrict__ wn,
                            double* __restrict__ red, unsigned* bar, int* err,
                            int64_t rows32) {
  extern __shared__ __align__(16) unsigned char coop_smem[];
  __shared__ double swarp[kCoopThreads / 32][kNP];
  __shared__ double ssum[kNP];
  __shared__ double hs[kGrp];
  const int G = gridDim.x;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const float* vj = V + static_cast<int64_t>(j) * ld;
  float* w = V + static_cast<int64_t>(j + 1) * ld;
  double* pin = red;
  double* pout = red + static_cast<int64_t>(G) * kNP;
  double* pW = red + 2 * static_cast<int64_t>(G) * kNP;
  const int64_t stride = static_cast<int64_t>(G) * kCoopThreads;
  const int64_t i0 = blockIdx.x * static_cast<int64_t>(kCoopThreads) + t;

  // block sums of acc[0..np) -> dst[blockIdx.x * dstride + p]: FP32
  // shuffles within each warp, FP64 only in the one warp that combines
  // the 32 warp sums (FP64 instructions in every warp made the FP64 pipe
  // the limit of this FP32 kernel)
  auto block_partials = [&](const float* acc, int np, double* dst, int dstride) {
    for (int p = 0; p < np; ++p) {
      const float v = warp_sum_f(acc[p]);
      if (lane == 0) swarp[warp][p] = static_cast<double>(v);
    }
    __syncthreads();
    if (warp == 0) {
      for (int p = 0; p < np; ++p) {
        const double v = warp_sum_d<kCoopThreads>(swarp[lane][p]);
        if (lane == 0) dst[static_cast<int64_t>(blockIdx.x) * dstride + p] = v;
      }
    }
    __syncthreads();
  };
  // fixed-order sums over the G blocks' partials -> ssum[0..np)
  auto gather = [&](const double* src, int np) {
    if (warp < np) {
      double v = 0.0;
      for (int c = lane; c < G; c += 32) v += src[static_cast<int64_t>(c) * kNP + warp];
      v = warp_sum_d<kCoopThreads>(v);
      if (lane == 0) ssum[warp] = v;
    }
    __syncthreads();
  };

  const int ncols = j + 1;  // basis vectors v_0 .. v_j to project out
  int g1 = ncols < kGrp ? ncols : kGrp;
  // phase 0: w = A v_j; partials of w.w and of group 0's dots and Gram
  {
    float acc[kNP];
#pragma unroll
    for (int p = 0; p < kNP; ++p) acc[p] = 0.0f;
    float accw[1] = {0.0f};
    if (SELL) {
      for (int64_t row = i0; row < rows32; row += stride) {
        const float sum = sell_row(rowptr, colind, val, vj, row);
        if (row < n) {
          w[row] = sum;
          accw[0] = fmaf(sum, sum, accw[0]);
          group_sums(V, ld, row, 0, g1, sum, acc);
        }
      }
    } else {
      float* sval = reinterpret_cast<float*>(coop_smem);
      int* scol = reinterpret_cast<int*>(coop_smem + sizeof(float) * kCoopStage);
      for (int64_t r0 = static_cast<int64_t>(blockIdx.x) * rows_per_cta; r0 < n;
           r0 += static_cast<int64_t>(G) * rows_per_cta) {
        const int64_t r1 = (r0 + rows_per_cta < n) ? r0 + rows_per_cta : n;
        const int k0 = rowptr[r0];
        const int len = rowptr[r1] - k0;
        const bool staged = len <= kCoopStage;
        if (staged) {
          for (int e = t; e < len; e += kCoopThreads) {
            sval[e] = ld_stream(val + k0 + e);
            scol[e] = ld_stream(colind + k0 + e);
          }
        }
        __syncthreads();
        for (int64_t row = r0 + t; row < r1; row += kCoopThreads) {
          const int a = rowptr[row], b = rowptr[row + 1];
          float sum = 0.0f;
          if (staged) {
            for (int k = a - k0; k < b - k0; ++k) sum = fmaf(sval[k], __ldg(vj + scol[k]), sum);
          } else {
            for (int k = a; k < b; ++k)
              sum = fmaf(ld_stream(val + k), __ldg(vj + ld_stream(colind + k)), sum);
          }
          w[row] = sum;
          accw[0] = fmaf(sum, sum, accw[0]);
          group_sums(V, ld, row, 0, g1, sum, acc);
        }
        __syncthreads();
      }
    }
    block_partials(accw, 1, pW, 1);
    block_partials(acc, kNP, pin, kNP);
  }
  grid_barrier(bar, G, err);
  if (blockIdx.x == 0 && warp == 0) {
    double ww = 0.0;
    for (int c = lane; c < G; c += 32) ww += pW[c];
    ww = warp_sum_d<kCoopThreads>(ww);
    if (lane == 0) wn[j] = sqrt(ww);
  }
  // groups of kGrp basis vectors
  for (int l0 = 0; l0 < ncols; l0 += kGrp) {
    const int gs = g1;
    const int l1 = l0 + gs;
    const int gn = (ncols - l1) < kGrp ? (ncols - l1) : kGrp;  // next group (0: none)
    gather(pin, kNP);
    if (t == 0) {
      for (int k = 0; k < gs; ++k) {
        double hk = ssum[k];
        for (int q = 0; q < k; ++q) hk -= ssum[kGrp + k * (k - 1) / 2 + q] * hs[q];
        hs[k] = hk;
        if (blockIdx.x == 0) H[(l0 + k) + static_cast<int64_t>(j) * ldh] = hk;
      }
    }
    __syncthreads();
    float hf[kGrp];
#pragma unroll
    for (int k = 0; k < kGrp; ++k) hf[k] = k < gs ? static_cast<float>(hs[k]) : 0.0f;
    float acc[kNP];
#pragma unroll
    for (int p = 0; p < kNP; ++p) acc[p] = 0.0f;
    // two elements per iteration, so both elements' loads are in flight
    // together (one element at a time left each thread waiting on memory)
    int64_t i = i0;
    for (; i + stride < n; i += 2 * stride) {
      float wi[2], vu[2][kGrp];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        wi[e] = w[i + e * stride];
#pragma unroll
        for (int k = 0; k < kGrp; ++k)
          vu[e][k] = k < gs ? V[i + e * stride + static_cast<int64_t>(l0 + k) * ld] : 0.0f;
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
#pragma unroll
        for (int k = 0; k < kGrp; ++k)
          if (k < gs) wi[e] = fmaf(-hf[k], vu[e][k], wi[e]);
        w[i + e * stride] = wi[e];
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (gn > 0) group_sums(V, ld, i + e * stride, l1, gn, wi[e], acc);
        else acc[0] = fmaf(wi[e], wi[e], acc[0]);
      }
    }
    for (; i < n; i += stride) {
      float wi = w[i];
#pragma unroll
      for (int k = 0; k < kGrp; ++k)
        if (k < gs) wi = fmaf(-hf[k], V[i + static_cast<int64_t>(l0 + k) * ld], wi);
      w[i] = wi;
      if (gn > 0) group_sums(V, ld, i, l1, gn, wi, acc);
      else acc[0] = fmaf(wi, wi, acc[0]);
    }
    block_partials(acc, kNP, pout, kNP);
    grid_barrier(bar, G, err);
    double* tmp = pin; pin = pout; pout = tmp;
    g1 = gn;
  }
  // normalise: the last pass left the partials of ||w||^2 in slot 0
  gather(pin, 1);
  const double nrm = sqrt(ssum[0]);
  if (blockIdx.x == 0 && t == 0) H[(j + 1) + static_cast<int64_t>(j) * ldh] = nrm;
  const float inv = static_cast<float>(1.0 / nrm);
  for (int64_t i = i0; i < n; i += stride) w[i] *= inv;
}

// FP32 step with two grid barriers (the inverse compact WY form of MGS):
// for the basis v_0..v_j, the MGS coefficients of w = A v_j satisfy
//   h_k = d_k - sum_{q<k} G_kq h_q,  d_k = v_k.w,  G_kq = v_k.v_q,
// so with the lower triangle L of V^T V, h = (I + L)^{-1} d: the
// projections MGS takes one after another, in another rounding order
// (low-synchronisation MGS of Swirydowicz, Langou, Ananthan, Yang and
// Thomas).  Each step then reads the basis twice at full bandwidth:
//   pass A: w = A v_j chunk by chunk (a CTA's own rows, staged with v_j in
//           shared memory), and for every column q of the chunk the
//           partials of v_q.w and v_q.v_j (the new Gram row);
//   barrier; every CTA sums the partials in the same fixed order, keeps
//           row j of the Gram matrix, and solves (I + L) h = d;
//   pass B: w -= sum_q h_q v_q for the CTA's rows (q ascending, the MGS
//           order per element) with the partials of ||w||^2;
//   barrier; w /= ||w||.
// The Gram matrix is stored packed by rows (row k at k(k-1)/2) in global
// memory for the later steps and staged in shared memory before pass A.
constexpr int kIcChunk = 4096;                 // rows per staged chunk
constexpr int kIcMaxCols = 161;                // basis vectors v_0..v_j per step

__host__ __device__ constexpr int ic_tri(int ncols) { return ncols * (ncols - 1) / 2; }

// dynamic shared memory: sw, sv (chunk), column sums, Gram triangle, d, h,
// two scalars, -h in FP32
__host__ __device__ constexpr size_t ic_smem_bytes(int ncols) {
  return sizeof(float) * 2 * kIcChunk + sizeof(double) * 2 * ncols +
         sizeof(double) * (ic_tri(ncols) + 2 * ncols + 8) + sizeof(float) * ncols;
}

// partials: (2 ncols + 1) per CTA for pass A, then G for the norm, then the
// packed Gram matrix of up to kIcMaxCols vectors
int64_t ic_red_doubles(int G) {
  return static_cast<int64_t>(2 * kIcMaxCols + 2) * G + ic_tri(kIcMaxCols);
}

template <bool SELL>
__global__ void __launch_bounds__(kCoopThreads, 1)
arnoldi_step_icwy_kernel(int n, const int* __restrict__ rowptr,
                         const int* __restrict__ colind, const float* __restrict__ val,
                         float* __restrict__ V, int64_t ld, int j, double* __restrict__ H,
                         int ldh, double* __restrict__ wn, double* __restrict__ red,
                         unsigned* bar, int* err) {
  extern __shared__ __align__(16) unsigned char coop_smem[];
  __shared__ double swarp[kCoopThreads / 32];
  const int ncols = j + 1;
  const int G = gridDim.x;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  float* sw = reinterpret_cast<float*>(coop_smem);
  float* sv = sw + kIcChunk;
  double* slots = reinterpret_cast<double*>(sv + kIcChunk);  // [q][2]: v_q.w, v_q.v_j
  double* tri = slots + 2 * ncols;
  double* dk = tri + ic_tri(ncols);
  double* hk = dk + ncols;
  double* misc = hk + ncols;  // [0]: ||A v_j||^2, [1]: ||w||^2 after projection
  float* nh = reinterpret_cast<float*>(misc + 8);  // -h_q in FP32 for pass B

  const int P = 2 * ncols + 1;
  double* pA = red;                                                   // G x P
  double* pN = red + static_cast<int64_t>(2 * kIcMaxCols + 1) * G;    // G
  double* gram = red + static_cast<int64_t>(2 * kIcMaxCols + 2) * G;  // packed rows

  const float* vj = V + static_cast<int64_t>(j) * ld;
  float* w = V + static_cast<int64_t>(j + 1) * ld;
  // this CTA's rows: whole 32-row slices, as even as possible
  const int64_t nsl = (static_cast<int64_t>(n) + 31) / 32;
  const int64_t r0 = 32 * (nsl * blockIdx.x / G);
  int64_t r1 = 32 * (nsl * (blockIdx.x + 1) / G);
  if (r1 > n) r1 = n;

  // the Gram rows of the earlier steps (read during pass A's latency)
  for (int e = t; e < ic_tri(j); e += kCoopThreads) tri[e] = gram[e];
  for (int e = t; e < 2 * ncols; e += kCoopThreads) slots[e] = 0.0;

  // ------------------------------------------------------------ pass A
  float accww = 0.0f;
  for (int64_t c0 = r0; c0 < r1; c0 += kIcChunk) {
    const int len = static_cast<int>((r1 - c0) < kIcChunk ? (r1 - c0) : kIcChunk);
    __syncthreads();  // the previous chunk's readers are done with sw / sv
    for (int r = t; r < len; r += kCoopThreads) {
      const int64_t row = c0 + r;
      float sum;
      if (SELL) {
        sum = sell_row(rowptr, colind, val, vj, row);
      } else {
        sum = 0.0f;
        const int a = rowptr[row], b = rowptr[row + 1];
        for (int k = a; k < b; ++k) sum = fmaf(ld_stream(val + k), __ldg(vj + ld_stream(colind + k)), sum);
      }
      w[row] = sum;
      sw[r] = sum;
      sv[r] = vj[row];
      accww = fmaf(sum, sum, accww);
    }
    __syncthreads();
    // column q of the chunk belongs to warp q % 32: lane l adds the rows
    // 4 l + 128 it in FP32 (eight float4 loads in flight), the lanes are
    // combined by shuffles, and the chunk's sum is added in FP64 in chunk
    // order
    for (int q = warp; q < ncols; q += 32) {
      const float* vq = V + static_cast<int64_t>(q) * ld + c0;
      float d = 0.0f, gm = 0.0f;
      if (len == kIcChunk) {
#pragma unroll 1
        for (int it0 = 0; it0 < kIcChunk / 128; it0 += 8) {
          float4 a[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            a[u] = *reinterpret_cast<const float4*>(vq + (it0 + u) * 128 + lane * 4);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int r = (it0 + u) * 128 + lane * 4;
            const float4 x = *reinterpret_cast<const float4*>(sw + r);
            const float4 y = *reinterpret_cast<const float4*>(sv + r);
            d = fmaf(a[u].x, x.x, d); d = fmaf(a[u].y, x.y, d);
            d = fmaf(a[u].z, x.z, d); d = fmaf(a[u].w, x.w, d);
            gm = fmaf(a[u].x, y.x, gm); gm = fmaf(a[u].y, y.y, gm);
            gm = fmaf(a[u].z, y.z, gm); gm = fmaf(a[u].w, y.w, gm);
          }
        }
      } else {
        for (int r = lane; r < len; r += 32) {
          const float a = vq[r];
          d = fmaf(a, sw[r], d);
          gm = fmaf(a, sv[r], gm);
        }
      }
      d = warp_sum_f(d);
      gm = warp_sum_f(gm);
      if (lane == 0) {
        slots[2 * q] += static_cast<double>(d);
        slots[2 * q + 1] += static_cast<double>(gm);
      }
    }
  }
  // CTA partials: per column; ||A v_j||^2
  __syncthreads();
  for (int q = t; q < ncols; q += kCoopThreads) {
    pA[static_cast<int64_t>(blockIdx.x) * P + 2 * q] = slots[2 * q];
    pA[static_cast<int64_t>(blockIdx.x) * P + 2 * q + 1] = slots[2 * q + 1];
  }
  {
    const float v = warp_sum_f(accww);
    if (lane == 0) swarp[warp] = static_cast<double>(v);
    __syncthreads();
    if (warp == 0) {
      const double s = warp_sum_d<kCoopThreads>(swarp[lane]);
      if (lane == 0) pA[static_cast<int64_t>(blockIdx.x) * P + 2 * ncols] = s;
    }
  }
  grid_barrier(bar, G, err);

  // ------------------------------------------- sums and the coefficients
  // every CTA adds the G partials of each sum in the same fixed order
  for (int p = warp; p < P; p += 32) {
    double v = 0.0;
    for (int c = lane; c < G; c += 32) v += pA[static_cast<int64_t>(c) * P + p];
    v = warp_sum_d<kCoopThreads>(v);
    if (lane == 0) {
      if (p == 2 * ncols) misc[0] = v;
      else if (p & 1) { if ((p >> 1) < j) tri[ic_tri(j) + (p >> 1)] = v; }  // Gram row j
      else dk[p >> 1] = v;
    }
  }
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int q = t; q < j; q += kCoopThreads) gram[ic_tri(j) + q] = tri[ic_tri(j) + q];
    if (t == 0) wn[j] = sqrt(misc[0]);
  }
  // forward substitution (I + L) h = d by one warp: lanes own rows
  // k = lane + 32 m; column q's h_q is final once columns < q are applied
  if (warp == 0) {
    constexpr int kM = (kIcMaxCols + 31) / 32;
    double dr[kM];
#pragma unroll
    for (int m = 0; m < kM; ++m) {
      const int k = lane + 32 * m;
      dr[m] = k < ncols ? dk[k] : 0.0;
    }
    // the row groups m past the basis are left by a warp-uniform break:
    // predicated FP64 instructions would still take their pipe time
    const int mused = (ncols + 31) / 32;
    for (int q = 0; q < ncols; ++q) {
      double mine = dr[0];
#pragma unroll
      for (int m = 1; m < kM; ++m)
        if (m == (q >> 5)) mine = dr[m];
      const double hq = __shfl_sync(0xffffffffu, mine, q & 31);
      if (lane == 0) hk[q] = hq;
#pragma unroll
      for (int m = 0; m < kM; ++m) {
        if (m >= mused) break;
        const int k = lane + 32 * m;
        if (k > q && k < ncols) dr[m] = fma(-tri[ic_tri(k) + q], hq, dr[m]);
      }
    }
  }
  __syncthreads();
  for (int q = t; q < ncols; q += kCoopThreads) {
    nh[q] = -static_cast<float>(hk[q]);
    if (blockIdx.x == 0) H[q + static_cast<int64_t>(j) * ldh] = hk[q];
  }
  __syncthreads();

  // ------------------------------------------------------------ pass B
  float accn = 0.0f;
  for (int64_t r = r0 + 4 * static_cast<int64_t>(t); r < r1; r += 4 * kCoopThreads) {
    if (r + 3 < r1) {
      float4 wv = *reinterpret_cast<const float4*>(w + r);
      int q = 0;
      for (; q + 8 <= ncols; q += 8) {
        float4 vv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          vv[u] = *reinterpret_cast<const float4*>(V + static_cast<int64_t>(q + u) * ld + r);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float h = nh[q + u];
          wv.x = fmaf(h, vv[u].x, wv.x); wv.y = fmaf(h, vv[u].y, wv.y);
          wv.z = fmaf(h, vv[u].z, wv.z); wv.w = fmaf(h, vv[u].w, wv.w);
        }
      }
      for (; q < ncols; ++q) {
        const float4 vv = *reinterpret_cast<const float4*>(V + static_cast<int64_t>(q) * ld + r);
        const float h = nh[q];
        wv.x = fmaf(h, vv.x, wv.x); wv.y = fmaf(h, vv.y, wv.y);
        wv.z = fmaf(h, vv.z, wv.z); wv.w = fmaf(h, vv.w, wv.w);
      }
      *reinterpret_cast<float4*>(w + r) = wv;
      accn = fmaf(wv.x, wv.x, accn); accn = fmaf(wv.y, wv.y, accn);
      accn = fmaf(wv.z, wv.z, accn); accn = fmaf(wv.w, wv.w, accn);
    } else {
      for (int64_t rr = r; rr < r1; ++rr) {
        float wi = w[rr];
        for (int q = 0; q < ncols; ++q) wi = fmaf(nh[q], V[static_cast<int64_t>(q) * ld + rr], wi);
        w[rr] = wi;
        accn = fmaf(wi, wi, accn);
      }
    }
  }
  {
    const float v = warp_sum_f(accn);
    __syncthreads();  // swarp is free again
    if (lane == 0) swarp[warp] = static_cast<double>(v);
    __syncthreads();
    if (warp == 0) {
      const double s = warp_sum_d<kCoopThreads>(swarp[lane]);
      if (lane == 0) pN[blockIdx.x] = s;
    }
  }
  grid_barrier(bar, G, err);
  if (warp == 0) {
    double v = 0.0;
    for (int c = lane; c < G; c += 32) v += pN[c];
    v = warp_sum_d<kCoopThreads>(v);
    if (lane == 0) misc[1] = v;
  }
  __syncthreads();
  const double nrm = sqrt(misc[1]);
  if (blockIdx.x == 0 && t == 0) H[(j + 1) + static_cast<int64_t>(j) * ldh] = nrm;
  const float inv = static_cast<float>(1.0 / nrm);
  for (int64_t r = r0 + t; r < r1; r += kCoopThreads) w[r] *= inv;
}

// The two-barrier FP32 step while the basis has at most kIcMaxCols
// vectors and the partials buffer holds its sums; false: not launched.
template <bool SELL>
bool launch_arnoldi_icwy(const DevCsr& A, const float* val, float* V, int64_t ld, int j,
                         double* H, int ldh, double* wn, double* red, int red_cap,
                         unsigned* bar, int* err, cudaStream_t st) {
  if (j + 1 > kIcMaxCols) return false;
  const void* fn = reinterpret_cast<const void*>(arnoldi_step_icwy_kernel<SELL>);
  const int smax = static_cast<int>(ic_smem_bytes(kIcMaxCols));
  ensure_dynamic_smem(fn, smax);
  int per_sm = 0;
  SG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kCoopThreads, smax));
  const int mb = per_sm * device_sm_count();
  SG_REQUIRE(mb > 0, SG_ECUDA, "arnoldi step: no resident blocks");
  int G = device_sm_count();
  if (G > mb) G = mb;
  if (ic_red_doubles(G) > red_cap) return false;
  int n = A.n;
  const int* rp = SELL ? A.sptr : A.rowptr;
  const int* ci = SELL ? A.scol : A.colind;
  void* args[] = {&n, const_cast<int**>(&rp), const_cast<int**>(&ci), const_cast<float**>(&val),
                  &V, &ld, &j, &H, const_cast<int*>(&ldh), &wn, &red, &bar, &err};
  SG_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kCoopThreads), args,
                                      ic_smem_bytes(j + 1), st));
  count_launch();
  return true;
}

// Rows per CTA of the resident FP64 step for n rows, or 0 when a CTA's
// slice of w would not fit in shared memory next to the kernel's static
// reduction buffers (then the streaming step runs).  One CTA per SM, at
// least 2048 rows per CTA (fewer CTAs, cheaper barriers, on small systems).
int resident_rows_per_cta(int64_t n, int* grid) {
  static std::mutex mu;
  static std::map<int, int> limit;   // device -> dynamic bytes available
  const int dev = current_device();
  int avail;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = limit.find(dev);
    if (it == limit.end()) {
      int optin = 0;
      SG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      cudaFuncAttributes fa{};
      SG_CUDA(cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(arnoldi_mgs_resident_kernel)));
      it = limit.emplace(dev, optin - static_cast<int>(fa.sharedSizeBytes) - 1024).first;
    }
    avail = it->second;
  }
  const int64_t sms = device_sm_count();
  int64_t R = (n + sms - 1) / sms;
  if (R < 2048) R = 2048;
  R = (R + 31) / 32 * 32;
  if (R * static_cast<int64_t>(sizeof(double)) > avail) return 0;
  *grid = static_cast<int>((n + R - 1) / R);
  return static_cast<int>(R);
}

template <typename T, bool SELL>
void launch_arnoldi_step(const DevCsr& A, const T* val, T* V, int64_t ld, int j,
                         double* H, int ldh, double* wn, double* red, int red_cap,
                         unsigned* bar, int* err, cudaStream_t st) {
  if constexpr (sizeof(T) == 8 && SELL) {
    int G = 0;
    const int R = resident_rows_per_cta(A.n, &G);
    if (R > 0 && G <= device_sm_count() && 3 * G <= red_cap) {
      const void* fn = reinterpret_cast<const void*>(arnoldi_mgs_resident_kernel);
      const int smem = R * static_cast<int>(sizeof(double));
      ensure_dynamic_smem(fn, smem);
      int per_sm = 0;
      SG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kCoopThreads, smem));
      if (per_sm >= 1) {
        // w = A v_j into V's column j+1, then the MGS phases on chip
        dispatch<0, false, T>(A, A.val, val, V + static_cast<int64_t>(j) * ld, nullptr,
                              V + static_cast<int64_t>(j + 1) * ld, T(0), T(0), T(1), st);
        // barriers per step j: one after the w partials, one per MGS phase
        // (j + 1); the counter (word 16 of the barrier block, zeroed at the
        // start of the pre-pass) has seen G (j' + 2) arrivals per earlier step
        int n = A.n;
        int rc = R;
        unsigned* ctr = bar + 16;
        unsigned base = static_cast<unsigned>(G) * static_cast<unsigned>(j) *
                        static_cast<unsigned>(j + 3) / 2u;
        void* args[] = {&n, &rc, &V, &ld, &j, &H, const_cast<int*>(&ldh), &wn, &red, &ctr,
                        &base, &err};
        SG_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kCoopThreads), args, smem, st));
        count_launch();
        return;
      }
    }
  }
  const int smem = SELL ? 0 : kCoopStage * static_cast<int>(sizeof(T) + sizeof(int));
  // FP32: the two-barrier step while the basis fits it, then the grouped-
  // lookahead step; FP64 keeps one projection per phase, the rounding order
  // of the MGS oracle
  if constexpr (sizeof(T) == 4) {
    if (launch_arnoldi_icwy<SELL>(A, val, V, ld, j, H, ldh, wn, red, red_cap, bar, err, st))
      return;
  }
  const void* fn = reinterpret_cast<const void*>(arnoldi_step_kernel<T, SELL>);
  if constexpr (sizeof(T) == 4) fn = reinterpret_cast<const void*>(arnoldi_step_grouped_kernel<SELL>);
  ensure_dynamic_smem(fn, smem);
  int per_sm = 0;
  SG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kCoopThreads, smem));
  const int mb = per_sm * device_sm_count();
  SG_REQUIRE(mb > 0, SG_ECUDA, "arnoldi step: no resident blocks");
  int G = device_sm_count();  // one CTA per SM: fewer arrivals and partials
  if (G > mb) G = mb;
  const int need = sizeof(T) == 4 ? (2 * kNP + 1) * G : 3 * G;
  SG_REQUIRE(need <= red_cap, SG_EINVAL, "arnoldi step: partials buffer too small");
  // rows per tile: the staged nonzeros fit with 25% slack, <= one per thread
  const double per = A.mean_row > 0 ? A.mean_row * 1.25 : 1.0;
  int rpc = static_cast<int>(kCoopStage / per);
  if (rpc > kCoopThreads) rpc = kCoopThreads;
  if (rpc < 32) rpc = 32;
  int n = A.n;
  int64_t rows32 = static_cast<int64_t>(A.nslices) * 32;
  const int* rp = SELL ? A.sptr : A.rowptr;
  const int* ci = SELL ? A.scol : A.colind;
  void* args[] = {&n, &rpc, const_cast<int**>(&rp), const_cast<int**>(&ci),
                  const_cast<T**>(&val), &V, &ld, &j, &H, const_cast<int*>(&ldh), &wn, &red,
                  &bar, &err, &rows32};
  SG_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kCoopThreads), args, smem, st));
  count_launch();
}

__global__ void sampled_outer_kernel(int n, const int* __restrict__ rowptr,
                                     const int* __restrict__ colind,
                                     const double* __restrict__ lam,
                                     const double* __restrict__ x,
                                     double* __restrict__ dval) {
  // one warp per 32/8 rows, 8 lanes per row, like the SpMV
  constexpr int VEC = 8, RPW = 32 / VEC;
  const int lane = threadIdx.x & 31;
  const int sub = lane / VEC, l = lane % VEC;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t base = warp * RPW; base < n; base += nwarps * RPW) {
    const int64_t row = base + sub;
    if (row >= n) continue;
    const double li = -lam[row];
    const int s = rowptr[row], e = rowptr[row + 1];
    for (int k = s + l; k < e; k += VEC) dval[k] = li * __ldg(x + colind[k]);
  }
}

// --- transpose: count entries per column, scan, scatter, sort rows ---
__global__ void count_cols_kernel(int64_t nnz, const int* __restrict__ colind,
                                  int* __restrict__ counts) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       k < nnz; k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    atomicAdd(counts + colind[k], 1);
}

// single-block exclusive scan of n+1 counters (n up to a few million;
// each thread scans a contiguous chunk, then the chunk totals)
__global__ void scan_kernel(int n, const int* __restrict__ counts,
                            int* __restrict__ rowptr) {
  __shared__ long long tot[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int64_t chunk = (static_cast<int64_t>(n) + T - 1) / T;
  const int64_t a = t * chunk, b = (a + chunk < n) ? a + chunk : n;
  long long s = 0;
  for (int64_t i = a; i < b; ++i) s += counts[i];
  tot[t] = s;
  __syncthreads();
  if (t == 0) {
    long long run = 0;
    for (int i = 0; i < T; ++i) { long long v = tot[i]; tot[i] = run; run += v; }
  }
  __syncthreads();
  long long run = tot[t];
  for (int64_t i = a; i < b; ++i) { rowptr[i] = static_cast<int>(run); run += counts[i]; }
  if (b == n && a < b) rowptr[n] = static_cast<int>(run);
  if (n == 0 && t == 0) rowptr[0] = 0;
}

__global__ void scatter_kernel(int n, const int* __restrict__ rowptr,
                               const int* __restrict__ colind,
                               const double* __restrict__ val,
                               const int* __restrict__ trowptr,
                               int* __restrict__ fill, int* __restrict__ tcol,
                               double* __restrict__ tval) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       r < n; r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) {
      const int c = colind[k];
      const int pos = trowptr[c] + atomicAdd(fill + c, 1);
      tcol[pos] = static_cast<int>(r);
      tval[pos] = val[k];
    }
  }
}

// insertion sort of each (short) row by column index: makes the transpose
// independent of the atomic scatter order
__global__ void sort_rows_kernel(int n, const int* __restrict__ rowptr,
                                 int* __restrict__ col,
                                 double* __restrict__ val) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
       r < n; r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int a = rowptr[r], b = rowptr[r + 1];
    for (int i = a + 1; i < b; ++i) {
      const int ci = col[i];
      const double vi = val[i];
      int j = i - 1;
      while (j >= a && col[j] > ci) { col[j + 1] = col[j]; val[j + 1] = val[j]; --j; }
      col[j + 1] = ci;
      val[j + 1] = vi;
    }
  }
}

}  // namespace

void spmv_newton(const DevCsr& A, const double* x, const double* z,
                 double* y, double theta, double c, double gamma,
                 cudaStream_t st) {
  if (c != 0.0 && z)
    dispatch<0, true, double>(A, A.val, A.sval, x, z, y, theta, c, gamma, st);
  else
    dispatch<0, false, double>(A, A.val, A.sval, x, nullptr, y, theta, 0.0, gamma, st);
}

void spmv_newton32(const DevCsr& A, const float* x, const float* z, float* y,
                   float theta, float c, float gamma, cudaStream_t st) {
  if (c != 0.0f && z)
    dispatch<0, true, float>(A, A.val32, A.sval32, x, z, y, theta, c, gamma, st);
  else
    dispatch<0, false, float>(A, A.val32, A.sval32, x, nullptr, y, theta, 0.0f, gamma, st);
}

void residual(const DevCsr& A, const double* b, const double* x, double* r,
              cudaStream_t st) {
  dispatch<1, false, double>(A, A.val, A.sval, x, b, r, 0.0, 0.0, 1.0, st);
}

void sampled_outer(const DevCsr& A, const double* lam, const double* x,
                   double* dval, cudaStream_t st) {
  int64_t gb = (static_cast<int64_t>(A.n) + 31) / 32;
  const int64_t cap = static_cast<int64_t>(device_sm_count()) * 16;
  const int g = static_cast<int>(gb > cap ? cap : (gb < 1 ? 1 : gb));
  sampled_outer_kernel<<<g, kThreads, 0, st>>>(A.n, A.rowptr, A.colind, lam, x,
                                               dval);
  SG_LAUNCH_CHECK();
}

void csr_transpose(const DevCsr& A, DevCsr& T, int32_t* counts,
                   cudaStream_t st) {
  // counts: n+1 ints of scratch; T's arrays are allocated by the caller
  SG_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (A.n + 1), st));
  const int g = device_sm_count() * 8;
  count_cols_kernel<<<g, kThreads, 0, st>>>(A.nnz, A.colind, counts);
  SG_LAUNCH_CHECK();
  scan_kernel<<<1, 1024, 0, st>>>(A.n, counts, T.rowptr);
  SG_LAUNCH_CHECK();
  SG_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (A.n + 1), st));
  scatter_kernel<<<g, kThreads, 0, st>>>(A.n, A.rowptr, A.colind, A.val,
                                         T.rowptr, counts, T.colind, T.val);
  SG_LAUNCH_CHECK();
  sort_rows_kernel<<<g, kThreads, 0, st>>>(A.n, T.rowptr, T.colind, T.val);
  SG_LAUNCH_CHECK();
}

namespace {

// slice widths: width[q] = 32 * (longest row of slice q)
__global__ void sell_width_kernel(int n, int nslices, const int* __restrict__ rowptr,
                                  int* __restrict__ width) {
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < nslices;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r0 = q * 32, r1 = (r0 + 32 < n) ? r0 + 32 : n;
    int w = 0;
    for (int64_t r = r0; r < r1; ++r) w = max(w, rowptr[r + 1] - rowptr[r]);
    width[q] = 32 * w;
  }
}

// one thread per (padded) row: entry j of row 32q + l -> sptr[q] + 32 j + l
template <bool COLS>
__global__ void sell_fill_kernel(int n, int64_t rows32, const int* __restrict__ rowptr,
                                 const int* __restrict__ colind,
                                 const double* __restrict__ val,
                                 const int* __restrict__ sptr, int* __restrict__ scol,
                                 double* __restrict__ sval) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < rows32;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t q = r >> 5;
    const int base = sptr[q] + static_cast<int>(r & 31);
    const int w = (sptr[q + 1] - sptr[q]) >> 5;
    const int a = r < n ? rowptr[r] : 0;
    const int len = r < n ? rowptr[r + 1] - a : 0;
    for (int j = 0; j < w; ++j) {
      const int k = base + 32 * j;
      if (j < len) {
        if (COLS) scol[k] = colind[a + j];
        sval[k] = val[a + j];
      } else {
        if (COLS) scol[k] = -1;
        sval[k] = 0.0;
      }
    }
  }
}

// per slice: the smallest stored column (0 for an all-padding slice), and
// a flag when the slice's columns span 65535 or more
__global__ void sell_base_kernel(int nslices, const int* __restrict__ sptr,
                                 const int* __restrict__ scol, int* __restrict__ sbase,
                                 int* __restrict__ wide) {
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < nslices;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    int lo = 0x7FFFFFFF, hi = -1;
    for (int k = sptr[q]; k < sptr[q + 1]; ++k) {
      const int c = scol[k];
      if (c >= 0) {
        lo = min(lo, c);
        hi = max(hi, c);
      }
    }
    if (hi < 0) lo = hi = 0;
    sbase[q] = lo;
    if (hi - lo >= 0xFFFF) atomicOr(wide, 1);
  }
}

// 16-bit offsets of every stored entry from its slice's base
__global__ void sell_off_kernel(int64_t rows32, const int* __restrict__ sptr,
                                const int* __restrict__ scol, const int* __restrict__ sbase,
                                uint16_t* __restrict__ soff) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < rows32;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t q = r >> 5;
    const int w = (sptr[q + 1] - sptr[q]) >> 5;
    const int b = sbase[q];
    for (int j = 0; j < w; ++j) {
      const int k = sptr[q] + static_cast<int>(r & 31) + 32 * j;
      const int c = scol[k];
      soff[k] = c >= 0 ? static_cast<uint16_t>(c - b) : static_cast<uint16_t>(0xFFFF);
    }
  }
}

void free_sell(DevCsr& A) {
  if (A.sptr) cudaFree(A.sptr);
  if (A.scol) cudaFree(A.scol);
  if (A.sval) cudaFree(A.sval);
  if (A.sval32) cudaFree(A.sval32);
  if (A.sbase) cudaFree(A.sbase);
  if (A.soff) cudaFree(A.soff);
  A.sptr = A.scol = A.sbase = nullptr;
  A.soff = nullptr;
  A.sval = nullptr;
  A.sval32 = nullptr;
  A.nslices = 0;
  A.sell_nnz = 0;
}

// The 16-bit column offsets when every slice fits them; left null otherwise.
void build_sell_offsets(DevCsr& A, cudaStream_t st) {
  int* wide = nullptr;
  SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&wide), sizeof(int)));
  int hwide = 0;
  try {
    SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&A.sbase), sizeof(int) * A.nslices));
    SG_CUDA(cudaMemsetAsync(wide, 0, sizeof(int), st));
    sell_base_kernel<<<device_sm_count() * 8, kThreads, 0, st>>>(A.nslices, A.sptr, A.scol,
                                                                 A.sbase, wide);
    SG_LAUNCH_CHECK();
    SG_CUDA(cudaMemcpyAsync(&hwide, wide, sizeof(int), cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
    if (!hwide) {
      SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&A.soff), sizeof(uint16_t) * A.sell_nnz));
      sell_off_kernel<<<device_sm_count() * 8, kThreads, 0, st>>>(
          static_cast<int64_t>(A.nslices) * 32, A.sptr, A.scol, A.sbase, A.soff);
      SG_LAUNCH_CHECK();
      SG_CUDA(cudaStreamSynchronize(st));
    }
  } catch (...) {
    cudaFree(wide);
    throw;
  }
  cudaFree(wide);
  if (!A.soff) {
    cudaFree(A.sbase);
    A.sbase = nullptr;
  }
}

}  // namespace

void build_sell(DevCsr& A, cudaStream_t st) {
  free_sell(A);
  if (A.n <= 0 || A.nnz <= 0) return;
  const int nsl = static_cast<int>((static_cast<int64_t>(A.n) + 31) / 32);
  int* width = nullptr;
  SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&width), sizeof(int) * nsl));
  std::vector<int> hw(nsl);
  try {
    sell_width_kernel<<<device_sm_count() * 8, kThreads, 0, st>>>(A.n, nsl, A.rowptr, width);
    SG_LAUNCH_CHECK();
    SG_CUDA(cudaMemcpyAsync(hw.data(), width, sizeof(int) * nsl, cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    cudaFree(width);
    throw;
  }
  cudaFree(width);
  std::vector<int> hp(static_cast<size_t>(nsl) + 1);
  int64_t tot = 0;
  for (int q = 0; q < nsl; ++q) {
    hp[q] = static_cast<int>(tot < (int64_t(1) << 31) ? tot : 0);
    tot += hw[q];
  }
  // keep SELL only when the padding is modest and the offsets fit int32
  if (tot >= (int64_t(1) << 31) - 1 || tot > A.nnz + A.nnz / 5 + 32 * static_cast<int64_t>(nsl))
    return;
  hp[nsl] = static_cast<int>(tot);
  try {
    SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&A.sptr), sizeof(int) * (nsl + 1)));
    SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&A.scol), sizeof(int) * tot));
    SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&A.sval), sizeof(double) * tot));
    SG_CUDA(cudaMemcpyAsync(A.sptr, hp.data(), sizeof(int) * (nsl + 1), cudaMemcpyHostToDevice, st));
    A.nslices = nsl;
    A.sell_nnz = tot;
    const int64_t rows32 = static_cast<int64_t>(nsl) * 32;
    sell_fill_kernel<true><<<device_sm_count() * 8, kThreads, 0, st>>>(
        A.n, rows32, A.rowptr, A.colind, A.val, A.sptr, A.scol, A.sval);
    SG_LAUNCH_CHECK();
    SG_CUDA(cudaStreamSynchronize(st));  // the host offsets go out of scope
    build_sell_offsets(A, st);
  } catch (...) {
    free_sell(A);
    throw;
  }
}

void sell_refill_values(const DevCsr& A, cudaStream_t st) {
  if (!A.sptr) return;
  const int64_t rows32 = static_cast<int64_t>(A.nslices) * 32;
  sell_fill_kernel<false><<<device_sm_count() * 8, kThreads, 0, st>>>(
      A.n, rows32, A.rowptr, A.colind, A.val, A.sptr, nullptr, A.sval);
  SG_LAUNCH_CHECK();
}

namespace {

__global__ void colnorm_kernel(int n, const int* __restrict__ rowptr,
                               const double* __restrict__ val, double* __restrict__ d) {
  for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double ss = 0.0;
    for (int k = rowptr[r]; k < rowptr[r + 1]; ++k) ss = fma(val[k], val[k], ss);
    d[r] = ss > 0.0 ? 1.0 / sqrt(ss) : 1.0;
  }
}

__global__ void scale_cols_kernel(int64_t cnt, const int* __restrict__ col,
                                  const double* __restrict__ val,
                                  const double* __restrict__ d, double* __restrict__ out) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < cnt;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int c = col[k];
    out[k] = c >= 0 ? val[k] * d[c] : 0.0;
  }
}

__global__ void diag_kernel(int64_t n, const double* __restrict__ d,
                            const double* x, double* y, int div) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    y[i] = div ? x[i] / d[i] : x[i] * d[i];
}

}  // namespace

namespace {

// A grid barrier that cannot complete: it expects one block more than the
// grid has, so every block's bounded wait runs out and sets err.
__global__ void barrier_probe_kernel(unsigned* bar, int* err, uint64_t limit_ns) {
  grid_barrier(bar, gridDim.x + 1, err, limit_ns);
}

}  // namespace

bool probe_grid_barrier_timeout(uint64_t limit_ns, cudaStream_t st) {
  unsigned* bar = nullptr;
  SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&bar), 256));
  bool timed_out = false;
  try {
    SG_CUDA(cudaMemsetAsync(bar, 0, 256, st));
    int* err = reinterpret_cast<int*>(bar + 48);
    barrier_probe_kernel<<<2, 32, 0, st>>>(bar, err, limit_ns);
    SG_LAUNCH_CHECK();
    int host = 0;
    SG_CUDA(cudaMemcpyAsync(&host, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
    timed_out = host != 0;
  } catch (...) {
    cudaFree(bar);
    throw;
  }
  SG_CUDA(cudaFree(bar));
  return timed_out;
}

void column_scale_factors(const DevCsr& AT, double* d, cudaStream_t st) {
  colnorm_kernel<<<device_sm_count() * 8, kThreads, 0, st>>>(AT.n, AT.rowptr, AT.val, d);
  SG_LAUNCH_CHECK();
}

void scale_columns(const DevCsr& A, const double* d, DevCsr& E, cudaStream_t st) {
  const int g = device_sm_count() * 8;
  if (A.nnz) {
    scale_cols_kernel<<<g, kThreads, 0, st>>>(A.nnz, A.colind, A.val, d, E.val);
    SG_LAUNCH_CHECK();
  }
  if (A.sptr && E.sval) {
    scale_cols_kernel<<<g, kThreads, 0, st>>>(A.sell_nnz, A.scol, A.sval, d, E.sval);
    SG_LAUNCH_CHECK();
  }
}

void diag_apply(int64_t n, const double* d, const double* x, double* y, bool div,
                cudaStream_t st) {
  if (n <= 0) return;
  diag_kernel<<<device_sm_count() * 8, kThreads, 0, st>>>(n, d, x, y, div ? 1 : 0);
  SG_LAUNCH_CHECK();
}

int64_t prepass_red_doubles() { return ic_red_doubles(device_sm_count()); }

void arnoldi_step(const DevCsr& A, double* V, int64_t ld, int j, double* H,
                  int ldh, double* wn, double* red, int red_cap, unsigned* bar,
                  int* err, cudaStream_t st) {
  if (A.sptr && A.sval)
    launch_arnoldi_step<double, true>(A, A.sval, V, ld, j, H, ldh, wn, red, red_cap, bar, err, st);
  else
    launch_arnoldi_step<double, false>(A, A.val, V, ld, j, H, ldh, wn, red, red_cap, bar, err, st);
}

void arnoldi_step32(const DevCsr& A, float* V, int64_t ld, int j, double* H,
                    int ldh, double* wn, double* red, int red_cap, unsigned* bar,
                    int* err, cudaStream_t st) {
  if (A.sptr && A.sval32)
    launch_arnoldi_step<float, true>(A, A.sval32, V, ld, j, H, ldh, wn, red, red_cap, bar, err, st);
  else
    launch_arnoldi_step<float, false>(A, A.val32, V, ld, j, H, ldh, wn, red, red_cap, bar, err, st);
}

}  // namespace sg
