// Tensor-core block dot product for the FP32 basis: W = Q^T X (the BCGS
// projections of Alg. 4) on the 5th-generation tensor cores.
//
// Q (n x i) and X (n x s) are FP32 column-major, so Q^T and X^T are
// K-major operands (K = the n rows) of a tcgen05 MMA with M = 128 columns
// of Q per tile and N = s (rounded up to 16).  Each CTA reduces one range
// of rows for one 128-column tile:
//   * a producer warp (one lane) issues TMA loads of 32-row x 128 B tiles
//     (128-byte swizzle) into a 6-stage ring guarded by mbarriers, each as
//     soon as the MMAs of the stage's previous tile have completed; the
//     split results live in a separate 2-slot ring (the X remainder in
//     shared memory, Q's hi/lo in tensor memory), so the load ring only
//     holds raw tiles and keeps ~4 of them in flight;
//   * warps 0-3, the owners of tensor-memory lanes 0-127, read one 128 B
//     row of the Q tile each (32 values of one column of Q), split it into
//     a TF32 "hi" part (low 13 mantissa bits cleared) and the exact FP32
//     remainder "lo", and store both into tensor memory, where the MMA
//     takes its A operand: shared memory then carries Q once (the TMA
//     write and this read) instead of three more times;
//   * warps 4-7 write the X tile's FP32 remainder beside it in shared
//     memory; the raw tile itself serves as the hi part, because the tensor
//     core reads a TF32 operand from the top 19 bits of each 32-bit word
//     (measured on this chip: the same products as an explicit split);
//     the eight split warps signal a per-stage mbarrier and go on to the
//     next tile;
//   * an MMA warp (one lane) issues tcgen05.mma.kind::tf32 for
//     hi*hi + lo*hi + hi*lo (the low*low term is below FP32 rounding), with
//     the FP32 accumulator in tensor memory, and commits each stage's MMAs
//     to an mbarrier that frees the stage;
//   * the accumulator is read back with tcgen05.ld and written as one
//     split partial; the fixed-order split reduction is the SIMT path's.
// Shared-memory traffic per 32-row tile at i = s = 107 is ~130 KB (TMA
// writes, the two splits, the MMA's three reads of X) where the version with
// both splits in shared memory moved ~210 KB: shared-memory bandwidth, not
// HBM, bounded that version.
// Every wait is bounded: on timeout the kernel records an error code,
// drains its own copies, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "k_tc_common.cuh"
#include "sg_internal.h"

namespace sg {

namespace {

using namespace tc;

constexpr int kBM = 128;          // MMA M: columns of Q per tile
constexpr int kBK = 32;           // rows per stage: 32 FP32 = one 128 B row
constexpr int kStages = 6;        // load ring (Q tile + X tile)
constexpr int kSide = 2;          // split ring (X remainder, Q hi/lo in TMEM)
constexpr int kSplit = 256;       // 8 warps split tiles; warps 0-3 own TMEM lanes
constexpr int kThreads = kSplit + 64;  // + the TMA producer warp, the MMA warp
constexpr int kMaxN = 128;        // s <= 128 per launch
constexpr uint32_t kTmemCols = 256;    // accumulator 0..127, Q hi/lo slots from 128
constexpr uint32_t kSlot0 = 128;       // split slot p: hi at 128 + 64 p, lo at + 32

struct __align__(8) TcShared {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t split[kSide];
  uint64_t sfree[kSide];
  uint64_t done;
  uint32_t tmem_base;
  int fail;
};

// grid: (tiles of 128 Q columns, 1, splits); block: 320 threads
__global__ void __launch_bounds__(kThreads, 1)
tc_dot_kernel(const __grid_constant__ CUtensorMap mapQ,
              const __grid_constant__ CUtensorMap mapX, int64_t n, int M, int N,
              int BN, int64_t rows_per_split, double* __restrict__ part,
              int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  // 1024-byte aligned tiles: per stage A (128 x 128 B) and B (BN x 128 B),
  // then kSide B_lo slots (BN x 128 B)
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
  const int a_bytes = kBM * kBK * 4;
  const int b_bytes = BN * kBK * 4;
  const int stage_bytes = a_bytes + b_bytes;
  __shared__ TcShared sh;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int m0 = blockIdx.x * kBM;
  const int64_t k0 = static_cast<int64_t>(blockIdx.z) * rows_per_split;
  const int64_t k1 = (k0 + rows_per_split < n) ? k0 + rows_per_split : n;
  const int nk = static_cast<int>((k1 - k0 + kBK - 1) / kBK);
  const uint32_t idesc = idesc_tf32(kBM, BN);

  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) {
      mbar_init(&sh.full[q], 1);
      mbar_init(&sh.empty[q], 1);
    }
    for (int p = 0; p < kSide; ++p) {
      mbar_init(&sh.split[p], kSplit);
      mbar_init(&sh.sfree[p], 1);
    }
    mbar_init(&sh.done, 1);
    sh.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh.tmem_base;

  auto stA = [&](int q) { return base + q * stage_bytes; };
  auto stB = [&](int q) { return base + q * stage_bytes + a_bytes; };
  auto stBlo = [&](int p) { return base + kStages * stage_bytes + p * b_bytes; };

  if (warp == kSplit / 32) {
    // ---------------------------------------------- TMA producer (one lane)
    if ((tid & 31) == 0) {
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        if (*reinterpret_cast<volatile int*>(&sh.fail)) break;
        const int q = kb % kStages;
        if (kb >= kStages &&
            !mbar_wait(&sh.empty[q], static_cast<uint32_t>(((kb / kStages) - 1) & 1))) {
          sh.fail = 1;
          break;
        }
        mbar_expect_tx(&sh.full[q], static_cast<uint32_t>(a_bytes + b_bytes));
        const int x = static_cast<int>(k0 + static_cast<int64_t>(kb) * kBK);
        tma_load_2d(stA(q), &mapQ, &sh.full[q], x, m0);
        tma_load_2d(stB(q), &mapX, &sh.full[q], x, 0);
        issued = kb + 1;
      }
      if (*reinterpret_cast<volatile int*>(&sh.fail)) {
        // let this CTA's loads still in flight land (each is the latest
        // use of its stage, so its parity identifies it)
        for (int kb = (issued > kStages ? issued - kStages : 0); kb < issued; ++kb)
          mbar_wait(&sh.full[kb % kStages], static_cast<uint32_t>((kb / kStages) & 1));
      }
    }
  } else if (warp == kSplit / 32 + 1) {
    // ---------------------------------------------- MMA issuer (one lane)
    if ((tid & 31) == 0) {
      for (int kb = 0; kb < nk; ++kb) {
        const int q = kb % kStages, p = kb % kSide;
        if (*reinterpret_cast<volatile int*>(&sh.fail)) break;
        if (!mbar_wait(&sh.split[p], static_cast<uint32_t>((kb / kSide) & 1))) {
          sh.fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = tmem + kSlot0 + static_cast<uint32_t>(p * 64), al = ah + 32;
        const uint64_t b = sdesc(smem_u32(stB(q))), bl = sdesc(smem_u32(stBlo(p)));
#pragma unroll
        for (int k8 = 0; k8 < kBK / 8; ++k8) {  // K = 8 TF32 = 32 bytes per MMA
          const uint64_t adv = static_cast<uint64_t>((k8 * 32) >> 4);
          const uint32_t ak = static_cast<uint32_t>(k8 * 8);
          mma_tf32_tmem_a(tmem, ah + ak, b + adv, idesc, (kb > 0 || k8 > 0) ? 1u : 0u);
          mma_tf32_tmem_a(tmem, al + ak, b + adv, idesc, 1u);
          mma_tf32_tmem_a(tmem, ah + ak, bl + adv, idesc, 1u);
        }
        mma_commit(&sh.empty[q]);  // frees the stage for the producer
        mma_commit(&sh.sfree[p]);  // and the split slot for the split warps
      }
      // completes once every MMA issued above has (the accumulator is read,
      // or the tensor memory freed, only after it)
      mma_commit(&sh.done);
    }
  } else {
    // ---------------------------------------------- split (8 warps)
    for (int kb = 0; kb < nk; ++kb) {
      const int q = kb % kStages, p = kb % kSide;
      bool bad = *reinterpret_cast<volatile int*>(&sh.fail) != 0;
      if (!bad && !mbar_wait(&sh.full[q], static_cast<uint32_t>((kb / kStages) & 1))) {
        sh.fail = 1;
        bad = true;
      }
      // the split slot's previous tile has been consumed by its MMAs
      if (!bad && kb >= kSide &&
          !mbar_wait(&sh.sfree[p], static_cast<uint32_t>(((kb / kSide) - 1) & 1))) {
        sh.fail = 1;
        bad = true;
      }
      // the tensor-memory stores below are warp-collective: leave together
      if (__any_sync(0xffffffffu, bad)) break;
      if (warp < 4) {
        // row tid of the Q tile: 16-byte chunk c sits at chunk c ^ (row & 7)
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const float4* row = reinterpret_cast<const float4*>(stA(q) + tid * 128);
        float v[32];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 f = row[c ^ (tid & 7)];
          v[4 * c] = f.x; v[4 * c + 1] = f.y; v[4 * c + 2] = f.z; v[4 * c + 3] = f.w;
        }
        uint32_t h[32], l[32];
        split32(v, h, l);
        const uint32_t ta = tmem + (static_cast<uint32_t>(warp * 32) << 16) + kSlot0 +
                            static_cast<uint32_t>(p * 64);
        tmem_st32(ta, h);
        tmem_st32(ta + 32, l);
        tmem_st_wait();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      } else {
        split_lo_tf32<kSplit - 128>(reinterpret_cast<const float4*>(stB(q)),
                                    reinterpret_cast<float4*>(stBlo(p)), b_bytes / 16,
                                    tid - 128);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      mbar_arrive(&sh.split[p]);
    }
    // (twice the limit: after a failure the MMA warp may first spend one
    // limit on a stage that never came)
    if (warp < 4 && !mbar_wait(&sh.done, 0, 2 * kWaitNs)) sh.fail = 1;
  }
  __syncthreads();
  const bool good = !sh.fail;
  if (!good) {
    if (tid == 0) atomicExch(err, 1);
  } else if (warp < 4) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // TMEM lane = accumulator row m (warp w owns lanes 32w..32w+31)
    const int row = warp * 32 + (tid & 31);
    const int m = m0 + row;
    double* P = part + static_cast<int64_t>(blockIdx.z) * M * N;
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
            "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
            "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int nc = c0 + j;
          if (nc < N) P[m + static_cast<int64_t>(nc) * M] = static_cast<double>(__uint_as_float(v[j]));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
}

__device__ int g_tc_err;  // set to 1 by a CTA whose wait ran out

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool make_map(CUtensorMap* map, const float* base, int64_t rows, int64_t cols,
              int64_t ld, int box_cols) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(cols)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * sizeof(float)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kBK), static_cast<cuuint32_t>(box_cols)};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace

namespace {

// An mbarrier nothing arrives on: the bounded wait runs out and sets err.
__global__ void mbarrier_probe_kernel(int* err, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0u, limit_ns)) atomicExch(err, 1);
}

}  // namespace

bool probe_mbarrier_timeout(uint64_t limit_ns, cudaStream_t st) {
  int* err = nullptr;
  SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&err), sizeof(int)));
  bool timed_out = false;
  try {
    SG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    mbarrier_probe_kernel<<<1, 32, 0, st>>>(err, limit_ns);
    SG_LAUNCH_CHECK();
    int host = 0;
    SG_CUDA(cudaMemcpyAsync(&host, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
    timed_out = host != 0;
  } catch (...) {
    cudaFree(err);
    throw;
  }
  SG_CUDA(cudaFree(err));
  return timed_out;
}

bool tc_dot_supported(int64_t n, const float* Q, int64_t ldq, int i, const float* X,
                      int64_t ldx, int s) {
  if (n < 8 * kBK || i < 1 || s < 1 || s > kMaxN) return false;
  if ((reinterpret_cast<uintptr_t>(Q) | reinterpret_cast<uintptr_t>(X)) & 15) return false;
  if (((ldq * 4) & 15) || ((ldx * 4) & 15)) return false;
  if (n > (int64_t(1) << 31) - 1) return false;
  return encode_fn() != nullptr;
}

int64_t tc_dot_part_size(int64_t n, int i, int s) {
  const int tiles = (i + kBM - 1) / kBM;
  // one wave: a CTA holds a whole SM (shared memory, 512 TMEM columns)
  int64_t S = static_cast<int64_t>(device_sm_count()) / tiles;
  const int64_t maxS = n / (8 * kBK);
  if (S > maxS) S = maxS;
  if (S < 1) S = 1;
  return S * i * s;
}

int* tc_err_flag() {
  static int* ptr[64] = {};
  static std::mutex mu;
  int dev = 0;
  SG_CUDA(cudaGetDevice(&dev));
  SG_REQUIRE(dev >= 0 && dev < 64, SG_ECUDA, "device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    SG_CUDA(cudaGetSymbolAddress(&p, g_tc_err));
    ptr[dev] = static_cast<int*>(p);
  }
  return ptr[dev];
}

void tc_check_error(cudaStream_t st) {
  int* f = tc_err_flag();
  int host = 0;
  SG_CUDA(cudaMemcpyAsync(&host, f, sizeof(int), cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  if (host) {
    SG_CUDA(cudaMemsetAsync(f, 0, sizeof(int), st));
    throw Error(SG_ECUDA, "tensor-core block dot: a bounded wait ran out");
  }
}

void tc_dot(int64_t n, const float* Q, int64_t ldq, int i, const float* X, int64_t ldx,
            int s, double* part, int64_t part_cap, int* nsplit, cudaStream_t st) {
  int* err = tc_err_flag();
  const int BN = (s + 15) / 16 * 16;
  const int tiles = (i + kBM - 1) / kBM;
  // one wave: a CTA holds a whole SM (shared memory, 512 TMEM columns)
  int64_t S = static_cast<int64_t>(device_sm_count()) / tiles;
  const int64_t maxS = n / (8 * kBK);
  if (S > maxS) S = maxS;
  if (S < 1) S = 1;
  int64_t rows = (n + S - 1) / S;
  rows = (rows + kBK - 1) / kBK * kBK;
  S = (n + rows - 1) / rows;
  SG_REQUIRE(S * i * s <= part_cap, SG_EINVAL, "tc_dot: workspace too small");
  CUtensorMap mq, mx;
  SG_REQUIRE(make_map(&mq, Q, n, i, ldq, kBM) && make_map(&mx, X, n, s, ldx, BN), SG_ECUDA,
             "cuTensorMapEncodeTiled failed");
  auto smem_for = [](int bn) {
    return kStages * (kBM * kBK * 4 + bn * kBK * 4) + kSide * bn * kBK * 4 + 1024;
  };
  // the largest size for every s: one CTA per SM
  const int smem = smem_for(kMaxN);
  static bool configured = false;
  if (!configured) {
    SG_CUDA(cudaFuncSetAttribute(tc_dot_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_for(kMaxN)));
    configured = true;
  }
  dim3 grid(tiles, 1, static_cast<unsigned>(S));
  tc_dot_kernel<<<grid, kThreads, smem, st>>>(mq, mx, n, i, s, BN, rows, part, err);
  SG_LAUNCH_CHECK();
  *nsplit = static_cast<int>(S);
}

}  // namespace sg
