// Tensor-core block dot product for the FP32 basis: W = Q^T X (the BCGS
// projections of Alg. 4) on the 5th-generation tensor cores.
//
// Q (n x i) and X (n x s) are FP32 column-major, so Q^T and X^T are
// K-major operands (K = the n rows) of a tcgen05 MMA with M = 128 columns
// of Q per tile and N = s (rounded up to 16).  Each CTA reduces one range
// of rows for one 128-column tile, 64 rows (K) per step:
//   * TMA streams 128-byte lines at only ~4.7 TB/s on this chip and
//     256-byte lines at the full HBM rate.  Q never needs the MMA's swizzled
//     shared-memory layout (it reaches the MMA through tensor memory), so
//     its tile arrives as one unswizzled 64-row x 128-column box (a 256-byte
//     line per column of Q) in a 2-slot ring; X, the shared-memory operand,
//     arrives as two 128-byte-swizzled 32-row boxes per step in a 3-slot
//     ring.  One producer lane issues both.
//   * warps 0-3 own tensor-memory lanes 0-127, one column of Q each: a warp
//     first permutes its 32 rows' 16-byte chunks in place (chunk c of row m
//     to c ^ (m & 15), read and written two rows per instruction without
//     bank conflicts), then each thread reads its row conflict-free, splits
//     it into a TF32 hi part (low 13 mantissa bits cleared) and the exact
//     FP32 remainder, and stores both into tensor memory; the Q slot is
//     freed at once;
//   * warps 4-7 write X's FP32 remainder beside it (the raw tile is its own
//     hi part: kind::tf32 reads the top 19 bits of each 32-bit word); the
//     split results live in a 2-slot ring freed by the MMAs;
//   * an MMA warp (one lane) issues tcgen05.mma.kind::tf32 for
//     hi*hi + lo*hi + hi*lo (the low*low term is below FP32 rounding), A
//     from tensor memory, B from shared memory, with the FP32 accumulator
//     in tensor memory, and commits each step to the mbarriers that free
//     its X slot and split slot;
//   * the accumulator is read back with tcgen05.ld and written as one
//     split partial; the fixed-order split reduction is the SIMT path's.
// Every wait is bounded: on timeout the kernel records an error code,
// drains its own copies, frees its tensor memory and returns.
#include <atomic>
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "k_tc_common.cuh"
#include "sg_internal.h"

namespace sg {

namespace {

using namespace tc;

constexpr int kBM = 128;          // MMA M: columns of Q per tile
constexpr int kBK = 64;           // rows per step: two 32-row MMA K blocks
constexpr int kAStages = 2;       // Q ring (unswizzled 64 x 128 boxes)
constexpr int kBStages = 3;       // X ring (two swizzled 32-row boxes each)
constexpr int kSide = 2;          // split ring (X remainder, Q hi/lo in TMEM)
constexpr int kSplit = 256;       // 8 warps split tiles; warps 0-3 own TMEM lanes
constexpr int kThreads = kSplit + 64;  // + the TMA producer warp, the MMA warp
constexpr int kMaxN = 128;        // s <= 128 per launch
constexpr uint32_t kTmemCols = 512;    // accumulator 0..127, split slots from 128
constexpr uint32_t kSlot0 = 128;       // slot p: Q hi at 128 + 128 p, lo at + 64

struct __align__(8) TcShared {
  uint64_t afull[kAStages];
  uint64_t afree[kAStages];
  uint64_t bfull[kBStages];
  uint64_t bfree[kBStages];
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
  // 1024-byte aligned: kAStages Q slots (128 x 256 B), kBStages X slots
  // (two BN x 128 B boxes), kSide remainder slots (two BN x 128 B blocks)
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
  constexpr int a_bytes = kBM * kBK * 4;  // 32 KB
  const int b_half = BN * 32 * 4;         // one 32-row X box
  const int b_bytes = 2 * b_half;
  __shared__ TcShared sh;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int m0 = blockIdx.x * kBM;
  const int64_t k0 = static_cast<int64_t>(blockIdx.z) * rows_per_split;
  const int64_t k1 = (k0 + rows_per_split < n) ? k0 + rows_per_split : n;
  const int nk = static_cast<int>((k1 - k0 + kBK - 1) / kBK);
  const uint32_t idesc = idesc_tf32(kBM, BN);

  if (tid == 0) {
    for (int q = 0; q < kAStages; ++q) {
      mbar_init(&sh.afull[q], 1);
      mbar_init(&sh.afree[q], 128);
    }
    for (int q = 0; q < kBStages; ++q) {
      mbar_init(&sh.bfull[q], 1);
      mbar_init(&sh.bfree[q], 1);
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

  auto stA = [&](int q) { return base + q * a_bytes; };
  auto stB = [&](int q) { return base + kAStages * a_bytes + q * b_bytes; };
  auto stBlo = [&](int p) {
    return base + kAStages * a_bytes + kBStages * b_bytes + p * b_bytes;
  };
  auto failed = [&]() { return *reinterpret_cast<volatile int*>(&sh.fail) != 0; };

  if (warp == kSplit / 32) {
    // ---------------------------------------------- TMA producer (one lane)
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < nk; ++kb) {
        if (failed()) break;
        const int qa = kb % kAStages, qb = kb % kBStages;
        if ((kb >= kAStages &&
             !mbar_wait(&sh.afree[qa], static_cast<uint32_t>(((kb / kAStages) - 1) & 1))) ||
            (kb >= kBStages &&
             !mbar_wait(&sh.bfree[qb], static_cast<uint32_t>(((kb / kBStages) - 1) & 1)))) {
          sh.fail = 1;
          break;
        }
        const int x = static_cast<int>(k0 + static_cast<int64_t>(kb) * kBK);
        mbar_expect_tx(&sh.afull[qa], static_cast<uint32_t>(a_bytes));
        tma_load_2d(stA(qa), &mapQ, &sh.afull[qa], x, m0);
        mbar_expect_tx(&sh.bfull[qb], static_cast<uint32_t>(b_bytes));
        tma_load_2d(stB(qb), &mapX, &sh.bfull[qb], x, 0);
        tma_load_2d(stB(qb) + b_half, &mapX, &sh.bfull[qb], x + 32, 0);
        issued = kb + 1;
      }
      if (failed()) {
        // let this CTA's loads still in flight land (each is the latest use
        // of its slot, so its parity identifies it)
        for (int kb = (issued > kAStages ? issued - kAStages : 0); kb < issued; ++kb)
          mbar_wait(&sh.afull[kb % kAStages], static_cast<uint32_t>((kb / kAStages) & 1));
        for (int kb = (issued > kBStages ? issued - kBStages : 0); kb < issued; ++kb)
          mbar_wait(&sh.bfull[kb % kBStages], static_cast<uint32_t>((kb / kBStages) & 1));
      }
    }
  } else if (warp == kSplit / 32 + 1) {
    // ---------------------------------------------- MMA issuer (one lane)
    if (lane == 0) {
      for (int kb = 0; kb < nk; ++kb) {
        const int qb = kb % kBStages, p = kb % kSide;
        if (failed()) break;
        if (!mbar_wait(&sh.split[p], static_cast<uint32_t>((kb / kSide) & 1))) {
          sh.fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = tmem + kSlot0 + static_cast<uint32_t>(p * 128), al = ah + 64;
#pragma unroll
        for (int u = 0; u < 2; ++u) {  // 32-row K blocks
          const uint64_t b = sdesc(smem_u32(stB(qb) + u * b_half));
          const uint64_t bl = sdesc(smem_u32(stBlo(p) + u * b_half));
#pragma unroll
          for (int k8 = 0; k8 < 4; ++k8) {  // K = 8 TF32 = 32 bytes per MMA
            const uint64_t adv = static_cast<uint64_t>((k8 * 32) >> 4);
            const uint32_t ak = static_cast<uint32_t>(u * 32 + k8 * 8);
            mma_tf32_tmem_a(tmem, ah + ak, b + adv, idesc, (kb > 0 || u > 0 || k8 > 0) ? 1u : 0u);
            mma_tf32_tmem_a(tmem, al + ak, b + adv, idesc, 1u);
            mma_tf32_tmem_a(tmem, ah + ak, bl + adv, idesc, 1u);
          }
        }
        mma_commit(&sh.bfree[qb]);  // frees the X slot for the producer
        mma_commit(&sh.sfree[p]);   // and the split slot for the split warps
      }
      // completes once every MMA issued above has (the accumulator is read,
      // or the tensor memory freed, only after it)
      mma_commit(&sh.done);
    }
  } else {
    // ---------------------------------------------- split (8 warps)
    for (int kb = 0; kb < nk; ++kb) {
      const int qa = kb % kAStages, qb = kb % kBStages, p = kb % kSide;
      bool bad = failed();
      if (!bad) {
        const bool ok =
            (warp < 4 ? mbar_wait(&sh.afull[qa], static_cast<uint32_t>((kb / kAStages) & 1))
                      : mbar_wait(&sh.bfull[qb], static_cast<uint32_t>((kb / kBStages) & 1))) &&
            // the split slot's previous step has been consumed by its MMAs
            (kb < kSide ||
             mbar_wait(&sh.sfree[p], static_cast<uint32_t>(((kb / kSide) - 1) & 1)));
        if (!ok) {
          sh.fail = 1;
          bad = true;
        }
      }
      // the tensor-memory stores below are warp-collective: leave together
      if (__any_sync(0xffffffffu, bad)) break;
      if (warp < 4) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // this warp's rows 32w .. 32w + 31 of the Q slot, 256 B each:
        // chunk c of row m moves to c ^ (m & 15), two rows per instruction
        float4* rows = reinterpret_cast<float4*>(stA(qa)) + warp * 32 * 16;
#pragma unroll 4
        for (int pr = 0; pr < 16; ++pr) {
          const int r = 2 * pr + (lane >> 4), c = lane & 15;
          const float4 v = rows[r * 16 + c];
          __syncwarp();
          rows[r * 16 + (c ^ ((warp * 32 + r) & 15))] = v;
          __syncwarp();
        }
        // thread tid now reads its row: chunk c at c ^ (tid & 15)
        const float4* row = reinterpret_cast<const float4*>(stA(qa)) + tid * 16;
        const uint32_t ta = tmem + (static_cast<uint32_t>(warp * 32) << 16) + kSlot0 +
                            static_cast<uint32_t>(p * 128);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          float v[32];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 f = row[(half * 8 + c) ^ (tid & 15)];
            v[4 * c] = f.x; v[4 * c + 1] = f.y; v[4 * c + 2] = f.z; v[4 * c + 3] = f.w;
          }
          uint32_t h[32], l[32];
          split32(v, h, l);
          tmem_st32(ta + static_cast<uint32_t>(half * 32), h);
          tmem_st32(ta + 64 + static_cast<uint32_t>(half * 32), l);
        }
        tmem_st_wait();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&sh.afree[qa]);  // the Q slot is free for the producer
      } else {
        split_lo_tf32<kSplit - 128>(reinterpret_cast<const float4*>(stB(qb)),
                                    reinterpret_cast<float4*>(stBlo(p)), b_bytes / 16,
                                    tid - 128);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      mbar_arrive(&sh.split[p]);
    }
    // (twice the limit: after a failure the MMA warp may first spend one
    // limit on a step that never came)
    if (warp < 4 && !mbar_wait(&sh.done, 0, 2 * kWaitNs)) sh.fail = 1;
  }
  __syncthreads();
  const bool good = !sh.fail;
  if (!good) {
    if (tid == 0) atomicExch(err, 1);
  } else if (warp < 4) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // TMEM lane = accumulator row m (warp w owns lanes 32w..32w+31)
    const int row = warp * 32 + lane;
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
              int64_t ld, int box_rows, int box_cols, CUtensorMapSwizzle swz) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(cols)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * sizeof(float)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_rows), static_cast<cuuint32_t>(box_cols)};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
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

// Launches of this file's tensor-core kernels since the last check: the
// check reads the device's error flag (a synchronising copy) only after
// one.  The flag stays set until read, so a timeout is reported by a later
// check even if another thread's check consumed the count.
std::atomic<int> tc_check_error_pending{0};

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
  if (tc_check_error_pending.exchange(0) == 0) return;
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
  SG_REQUIRE(make_map(&mq, Q, n, i, ldq, kBK, kBM, CU_TENSOR_MAP_SWIZZLE_NONE) &&
                 make_map(&mx, X, n, s, ldx, 32, BN, CU_TENSOR_MAP_SWIZZLE_128B),
             SG_ECUDA, "cuTensorMapEncodeTiled failed");
  auto smem_for = [](int bn) {
    return kAStages * kBM * kBK * 4 + (kBStages + kSide) * bn * kBK * 4 + 1024;
  };
  // the largest size for every s: one CTA per SM
  const int smem = smem_for(kMaxN);
  ensure_dynamic_smem(reinterpret_cast<const void*>(tc_dot_kernel), smem);
  dim3 grid(tiles, 1, static_cast<unsigned>(S));
  tc_dot_kernel<<<grid, kThreads, smem, st>>>(mq, mx, n, i, s, BN, rows, part, err);
  tc_check_error_pending.fetch_add(1);
  SG_LAUNCH_CHECK();
  *nsplit = static_cast<int>(S);
}

}  // namespace sg
