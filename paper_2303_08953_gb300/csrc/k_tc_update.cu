// Tensor-core block update for the FP32 basis: X = beta X + alpha Q W
// (the BCGS updates and the CholQR triangular products of Alg. 4).
//
// D (128 rows of X x s) = Q (128 rows x i) . W (i x s) on tcgen05 (kind::tf32,
// FP32 accumulator in tensor memory).  Q is column-major, so TMA delivers
// its tile row-contiguous: one unswizzled 128-row x 32-column box per
// stage, a 512-byte line per column of Q (TMA streams 128-byte lines at
// only ~4.7 TB/s on this chip, 256- and 512-byte lines at the full HBM
// rate).  Each split thread owns one row of the tile (its tensor-memory
// lane), gathers that row's 32 values from the box (a warp reads 128
// contiguous bytes per column: no bank conflicts) and stores the TF32 hi
// part and the FP32 remainder into tensor memory, where the MMA takes its A
// operand -- the transpose to the K-major layout costs no shared-memory
// writes.  W is tiny: a prologue kernel writes its hi part and remainder as
// FP32 arrays that TMA loads as K-major tiles (128-byte swizzle, the MMA's
// B operand).  When all of W's chunks fit beside two Q stages and the X
// tile, they are loaded once per CTA and stay resident; otherwise each
// stage carries its chunk (re-fetching W per tile costs ~2.5x the TMA lines
// of the tile's own data).  hi*hi + lo*hi + hi*lo is accumulated.
//
// Persistent and warp-specialised: one CTA per SM walks 128-row tiles;
//   warp 8 (one lane) issues the TMA loads of a ring of up to 3 stages,
//   warps 4-7 split each Q tile into hi/lo in tensor memory,
//   warp 9 (one lane) issues the MMAs into one of two TMEM accumulators,
//   warps 0-3 (the TMEM lane owners) read an accumulator back while the
//   next tile accumulates into the other.  The tile of X goes through
//   shared memory both ways: a TMA load (beta != 0) issued as soon as the
//   previous tile's store has read the buffer, the update in place, and a
//   TMA store, so HBM sees whole 512-byte column segments in flight instead
//   of the epilogue threads' dependent loads.
// Every wait is time-bounded; a timeout records an error flag, the roles
// stop, in-flight copies and MMAs are drained and the TMEM is freed.
#include <atomic>
#include <cudaTypedefs.h>

#include <mutex>

#include "k_tc_common.cuh"
#include "sg_internal.h"

namespace sg {

namespace {

using namespace tc;

constexpr int kRows = 128;      // rows of X per tile (MMA M)
constexpr int kKC = 32;         // columns of Q (K) per stage
constexpr int kStages = 3;
constexpr int kThreads = 320;   // 10 warps
constexpr int kMaxN = 128;
constexpr uint32_t kTmemCols = 512;  // accumulators at 0 and 128, Q hi/lo slots
constexpr uint32_t kSlot0 = 256;     // stage q: hi at 256 + 64 q, lo at + 32
constexpr int kSmemBytes = 230400;   // dynamic shared memory (+1 KB alignment slack)

struct __align__(8) UpdShared {
  uint64_t full[kStages];
  uint64_t split[kStages];
  uint64_t empty[kStages];
  uint64_t accf[2];
  uint64_t acce[2];
  uint64_t xfull;
  uint64_t wfull;  // the resident W (one load per CTA)
  uint64_t done;
  uint32_t tmem_base;
  int fail;
  int epi_stop;  // the epilogue warps' common stop decision
};

__global__ void __launch_bounds__(kThreads, 1)
tc_update_kernel(const __grid_constant__ CUtensorMap mapQ,
                 const __grid_constant__ CUtensorMap mapWh,
                 const __grid_constant__ CUtensorMap mapWl,
                 const __grid_constant__ CUtensorMap mapX, int64_t n, int i, int s,
                 int BN, float alpha, float beta, int nst, int wres,
                 int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
  constexpr int a_bytes = kRows * kKC * 4;  // 16 KB: one 128 x 32 box of Q
  const int b_bytes = BN * kKC * 4;
  // nst stages of the Q ring (<= kStages).  wres: W's hi/lo chunks for
  // all K stay resident (loaded once per CTA) ahead of a Q-only ring;
  // otherwise every stage carries its chunk of W hi and lo as well.
  const int stage_bytes = wres ? a_bytes : a_bytes + 2 * b_bytes;
  __shared__ UpdShared sh;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int64_t tiles = (n + kRows - 1) / kRows;
  const int KC = (i + kKC - 1) / kKC;
  const int my_tiles = static_cast<int>((tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
  const int total = my_tiles * KC;  // (tile, k-chunk) pairs of this CTA
  const uint32_t idesc = idesc_tf32(kRows, BN);

  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) {
      mbar_init(&sh.full[q], 1);
      mbar_init(&sh.split[q], 128);
      mbar_init(&sh.empty[q], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.accf[b], 1);
      mbar_init(&sh.acce[b], 128);
    }
    mbar_init(&sh.xfull, 1);
    mbar_init(&sh.wfull, 1);
    mbar_init(&sh.done, 1);
    sh.fail = 0;
    sh.epi_stop = 0;
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

  const int KCr = wres ? KC : 0;  // resident W chunks
  unsigned char* ring = base + KCr * 2 * b_bytes;
  auto stRaw = [&](int q) { return ring + q * stage_bytes; };
  // W hi / lo of stage q (its chunk kc when resident)
  auto stB = [&](int q, int kc) {
    return wres ? base + kc * 2 * b_bytes : ring + q * stage_bytes + a_bytes;
  };
  auto stBlo = [&](int q, int kc) { return stB(q, kc) + b_bytes; };
  float* xs = reinterpret_cast<float*>(ring + nst * stage_bytes);  // [BN][128]
  const uint32_t x_bytes = static_cast<uint32_t>(kRows * BN * 4);
  auto fail_now = [&]() {
    sh.fail = 1;
    atomicExch(err, 1);
  };

  if (warp == 8) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      if (wres && total > 0) {
        // every chunk of W hi and lo, once (2 KC boxes of BN 128-byte lines)
        mbar_expect_tx(&sh.wfull, static_cast<uint32_t>(KC * 2 * b_bytes));
        for (int kc = 0; kc < KC; ++kc) {
          tma_load_2d(stB(0, kc), &mapWh, &sh.wfull, kc * kKC, 0);
          tma_load_2d(stBlo(0, kc), &mapWl, &sh.wfull, kc * kKC, 0);
        }
      }
      int issued = 0;
      for (int c = 0; c < total; ++c) {
        if (*reinterpret_cast<volatile int*>(&sh.fail)) break;
        const int q = c % nst;
        if (c >= nst &&
            !mbar_wait(&sh.empty[q], static_cast<uint32_t>(((c / nst) - 1) & 1))) {
          fail_now();
          break;
        }
        const int lt = c / KC, kc = c % KC;
        const int64_t row0 = (static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(lt) * gridDim.x) * kRows;
        mbar_expect_tx(&sh.full[q], static_cast<uint32_t>(wres ? a_bytes : a_bytes + 2 * b_bytes));
        tma_load_2d(stRaw(q), &mapQ, &sh.full[q], static_cast<int>(row0), kc * kKC);
        if (!wres) {
          tma_load_2d(stB(q, kc), &mapWh, &sh.full[q], kc * kKC, 0);
          tma_load_2d(stBlo(q, kc), &mapWl, &sh.full[q], kc * kKC, 0);
        }
        ++issued;
      }
      if (*reinterpret_cast<volatile int*>(&sh.fail)) {
        // drain the loads still in flight (the latest use of each stage,
        // and the resident W)
        for (int c = (issued > nst ? issued - nst : 0); c < issued; ++c)
          mbar_wait(&sh.full[c % nst], static_cast<uint32_t>((c / nst) & 1));
        if (wres && total > 0) mbar_wait(&sh.wfull, 0);
      }
    }
  } else if (warp >= 4 && warp < 8) {
    // ------------------------------------------------ hi/lo split of Q
    const int st = tid - 128;
    for (int c = 0; c < total; ++c) {
      const int q = c % nst;
      bool bad = *reinterpret_cast<volatile int*>(&sh.fail) != 0;
      if (!bad && !mbar_wait(&sh.full[q], static_cast<uint32_t>((c / nst) & 1))) {
        fail_now();
        bad = true;
      }
      // the tensor-memory stores below are warp-collective: leave together
      if (__any_sync(0xffffffffu, bad)) break;
      // element (row st, column k) of the Q box sits at k * 128 + st (one
      // 512-byte line per column of Q): a warp reads 128 contiguous bytes
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const float* raw = reinterpret_cast<const float*>(stRaw(q));
      float v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = raw[k * kRows + st];
      uint32_t h[32], l[32];
      split32(v, h, l);
      const uint32_t ta = tmem + (static_cast<uint32_t>((warp - 4) * 32) << 16) + kSlot0 +
                          static_cast<uint32_t>(q * 64);
      tmem_st32(ta, h);
      tmem_st32(ta + 32, l);
      tmem_st_wait();
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&sh.split[q]);
    }
  } else if (warp == 9) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      for (int lt = 0; lt < my_tiles && !*reinterpret_cast<volatile int*>(&sh.fail); ++lt) {
        const int b = lt & 1;
        if (lt >= 2 &&
            !mbar_wait(&sh.acce[b], static_cast<uint32_t>(((lt / 2) - 1) & 1))) {
          fail_now();
          break;
        }
        const uint32_t dt = tmem + static_cast<uint32_t>(b * 128);
        bool ok = true;
        for (int kc = 0; kc < KC; ++kc) {
          const int c = lt * KC + kc;
          const int q = c % nst;
          if ((c == 0 && wres && !mbar_wait(&sh.wfull, 0)) ||
              !mbar_wait(&sh.split[q], static_cast<uint32_t>((c / nst) & 1))) {
            fail_now();
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t ah = tmem + kSlot0 + static_cast<uint32_t>(q * 64), al = ah + 32;
          const uint64_t bh = sdesc(smem_u32(stB(q, kc))), bl = sdesc(smem_u32(stBlo(q, kc)));
#pragma unroll
          for (int k8 = 0; k8 < kKC / 8; ++k8) {  // K = 8 TF32 = 32 bytes per MMA
            const uint64_t adv = static_cast<uint64_t>((k8 * 32) >> 4);
            const uint32_t ak = static_cast<uint32_t>(k8 * 8);
            mma_tf32_tmem_a(dt, ah + ak, bh + adv, idesc, (kc > 0 || k8 > 0) ? 1u : 0u);
            mma_tf32_tmem_a(dt, al + ak, bh + adv, idesc, 1u);
            mma_tf32_tmem_a(dt, ah + ak, bl + adv, idesc, 1u);
          }
          mma_commit(&sh.empty[q]);
        }
        if (!ok) break;
        mma_commit(&sh.accf[b]);
      }
      mma_commit(&sh.done);  // every MMA issued above has completed
      if (!mbar_wait(&sh.done, 0)) fail_now();
    }
  } else {
    // ------------------------------------------------ epilogue (warps 0-3)
    auto row0_of = [&](int lt) {
      return (static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(lt) * gridDim.x) * kRows;
    };
    const bool load_x = beta != 0.0f;
    int x_issued = 0;        // (thread 0) X loads issued
    bool x_pending = false;  // (thread 0) one of them has not been waited for
    if (tid == 0 && load_x && my_tiles > 0) {
      mbar_expect_tx(&sh.xfull, x_bytes);
      tma_load_2d(xs, &mapX, &sh.xfull, static_cast<int>(row0_of(0)), 0);
      ++x_issued;
      x_pending = true;
    }
    const int r = warp * 32 + lane;  // this thread's row of the tile
    for (int lt = 0; lt < my_tiles; ++lt) {
      const int b = lt & 1;
      const bool ok = !*reinterpret_cast<volatile int*>(&sh.fail) &&
                      mbar_wait(&sh.accf[b], static_cast<uint32_t>((lt / 2) & 1)) &&
                      (!load_x || mbar_wait(&sh.xfull, static_cast<uint32_t>(lt & 1)));
      if (!ok) fail_now();
      // one decision for all 128 epilogue threads (they meet at named
      // barriers below): thread 0 snapshots the flag between two barriers
      named_sync(1, 128);
      if (tid == 0) sh.epi_stop = *reinterpret_cast<volatile int*>(&sh.fail);
      named_sync(1, 128);
      if (*reinterpret_cast<volatile int*>(&sh.epi_stop)) break;
      if (tid == 0) x_pending = false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) +
                               static_cast<uint32_t>(b * 128 + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
              "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float* p = xs + (c0 + j) * kRows + r;
          const float y = alpha * __uint_as_float(v[j]);
          *p = load_x ? fmaf(beta, *p, y) : y;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&sh.acce[b]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      named_sync(1, 128);
      if (tid == 0) {
        // rows >= n and columns >= s of the box are not written
        tma_store_2d(&mapX, xs, static_cast<int>(row0_of(lt)), 0);
        bulk_commit();
        bulk_wait_read();
        if (load_x && lt + 1 < my_tiles) {
          mbar_expect_tx(&sh.xfull, x_bytes);
          tma_load_2d(xs, &mapX, &sh.xfull, static_cast<int>(row0_of(lt + 1)), 0);
          ++x_issued;
          x_pending = true;
        }
      }
      named_sync(1, 128);  // the buffer is free (beta == 0) or being refilled
    }
    if (tid == 0) {
      // after a failure, let the X load in flight land before the shared
      // memory is released (the k-th load completes phase k of xfull)
      if (x_pending) mbar_wait(&sh.xfull, static_cast<uint32_t>((x_issued - 1) & 1));
      bulk_wait_all();
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

// W (FP64, i x s, ld ldw) -> TF32 hi part and FP32 remainder, ld ldp >= i
// (16-byte rows for TMA); padding and, for an upper-triangular W, the
// entries below the diagonal are zero.
__global__ void split_w_kernel(int i, int s, const double* __restrict__ W, int ldw,
                               float* __restrict__ hi, float* __restrict__ lo, int ldp,
                               int upper) {
  const int64_t tot = static_cast<int64_t>(ldp) * s;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < tot;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(e % ldp), c = static_cast<int>(e / ldp);
    double w = 0.0;
    if (k < i && !(upper && k > c)) w = W[k + static_cast<int64_t>(c) * ldw];
    const float h = __uint_as_float(__float_as_uint(static_cast<float>(w)) & 0xFFFFE000u);
    hi[e] = h;
    lo[e] = static_cast<float>(w - static_cast<double>(h));
  }
}

__device__ int g_tcu_err;

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

bool make_map(CUtensorMap* map, const float* base, int64_t inner, int64_t outer,
              int64_t ld, int box_inner, int box_outer,
              CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_128B) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(outer)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * sizeof(float)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_inner), static_cast<cuuint32_t>(box_outer)};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Launches of this file's tensor-core kernels since the last check: the
// check reads the device's error flag (a synchronising copy) only after
// one.  The flag stays set until read, so a timeout is reported by a later
// check even if another thread's check consumed the count.
std::atomic<int> tc_update_check_error_pending{0};

int* err_flag() {
  static int* ptr[64] = {};
  static std::mutex mu;
  int dev = 0;
  SG_CUDA(cudaGetDevice(&dev));
  SG_REQUIRE(dev >= 0 && dev < 64, SG_ECUDA, "device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    SG_CUDA(cudaGetSymbolAddress(&p, g_tcu_err));
    ptr[dev] = static_cast<int*>(p);
  }
  return ptr[dev];
}

}  // namespace

bool tc_update_supported(int64_t n, const float* Q, int64_t ldq, int i, const float* X,
                         int64_t ldx, int s) {
  if (n < kRows || i < 1 || s < 1 || s > kMaxN) return false;
  if (reinterpret_cast<uintptr_t>(Q) & 15) return false;
  if ((ldq * 4) & 15) return false;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || ((ldx * 4) & 15)) return false;
  return encode_fn() != nullptr;
}

int64_t tc_update_scratch(int i, int s) {  // floats
  const int ldp = (i + 3) / 4 * 4;
  return 2 * static_cast<int64_t>(ldp) * s + 8;
}

void tc_update(int64_t n, const float* Q, int64_t ldq, int i, const double* W, int ldw,
               float* X, int64_t ldx, int s, double alpha, double beta, bool upper,
               float* scratch, int64_t scratch_floats, cudaStream_t st) {
  const int ldp = (i + 3) / 4 * 4;
  SG_REQUIRE(tc_update_scratch(i, s) <= scratch_floats, SG_EINVAL, "tc_update: scratch too small");
  float* hi = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(scratch) + 15) & ~uintptr_t(15));
  float* lo = hi + static_cast<int64_t>(ldp) * s;
  split_w_kernel<<<64, 256, 0, st>>>(i, s, W, ldw, hi, lo, ldp, upper ? 1 : 0);
  SG_LAUNCH_CHECK();
  const int BN = (s + 15) / 16 * 16;
  CUtensorMap mq, mh, ml, mx;
  SG_REQUIRE(make_map(&mq, Q, n, i, ldq, kRows, kKC, CU_TENSOR_MAP_SWIZZLE_NONE) &&
                 make_map(&mh, hi, ldp, s, ldp, kKC, BN) &&
                 make_map(&ml, lo, ldp, s, ldp, kKC, BN) &&
                 make_map(&mx, X, n, s, ldx, kRows, BN, CU_TENSOR_MAP_SWIZZLE_NONE),
             SG_ECUDA, "cuTensorMapEncodeTiled failed");
  // one shared-memory size for every shape (one CTA per SM; the kernel
  // allocates all 512 TMEM columns): W resident when its chunks fit beside
  // two Q stages and the X tile, else W chunks ride in the ring
  constexpr int smem = kSmemBytes;
  const int avail = smem - 1024;
  const int a_b = kRows * kKC * 4, b_b = BN * kKC * 4, x_b = kRows * BN * 4;
  const int KC = (i + kKC - 1) / kKC;
  int wres = (KC * 2 * b_b + 2 * a_b + x_b <= avail) ? 1 : 0;
  int nst = wres ? (avail - KC * 2 * b_b - x_b) / a_b : (avail - x_b) / (a_b + 2 * b_b);
  if (nst > kStages) nst = kStages;
  SG_REQUIRE(nst >= 1, SG_EINVAL, "tc_update: shared memory too small");
  ensure_dynamic_smem(reinterpret_cast<const void*>(tc_update_kernel), smem);
  const int64_t tiles = (n + kRows - 1) / kRows;
  int grid = device_sm_count();
  if (grid > tiles) grid = static_cast<int>(tiles);
  tc_update_kernel<<<grid, kThreads, smem, st>>>(mq, mh, ml, mx, n, i, s, BN,
                                                  static_cast<float>(alpha),
                                                  static_cast<float>(beta), nst, wres, err_flag());
  tc_update_check_error_pending.fetch_add(1);
  SG_LAUNCH_CHECK();
}

void tc_update_check_error(cudaStream_t st) {
  if (tc_update_check_error_pending.exchange(0) == 0) return;
  int* f = err_flag();
  int host = 0;
  SG_CUDA(cudaMemcpyAsync(&host, f, sizeof(int), cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  if (host) {
    SG_CUDA(cudaMemsetAsync(f, 0, sizeof(int), st));
    throw Error(SG_ECUDA, "tensor-core block update: a bounded wait ran out");
  }
}

}  // namespace sg
