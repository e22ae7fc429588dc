// FP64 block products of BCGS (Alg. 4) on the tensor cores, exactly: the
// projections W = Q^T X and Gram matrices, and the update X = beta X +
// alpha Q W, for the FP64 basis.
//
// GB300's FP64 pipe gives ~1.26 TFLOP/s, so the FP64 block products are
// FP64-ALU bound; its 16-bit tensor cores give ~1.9 PFLOP/s.  Every FP64
// value is written exactly (to 62 bits below its column's largest
// magnitude) as a sum of eight 8-bit digit slices, each slice an FP16 tile:
//   x = 2^(e - 62) * sum_{t=1..8} d_t 256^(8 - t),   |d_t| <= 128 integers,
// with e the exponent of the column's largest |x| (balanced digits: a digit
// >= 128 becomes d - 256 and carries one into the next higher digit).  A
// digit product is an integer of at most 2^14, exact in the MMA's FP32
// accumulator; products of equal level l = t + u have the same weight
// 256^(16 - l), so the MMA sums them into one FP32 accumulator per level.
// A level has at most 8 digit pairs, so its sum over 128 rows stays below
// 8 * 128 * 2^14 = 2^24: every level sum is an exact integer in FP32.  Every
// 128 rows the eight level sums are read from tensor memory and added,
// with their weights 256^(9 - l), into an exact integer per output (two
// int64 halves); levels above 9 (weights below 2^-56 of the leading term)
// are not formed.  The result is the dot product of the 62-bit truncations,
// exact up to the final rounding to FP64 -- more accurate than an FP64
// FMA chain.
//
// Dot tile: 128 columns of Q (MMA M) x 32 columns of X (MMA N) per CTA,
// 32 rows (K) per stage; one CTA per SM (the tile uses all 512
// tensor-memory columns: 256 for the level sums, two A buffers of 128);
// splits of the rows across CTAs are reduced afterwards in a fixed order,
// like the other block dots.
//   * warp 16 (one lane) streams each stage's Q and X boxes with TMA (16
//     rows x 128 or 32 columns, 128-byte swizzled, so every thread reads
//     its column conflict-free) into a two-deep ring;
//   * warps 0-15 cut stage k into digits while warp 17 (one lane) runs
//     stage k-1's MMAs: Q's into one of two tensor-memory A buffers (lane
//     = Q column, two FP16 digits per 32-bit column), X's into one of two
//     sets of 128-byte-swizzled shared-memory B slices;
//   * the eight B slices of a stage lie one after another along N, so one
//     MMA of N = 32 (8 - t) multiplies A's digit t by B's digits 0 .. 7 - t
//     and, written 32 t columns into the level sums, adds each pair (t, u)
//     to level t + u: 8 MMAs per 16 rows form the 36 digit pairs of levels
//     0 .. 7 (36 MMAs of N = 32 would issue the same tensor work);
//     every four stages, one stage late, they read the level sums, eight
//     output columns each.
// Every wait is bounded: on timeout the kernel records an error, drains
// its own copies, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "k_tc_common.cuh"
#include "sg_internal.h"

namespace sg {

namespace {

using namespace tc;

constexpr int kOM = 128;          // columns of Q per tile (MMA M)
constexpr int kON = 32;           // columns of X per tile (MMA N)
constexpr int kOK = 32;           // rows per stage (two MMA K steps)
constexpr int kDig = 8;           // digit slices per value
constexpr int kLev = 8;           // levels l = 2..9 kept
constexpr int kChunk = 4;         // stages per exact level sum (128 rows)
constexpr uint32_t kOTmemCols = 512;
constexpr uint32_t kAccCol = 0;     // level L = l - 2 at column 32 L
constexpr uint32_t kDACol = 256;    // A buffer b at 256 + 128 b, digit slice t at + 16 t
constexpr int kQBox = 16 * kOM * 8;           // one 16-row Q box: 16 KB
constexpr int kQBytes = (kOK / 16) * kQBox;   // 32 KB per stage
constexpr int kXBox = 16 * kON * 8;           // 4 KB
constexpr int kXBytes = (kOK / 16) * kXBox;   // 8 KB per stage
constexpr int kBSlice = kON * 128;            // 32 rows x 64 FP16 (the stage fills 32): 4 KB
constexpr int kBBytes = kDig * kBSlice;       // 32 KB
static_assert(kLev == kDig, "one MMA per digit of A covers levels t .. kLev - 1");
constexpr int kDWarps = 16;                   // split / readout warps
constexpr int kDThreads = (kDWarps + 2) * 32; // + warp 16 TMA, warp 17 MMA
constexpr int kDSplit = kDWarps * 32;

struct __align__(8) OzShared {
  uint64_t qfull[2], qfree[2], afull[2], afree[2];
  uint64_t accfull, accfree, done;
  uint32_t tmem_base;
  int fail;
};

// dynamic shared memory of the dot: Q and X boxes and B slices, two of
// each, then the barriers
constexpr int kOzSmem = 2 * (kQBytes + kXBytes + kBBytes) + static_cast<int>(sizeof(OzShared)) + 1024;

__device__ __forceinline__ void mma_bf16_tmem_a(uint32_t dtmem, uint32_t atmem, uint64_t b,
                                                uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(dtmem),
      "r"(atmem), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// x relative to 2^e (|x| < 2^e) as the signed integer m = x 2^(62 - e),
// |m| < 2^62, truncated toward zero.
__device__ __forceinline__ int64_t scaled62(double x, int e) {
  const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(x));
  const int E = static_cast<int>((bits >> 52) & 0x7FF);
  uint64_t m = 0;
  if (E != 0 && E != 0x7FF) {
    const uint64_t mant = (bits & ((uint64_t(1) << 52) - 1)) | (uint64_t(1) << 52);
    const int sh = E - 1013 - e;   // <= 9 when |x| < 2^e
    if (sh >= 0) m = sh < 10 ? mant << sh : 0;
    else if (sh > -64) m = mant >> (-sh);
  }
  return (bits >> 63) ? -static_cast<int64_t>(m) : static_cast<int64_t>(m);
}

// The integer value of an FP32 level sum (an exact integer, |v| < 2^24)
// on the FP32 pipe: adding 1.5 2^25 (whose unit in the last place is 4)
// rounds v to a multiple of 4 and leaves v / 4 in the low bits of the sum's
// bit pattern; the remainder (-2 .. 2, exact) converts through 1.5 2^23 the
// same way.  Profiles showed the F2I conversion occupying the FP64 pipe.
__device__ __forceinline__ int32_t level_int(uint32_t vb) {
  const float v = __uint_as_float(vb);
  const float t = __fadd_rn(v, 50331648.0f);
  const float r = __fsub_rn(v, __fsub_rn(t, 50331648.0f));
  return 4 * (__float_as_int(t) - 0x4C400000) + (__float_as_int(__fadd_rn(r, 12582912.0f)) - 0x4B400000);
}

__device__ __forceinline__ uint32_t f16x2_sub(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// Balanced base-256 digits of two numbers as FP16 pairs: w[t] holds digit
// t (most significant first) of ma in its low half and of mb in its high
// half.  Adding 0x80 to every byte of m makes each byte of the sum the
// digit plus 128 (the carries do the balancing; for |m| < 2^62 the top
// byte stays in [64, 192]).  The FP16 number with bit pattern 0x6600 + b
// is 1536 + b exactly (the unit in the last place is 1 on [1024, 2048)),
// so one packed subtraction of 1664 leaves the digits, exactly.
__device__ __forceinline__ void digits_f16x2(int64_t ma, int64_t mb, uint32_t* w) {
  const uint64_t sa = static_cast<uint64_t>(ma) + 0x8080808080808080ull;
  const uint64_t sb = static_cast<uint64_t>(mb) + 0x8080808080808080ull;
  const uint32_t ahi = static_cast<uint32_t>(sa >> 32), alo = static_cast<uint32_t>(sa);
  const uint32_t bhi = static_cast<uint32_t>(sb >> 32), blo = static_cast<uint32_t>(sb);
  constexpr uint32_t kHi = 0x66666666u;
  constexpr uint32_t kOff = 0x66806680u;              // 1664 in both halves
  // byte pairs (a_j, b_j) of digits 0-1, 2-3, 4-5, 6-7
  const uint32_t p[4] = {__byte_perm(ahi, bhi, 0x6273), __byte_perm(ahi, bhi, 0x4051),
                         __byte_perm(alo, blo, 0x6273), __byte_perm(alo, blo, 0x4051)};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    w[2 * k] = f16x2_sub(__byte_perm(p[k], kHi, 0x4140), kOff);
    w[2 * k + 1] = f16x2_sub(__byte_perm(p[k], kHi, 0x4342), kOff);
  }
}

// This thread's lane, 4 consecutive 32-bit columns from taddr.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}

// This thread's lane, 2 consecutive 32-bit columns from taddr.
__device__ __forceinline__ void tmem_st2(uint32_t taddr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(taddr), "r"(v[0]),
               "r"(v[1])
               : "memory");
}

// This thread's lane, 8 consecutive 32-bit columns from taddr.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Instruction descriptor: kind::f16 with FP16 A and B, FP32 accumulator,
// K-major A and B.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

// the same on the FP64 pipe, for results outside the normal range (kept
// out of line so that the common path does not evaluate it)
__device__ __noinline__ double int96_to_double_slow(int64_t hi, uint32_t lo, int e2) {
  return ldexp(ldexp(static_cast<double>(hi), 32) + static_cast<double>(lo), e2);
}

// (hi 2^32 + lo) 2^e2 rounded to the nearest double (ties to even), in
// integer arithmetic: the 96-bit value is normalised with a count of its
// leading zeros, its top 53 bits are rounded with the guard bit and a
// sticky bit, and the exponent field is added on.  Falls back to the FP64
// pipe when the result would leave the normal range.
__device__ __forceinline__ double int96_to_double(int64_t hi, uint32_t lo, int e2) {
  const bool neg = hi < 0;
  uint64_t h = static_cast<uint64_t>(hi);
  uint32_t l = lo;
  if (neg) {                                   // magnitude: two's complement of 96 bits
    l = 0u - lo;
    h = ~h + (lo == 0u ? 1u : 0u);
  }
  if ((h | l) == 0) return 0.0;
  uint64_t t;
  uint32_t low;
  int z;
  if (h != 0) {
    z = __clzll(static_cast<long long>(h));    // 1 .. 63 (|hi| < 2^62)
    if (z < 32) {
      t = (h << z) | (static_cast<uint64_t>(l) >> (32 - z));
      low = l << z;
    } else {
      t = (h << z) | (static_cast<uint64_t>(l) << (z - 32));
      low = 0;
    }
  } else {
    const int zl = __clz(static_cast<int>(l));
    t = static_cast<uint64_t>(l) << (32 + zl);
    low = 0;
    z = 64 + zl;
  }
  // t holds the top 64 bits (MSB at bit 63) of the value times 2^(z - 32)
  uint64_t mant = t >> 11;
  const uint64_t up = ((t >> 10) & 1u) & (((t & 0x3FFu) | low | (mant & 1u)) != 0 ? 1u : 0u);
  mant += up;
  const int E = 1118 - z + e2;                 // exponent field of mant 2^(43 - z + e2)
  if (E < 1 || E > 2045) return int96_to_double_slow(hi, lo, e2);
  const uint64_t bits = (static_cast<uint64_t>(E - 1) << 52) + mant;
  return __longlong_as_double(static_cast<long long>(bits | (neg ? (uint64_t(1) << 63) : 0)));
}

constexpr int kUWarps = 16;                    // split / readout / epilogue warps
constexpr int kUThreads = (kUWarps + 2) * 32;  // + warp 16 TMA, warp 17 MMA
constexpr int kUSplit = kUWarps * 32;

// grid: (tiles of 128 Q columns, tiles of 32 X columns, splits)
__global__ void __launch_bounds__(kDThreads, 1)
oz_dot_kernel(const __grid_constant__ CUtensorMap mapQ,
              const __grid_constant__ CUtensorMap mapX, int64_t n, int M, int N,
              const int* __restrict__ eq, const int* __restrict__ ex, int64_t rows_per_split,
              double* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int m0 = blockIdx.x * kOM;
  const int n0 = blockIdx.y * kON;
  const int64_t k0 = static_cast<int64_t>(blockIdx.z) * rows_per_split;
  const int64_t k1 = (k0 + rows_per_split < n) ? k0 + rows_per_split : n;
  const int nk = static_cast<int>((k1 - k0 + kOK - 1) / kOK);
  auto stQ = [&](int b) { return base + b * kQBytes; };
  auto stX = [&](int b) { return base + 2 * kQBytes + b * kXBytes; };
  auto stB = [&](int b) { return base + 2 * (kQBytes + kXBytes) + b * kBBytes; };
  OzShared& sh = *reinterpret_cast<OzShared*>(base + 2 * (kQBytes + kXBytes + kBBytes));
  auto failed = [&]() { return *reinterpret_cast<volatile int*>(&sh.fail) != 0; };
  auto group_end = [&](int k) { return (k % kChunk) == kChunk - 1 || k == nk - 1; };

  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.qfull[b], 1);
      mbar_init(&sh.qfree[b], kDSplit);
      mbar_init(&sh.afull[b], kDSplit);
      mbar_init(&sh.afree[b], 1);
    }
    mbar_init(&sh.accfull, 1);
    mbar_init(&sh.accfree, kDSplit);
    mbar_init(&sh.done, 1);
    sh.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh.tmem_base)),
                 "r"(kOTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh.tmem_base;

  // per-thread sums of 8 outputs (warp w reads tensor-memory lanes
  // 32 (w % 4) .. + 31 = Q columns, and X columns 8 (w / 4) .. + 7), each
  // as two int64 halves: ahi = sum of S_L 256^(3-L) over levels L = 0..3,
  // alo = sum of S_L 256^(7-L) over L = 4..7 (|S_L| < 2^24, so each half
  // grows by < 2^50 per readout and stays exact for 2^12 readouts), and
  // the output's V' = ahi 2^32 + alo
  constexpr int kCols = kON / 4;
  const int cg = warp >> 2;
  int64_t alo[kCols];
  int64_t ahi[kCols];
#pragma unroll
  for (int c = 0; c < kCols; ++c) { alo[c] = 0; ahi[c] = 0; }
  auto readout = [&](int k) -> bool {
    if (!mbar_wait(&sh.accfull, static_cast<uint32_t>((k / kChunk) & 1))) sh.fail = 1;
    if (__any_sync(0xffffffffu, failed())) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tl = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16) +
                        static_cast<uint32_t>(cg * kCols);
#pragma unroll
    for (int L = 0; L < kLev; ++L) {
      uint32_t v[kCols];
      tmem_ld8(tl + kAccCol + static_cast<uint32_t>(32 * L), v);
#pragma unroll
      for (int cc = 0; cc < kCols; ++cc) {
        const int64_t sv = level_int(v[cc]);
        if (L < 4) ahi[cc] += sv * (int64_t(1) << (8 * (3 - L)));
        else alo[cc] += sv * (int64_t(1) << (8 * (7 - L)));
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    mbar_arrive(&sh.accfree);
    return true;
  };

  if (warp == kDWarps) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      int nq0 = 0, nq1 = 0;
      for (int k = 0; k < nk; ++k) {
        if (failed()) break;
        const int b = k & 1;
        if (k >= 2 && !mbar_wait(&sh.qfree[b], static_cast<uint32_t>(((k >> 1) - 1) & 1))) {
          sh.fail = 1;
          break;
        }
        const int x = static_cast<int>(k0 + static_cast<int64_t>(k) * kOK);
        mbar_expect_tx(&sh.qfull[b], static_cast<uint32_t>(kQBytes + kXBytes));
        for (int bx = 0; bx < kOK / 16; ++bx) {
          tma_load_2d(stQ(b) + bx * kQBox, &mapQ, &sh.qfull[b], x + 16 * bx, m0);
          tma_load_2d(stX(b) + bx * kXBox, &mapX, &sh.qfull[b], x + 16 * bx, n0);
        }
        if (b) ++nq1; else ++nq0;
      }
      if (failed()) {
        // drain this CTA's copies in flight (at most one stage per buffer)
        if (nq0 > 0) mbar_wait(&sh.qfull[0], static_cast<uint32_t>((nq0 - 1) & 1));
        if (nq1 > 0) mbar_wait(&sh.qfull[1], static_cast<uint32_t>((nq1 - 1) & 1));
      }
    }
  } else if (warp == kDWarps + 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      int grp = 0;
      for (int k = 0; k < nk; ++k) {
        if (failed()) break;
        const int b = k & 1;
        const bool fresh = (k % kChunk) == 0;
        if (!mbar_wait(&sh.afull[b], static_cast<uint32_t>((k >> 1) & 1)) ||
            (fresh && grp > 0 && !mbar_wait(&sh.accfree, static_cast<uint32_t>((grp - 1) & 1)))) {
          sh.fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t bbase = smem_u32(stB(b));
#pragma unroll 1
        for (int kk = 0; kk < kOK / 16; ++kk) {
          const uint64_t bd = sdesc(bbase) + static_cast<uint64_t>((kk * 32) >> 4);
#pragma unroll
          for (int t = 0; t < kDig; ++t) {
            // A's digit t against B's digits 0 .. 7 - t in one MMA: the B
            // slices lie one after another along N, so output column
            // 32 u + c holds the pair (t, u), which belongs to level t + u
            // at accumulator column 32 (t + u) + c
            const uint32_t acc = (!fresh || kk > 0 || t > 0) ? 1u : 0u;
            mma_bf16_tmem_a(tmem + kAccCol + static_cast<uint32_t>(32 * t),
                            tmem + kDACol + static_cast<uint32_t>(128 * b + 16 * t + 8 * kk),
                            bd, idesc_f16(kOM, kON * (kLev - t)), acc);
          }
        }
        mma_commit(&sh.afree[b]);     // A and B buffers b reusable
        if (group_end(k)) {
          mma_commit(&sh.accfull);
          ++grp;
        }
      }
      mma_commit(&sh.done);
    }
  } else {
    // ------------------------------------------------ split, readout
    // A (Q, into tensor memory): warp w covers lanes 32 (w % 4) .. + 31 (Q
    // columns) for the stage's rows 8 (w / 4) .. + 7 (box (w / 4) / 2,
    // chunks 4 ((w / 4) % 2) .. + 3 of the column's 128-byte line);
    // B (X, into shared-memory slices): warp w takes rows 2w, 2w + 1 of all
    // 32 columns (box w / 8, chunk w % 8), lane = column.
    const int m = (warp & 3) * 32 + lane;    // Q column m0 + m
    const int eM = (m0 + m < M) ? eq[m0 + m] : -4000;
    const int eN = (n0 + lane < N) ? ex[n0 + lane] : -4000;
    const uint32_t tlane = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
    int pend = -1;
    bool stop = false;
    for (int k = 0; k < nk; ++k) {
      const int b = k & 1;
      bool bad = failed();
      if (!bad) {
        const bool ok = mbar_wait(&sh.qfull[b], static_cast<uint32_t>((k >> 1) & 1)) &&
                        (k < 2 || mbar_wait(&sh.afree[b], static_cast<uint32_t>(((k >> 1) - 1) & 1)));
        if (!ok) {
          sh.fail = 1;
          bad = true;
        }
      }
      if (__any_sync(0xffffffffu, bad)) {
        stop = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      {
        // B: rows 2w, 2w + 1 of X column `lane`, one FP16 pair per digit at
        // K offset 2w of the column's 128-byte swizzled row
        const unsigned char* line = stX(b) + (warp >> 3) * kXBox + lane * 128;
        const double2 v = *reinterpret_cast<const double2*>(line + (((warp & 7) ^ (lane & 7)) << 4));
        uint32_t d8[kDig];
        digits_f16x2(scaled62(v.x, eN), scaled62(v.y, eN), d8);
        unsigned char* bs = stB(b) + (lane >> 3) * 1024 + (lane & 7) * 128 + (warp & 3) * 4;
        const int chunk = (warp >> 2) ^ (lane & 7);
#pragma unroll
        for (int t = 0; t < kDig; ++t)
          *reinterpret_cast<uint32_t*>(bs + t * kBSlice + (chunk << 4)) = d8[t];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      {
        // A: column m's rows 8 cg .. + 7: box cg / 2, chunks 4 (cg % 2) + j
        // (rows 2j, 2j + 1 of the box) -> tensor-memory column 4 cg + j of
        // each digit slice of buffer b
        const unsigned char* line = stQ(b) + (cg >> 1) * kQBox + m * 128;
        uint32_t words[kDig][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int jj = 4 * (cg & 1) + j;
          const double2 v = *reinterpret_cast<const double2*>(line + ((jj ^ (m & 7)) << 4));
          uint32_t d8[kDig];
          digits_f16x2(scaled62(v.x, eM), scaled62(v.y, eM), d8);
#pragma unroll
          for (int t = 0; t < kDig; ++t) words[t][j] = d8[t];
        }
#pragma unroll
        for (int t = 0; t < kDig; ++t)
          tmem_st4(tlane + kDACol + static_cast<uint32_t>(128 * b + 16 * t + 4 * cg), words[t]);
      }
      mbar_arrive(&sh.qfree[b]);
      tmem_st_wait();
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&sh.afull[b]);
      if (pend >= 0) {
        if (!readout(pend)) {
          stop = true;
          break;
        }
        pend = -1;
      }
      if (group_end(k)) pend = k;
    }
    if (!stop && pend >= 0) readout(pend);
  }
  // (twice the limit: after a failure the MMA warp may first spend one
  // limit on a step that never came)
  if (warp < 4 && !mbar_wait(&sh.done, 0, 2 * kWaitNs)) sh.fail = 1;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  const bool good = !sh.fail;
  if (!good) {
    if (tid == 0) atomicExch(err, 1);
  } else if (warp < kDWarps) {
    const int gm = m0 + (warp & 3) * 32 + lane;
    if (gm < M) {
      double* P = part + static_cast<int64_t>(blockIdx.z) * M * N;
      const int eM = eq[gm];
#pragma unroll
      for (int cc = 0; cc < kCols; ++cc) {
        const int gc = n0 + cg * kCols + cc;
        if (gc < N) {
          // V' = (ahi + carry) 2^32 + the low 32 bits of alo, rounded once
          const int64_t hi = ahi[cc] + (alo[cc] >> 32);
          const uint32_t lo = static_cast<uint32_t>(alo[cc]);
          P[gm + static_cast<int64_t>(gc) * M] =
              (eM < -2000 || ex[gc] < -2000) ? 0.0 : int96_to_double(hi, lo, eM + ex[gc] - 68);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kOTmemCols)
                 : "memory");
  }
}

// ---------------------------------------------------------------- update
// X = beta X + alpha Q W on the tensor cores, exactly in the same sense.
// Output (r, c) sums Q[r,k] W[k,c] over k; with Q's digits relative to its
// column exponents e_k (as in the dot) and W' = W 2^(e_k) cut into digits
// relative to W' column c's exponent g_c, every product of the sum carries
// the one weight 2^(g_c - 124), so the level sums are exact as above.  The
// digits are FP16 numbers here (integers of at most 8 bits are exact in
// either 16-bit type; FP16's wider mantissa lets one packed subtraction
// turn two digit bytes into two FP16 digits).
// Tile: 128 rows (MMA M, tensor-memory lanes) x 32 columns of X (MMA N);
// one CTA per SM walks the row tiles of one column tile in stages of 32
// columns of Q (two MMA K steps), software-pipelined:
//   * warp 16 (one lane) loads each stage's Q box (128 rows x 32 columns,
//     unswizzled: a row's values are 1 KB apart, so a warp reads 32
//     consecutive rows conflict-free) into a two-deep ring, and each
//     tile's X box for the epilogue;
//   * warps 0-15 cut stage q into one of two tensor-memory A buffers while
//     warp 17 (one lane) runs stage q-1's MMAs from the other (8 per 16
//     columns of Q, one per digit of Q against the consecutive digit
//     slices of W', as in the dot);
//     W' is cut once per CTA into shared-memory B slices (one 32 KB group
//     of eight slices per 64 columns of Q, i <= 256);
//   * level sums are read every four stages (128 columns of Q) and at the
//     end of a tile, one stage late so that the split of the next stage
//     overlaps the last MMAs; the epilogue writes beta X + alpha V 2^(g_c-68)
//     from the prefetched X box.
// K steps that lie wholly beyond column i are not issued.
constexpr int kUM = 128;
constexpr int kUN = 32;
constexpr int kUS = 32;                                 // columns of Q per stage
constexpr int kUMaxK = 256;
constexpr int kUBox = kUM * kUS * 8;                    // 32 KB: a Q stage or the X tile
constexpr int kUBChunk = kDig * kBSlice;                // 32 KB per 64 columns of Q
constexpr uint32_t kUACol = 256;                        // A buffer b: 256 + 128 b

// per-column tables after the W' slices: Q's column exponents e_k, W'
// column exponents g_c
struct OzUTables {
  int eq[kUMaxK];
  int g[kUN];
};

struct __align__(8) OzUShared {
  uint64_t qfull[2], qfree[2], afull[2], afree[2];
  uint64_t accfull, accfree, xfull, xfree, done;
  uint32_t tmem_base;
  int fail;
};

// dynamic shared memory: Q ring, X box, W' slices, tables, barriers (all of
// it dynamic, so the 1 KB alignment slack fits under the 227 KB limit)
int oz_update_smem(int i) {
  return 3 * kUBox + ((i + 63) / 64) * kUBChunk + static_cast<int>(sizeof(OzUTables)) +
         static_cast<int>(sizeof(OzUShared)) + 1024;
}

// grid: (tiles of 32 X columns, row groups); row tiles g, g + G, ...
__global__ void __launch_bounds__(kUThreads, 1)
oz_update_kernel(const __grid_constant__ CUtensorMap mapQ, const __grid_constant__ CUtensorMap mapX,
                 int64_t n, int i, int s, const double* __restrict__ W, int ldw,
                 double* __restrict__ X, int64_t ldx, double alpha, double beta, int upper,
                 const int* __restrict__ eq, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int n0 = blockIdx.x * kUN;
  const int64_t ntiles = (n + kUM - 1) / kUM;
  const int G = gridDim.y;
  const int my_tiles = static_cast<int>((ntiles - blockIdx.y + G - 1) / G);
  const int nsub = (i + kUS - 1) / kUS;          // stages per row tile
  const int nkc = (i + 63) / 64;                 // groups of W' slices
  const int gpt = (nsub + 3) / 4;                // level readouts per row tile
  const bool loadx = beta != 0.0;
  unsigned char* stX = base + 2 * kUBox;
  unsigned char* bsl = base + 3 * kUBox;
  OzUTables& tb = *reinterpret_cast<OzUTables*>(bsl + nkc * kUBChunk);
  OzUShared& sh = *reinterpret_cast<OzUShared*>(bsl + nkc * kUBChunk + sizeof(OzUTables));
  auto failed = [&]() { return *reinterpret_cast<volatile int*>(&sh.fail) != 0; };
  auto group_end = [&](int kq) { return (kq & 3) == 3 || kq == nsub - 1; };
  // alpha = +-2^(ka - 1) folds into the exponent and the sign of the sums
  int ka = 0;
  const double fa = frexp(alpha, &ka);
  const bool apow2 = fabs(fa) == 0.5;

  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.qfull[b], 1);
      mbar_init(&sh.qfree[b], kUSplit);
      mbar_init(&sh.afull[b], kUSplit);
      mbar_init(&sh.afree[b], 1);
    }
    mbar_init(&sh.accfull, 1);
    mbar_init(&sh.accfree, kUSplit);
    mbar_init(&sh.xfull, 1);
    mbar_init(&sh.xfree, kUSplit);
    mbar_init(&sh.done, 1);
    sh.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh.tmem_base)),
                 "r"(kOTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // W' = W 2^(e_k) (zero below the diagonal when `upper`) cut into digits
  // relative to its column exponents g_c: B slices of every 64 columns of Q
  if (warp < kUWarps) {
    for (int k = tid; k < kUMaxK; k += kUSplit) tb.eq[k] = k < i ? eq[k] : -4000;
    if (tid < kUN) tb.g[tid] = -2147483647;
    uint4* z = reinterpret_cast<uint4*>(bsl);
    for (int e = tid; e < nkc * kUBChunk / 16; e += kUSplit) z[e] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  auto wprime = [&](int k, int c) -> double {
    const int gc = n0 + c;
    if (k >= i || gc >= s || (upper && k > gc) || tb.eq[k] < -2000) return 0.0;
    return ldexp(W[k + static_cast<int64_t>(gc) * ldw], tb.eq[k]);
  };
  if (warp < kUWarps) {
    const int c = lane;
    double mx = 0.0;
    for (int k = warp; k < i; k += kUWarps) mx = fmax(mx, fabs(wprime(k, c)));
    if (mx > 0.0) {
      int ee = 0;
      frexp(mx, &ee);
      atomicMax(&tb.g[c], ee);
    }
  }
  __syncthreads();
  if (warp < kUWarps) {
    const int c = lane;
    const int gc = tb.g[c] > -2000 ? tb.g[c] : -4000;
    for (int k = warp; k < i; k += kUWarps) {
      const int64_t mk = scaled62(wprime(k, c), gc);
      uint32_t w8[kDig];
      digits_f16x2(mk, mk, w8);
      const int kc = k / 64, kk = k % 64;
#pragma unroll
      for (int t = 0; t < kDig; ++t) {
        unsigned char* row = bsl + kc * kUBChunk + t * kBSlice + (c >> 3) * 1024 + (c & 7) * 128;
        *reinterpret_cast<uint16_t*>(row + (((kk >> 3) ^ (c & 7)) << 4) + (kk & 7) * 2) =
            static_cast<uint16_t>(w8[t] & 0xFFFFu);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh.tmem_base;
  const int nstages = my_tiles * nsub;

  if (warp == kUWarps) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      int nq0 = 0, nq1 = 0;
      int nx = 0;
      for (int q = 0; q < nstages; ++q) {
        if (failed()) break;
        const int b = q & 1;
        if (q >= 2 && !mbar_wait(&sh.qfree[b], static_cast<uint32_t>(((q >> 1) - 1) & 1))) {
          sh.fail = 1;
          break;
        }
        const int kq = q % nsub;
        const int rtl = q / nsub;
        const int rt = blockIdx.y + rtl * G;
        mbar_expect_tx(&sh.qfull[b], static_cast<uint32_t>(kUBox));
        tma_load_2d(base + b * kUBox, &mapQ, &sh.qfull[b], rt * kUM, kq * kUS);
        if (b) ++nq1; else ++nq0;
        if (loadx && kq == nsub - 1) {
          if (rtl > 0 && !mbar_wait(&sh.xfree, static_cast<uint32_t>((rtl - 1) & 1))) {
            sh.fail = 1;
            break;
          }
          mbar_expect_tx(&sh.xfull, static_cast<uint32_t>(kUBox));
          tma_load_2d(stX, &mapX, &sh.xfull, rt * kUM, n0);
          ++nx;
        }
      }
      if (failed()) {
        // drain this CTA's copies in flight (at most one per buffer)
        if (nq0 > 0) mbar_wait(&sh.qfull[0], static_cast<uint32_t>((nq0 - 1) & 1));
        if (nq1 > 0) mbar_wait(&sh.qfull[1], static_cast<uint32_t>((nq1 - 1) & 1));
        if (nx > 0) mbar_wait(&sh.xfull, static_cast<uint32_t>((nx - 1) & 1));
      }
    }
  } else if (warp == kUWarps + 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      int grp = 0;
      for (int q = 0; q < nstages; ++q) {
        if (failed()) break;
        const int b = q & 1;
        const int kq = q % nsub;
        const bool fresh = (kq & 3) == 0;
        if (!mbar_wait(&sh.afull[b], static_cast<uint32_t>((q >> 1) & 1)) ||
            (fresh && grp > 0 && !mbar_wait(&sh.accfree, static_cast<uint32_t>((grp - 1) & 1)))) {
          sh.fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t bbase = smem_u32(bsl + (kq >> 1) * kUBChunk);
        const int ksteps = (i - kq * kUS) >= 17 ? 2 : 1;     // K steps holding columns < i
#pragma unroll 1
        for (int kk = 0; kk < ksteps; ++kk) {
          const int kb = (kq & 1) * 2 + kk;                  // 16-column step of the 64
          const uint64_t bd = sdesc(bbase) + static_cast<uint64_t>((kb * 32) >> 4);
#pragma unroll
          for (int t = 0; t < kDig; ++t) {
            // digit t of Q against W' digits 0 .. 7 - t (consecutive along
            // N): levels t .. 7 in one MMA
            const uint32_t acc = (!fresh || kk > 0 || t > 0) ? 1u : 0u;
            mma_bf16_tmem_a(tmem + kAccCol + static_cast<uint32_t>(32 * t),
                            tmem + kUACol + static_cast<uint32_t>(128 * b + 16 * t + 8 * kk), bd,
                            idesc_f16(kUM, kUN * (kLev - t)), acc);
          }
        }
        mma_commit(&sh.afree[b]);
        if (group_end(kq)) {
          mma_commit(&sh.accfull);
          ++grp;
        }
      }
      mma_commit(&sh.done);
    }
  } else {
    // ------------------------------------------------ split, readout, epilogue
    // warp w: rows 32 (w % 4) .. + 31 (its tensor-memory lane quarter) and
    // column group cg = w / 4: Q columns 8 cg .. 8 cg + 7 of each stage,
    // output columns 8 cg .. 8 cg + 7 of the tile
    constexpr int kCols = kUN / 4;
    const int m = (warp & 3) * 32 + lane;
    const int cg = warp >> 2;
    const uint32_t tlane = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);
    int64_t alo[kCols], ahi[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) { alo[c] = 0; ahi[c] = 0; }
    // level sums of the group ending at stage pq; the epilogue after a
    // tile's last group
    auto readout = [&](int pq) -> bool {
      const int kq = pq % nsub;
      const int rtl = pq / nsub;
      const int grp = rtl * gpt + kq / 4;
      if (!mbar_wait(&sh.accfull, static_cast<uint32_t>(grp & 1))) sh.fail = 1;
      if (__any_sync(0xffffffffu, failed())) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tl = tlane + static_cast<uint32_t>(cg * kCols);
#pragma unroll
      for (int L = 0; L < kLev; ++L) {
        uint32_t v[kCols];
        tmem_ld8(tl + kAccCol + static_cast<uint32_t>(32 * L), v);
#pragma unroll
        for (int cc = 0; cc < kCols; ++cc) {
          const int64_t sv = level_int(v[cc]);
          if (L < 4) ahi[cc] += sv * (int64_t(1) << (8 * (3 - L)));
          else alo[cc] += sv * (int64_t(1) << (8 * (7 - L)));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&sh.accfree);
      if (kq == nsub - 1) {
        // epilogue of the row tile: X = beta X + alpha V' 2^(g_c - 68)
        if (loadx && !mbar_wait(&sh.xfull, static_cast<uint32_t>(rtl & 1))) sh.fail = 1;
        if (__any_sync(0xffffffffu, failed())) return false;
        const int64_t r = (blockIdx.y + static_cast<int64_t>(rtl) * G) * kUM + m;
        const int c0 = n0 + cg * kCols;
        const double* xs = reinterpret_cast<const double*>(stX) + cg * kCols * kUM + m;
        double* xr = X + r + static_cast<int64_t>(c0) * ldx;
#pragma unroll
        for (int cc = 0; cc < kCols; ++cc) {
          // V' = (ahi + carry) 2^32 + the low 32 bits of alo
          const int64_t hi = ahi[cc] + (alo[cc] >> 32);
          const uint32_t lo = static_cast<uint32_t>(alo[cc]);
          const int gcol = tb.g[cg * kCols + cc];
          double p;
          if (gcol < -2000) p = 0.0;
          else if (apow2) {
            p = int96_to_double(hi, lo, gcol - 68 + ka - 1);
            if (fa < 0.0) p = -p;
          } else {
            p = int96_to_double(hi, lo, gcol - 68) * alpha;
          }
          if (r < n && c0 + cc < s)
            xr[static_cast<int64_t>(cc) * ldx] = loadx ? fma(beta, xs[cc * kUM], p) : p;
          alo[cc] = 0;
          ahi[cc] = 0;
        }
        if (loadx) mbar_arrive(&sh.xfree);
      }
      return true;
    };
    int pend = -1;
    bool stop = false;
    for (int q = 0; q < nstages; ++q) {
      const int b = q & 1;
      const int kq = q % nsub;
      bool bad = failed();
      if (!bad) {
        const bool ok = mbar_wait(&sh.qfull[b], static_cast<uint32_t>((q >> 1) & 1)) &&
                        (q < 2 || mbar_wait(&sh.afree[b], static_cast<uint32_t>(((q >> 1) - 1) & 1)));
        if (!ok) {
          sh.fail = 1;
          bad = true;
        }
      }
      if (__any_sync(0xffffffffu, bad)) {
        stop = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // row m's 8 values: column 8 cg + c of the stage at byte
      // (8 cg + c) * 1024 + 8 m; two columns per tensor-memory word, the
      // lower column in the low half; a K step (16 columns) wholly past
      // column i is not issued, so its digits are not needed
      const int k0 = kq * kUS + kCols * cg;
      if (kq * kUS + 16 * (cg >> 1) < i) {
        const unsigned char* col = base + b * kUBox + kCols * cg * 1024 + m * 8;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t words[kDig][2];
#pragma unroll
          for (int w = 0; w < 2; ++w) {
            const int c = 4 * h + 2 * w;
            const double va = *reinterpret_cast<const double*>(col + c * 1024);
            const double vb = *reinterpret_cast<const double*>(col + (c + 1) * 1024);
            uint32_t d8[kDig];
            digits_f16x2(scaled62(va, tb.eq[k0 + c]), scaled62(vb, tb.eq[k0 + c + 1]), d8);
#pragma unroll
            for (int t = 0; t < kDig; ++t) words[t][w] = d8[t];
          }
#pragma unroll
          for (int t = 0; t < kDig; ++t)
            tmem_st2(tlane + kUACol + static_cast<uint32_t>(128 * b + 16 * t + 4 * cg + 2 * h),
                     words[t]);
        }
      }
      mbar_arrive(&sh.qfree[b]);
      tmem_st_wait();
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&sh.afull[b]);
      if (pend >= 0) {
        if (!readout(pend)) {
          stop = true;
          break;
        }
        pend = -1;
      }
      if (group_end(kq)) pend = q;
    }
    if (!stop && pend >= 0) readout(pend);
  }
  if (warp < 4 && !mbar_wait(&sh.done, 0, 2 * kWaitNs)) sh.fail = 1;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (sh.fail && tid == 0) atomicExch(err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kOTmemCols)
                 : "memory");
  }
}

// e[c] = the exponent of column c's largest magnitude (|x| < 2^e): CTA
// (c, z) takes rows [z rows, (z+1) rows) and merges its exponent with
// atomicMax into e[c], which starts at a large negative value (all-zero
// columns keep it).
__global__ void __launch_bounds__(256)
col_exponent_kernel(int64_t n, const double* __restrict__ X, int64_t ld, int64_t rows,
                    int* __restrict__ e) {
  // The largest |x| is found in integer arithmetic (the FP64 pipe would
  // bound this kernel far below HBM speed): for finite doubles, |x| orders
  // like its bit pattern with the sign cleared.  NaNs (patterns above that
  // of infinity) are skipped, as fmax would skip them.
  const uint64_t* col = reinterpret_cast<const uint64_t*>(X + static_cast<int64_t>(blockIdx.x) * ld);
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rows;
  const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
  constexpr uint64_t kMag = 0x7FFFFFFFFFFFFFFFull, kInf = 0x7FF0000000000000ull;
  auto take = [&](uint64_t& mx, uint64_t b) {
    b &= kMag;
    if (b <= kInf && b > mx) mx = b;
  };
  uint64_t mx = 0;
  int64_t r = r0;
  // one element to reach a 16-byte boundary, pairs with four loads in
  // flight per thread, one element of tail
  if ((reinterpret_cast<uintptr_t>(col + r) & 15) && r < r1) {
    if (threadIdx.x == 0) take(mx, __ldg(col + r));
    ++r;
  }
  const ulonglong2* pr = reinterpret_cast<const ulonglong2*>(col + r);
  const int64_t np = (r1 - r) / 2;
  for (int64_t p = threadIdx.x; p < np; p += 4 * 256) {
    ulonglong2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      v[u] = (p + u * 256 < np) ? __ldg(pr + p + u * 256) : make_ulonglong2(0, 0);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      take(mx, v[u].x);
      take(mx, v[u].y);
    }
  }
  if (((r1 - r) & 1) && threadIdx.x == 0) take(mx, __ldg(col + r1 - 1));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t o = __shfl_xor_sync(0xffffffffu, mx, off);
    if (o > mx) mx = o;
  }
  __shared__ uint64_t wm[8];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t tb = 0;
    for (int w = 0; w < 8; ++w) tb = wm[w] > tb ? wm[w] : tb;
    const double t = __longlong_as_double(static_cast<long long>(tb));
    if (tb != 0) {
      int ee = 0;
      frexp(t, &ee);   // t = f 2^ee, f in [0.5, 1): |x| <= t < 2^ee
      atomicMax(e + blockIdx.x, ee);
    }
  }
}

void col_exponents(int64_t n, const double* X, int64_t ld, int cols, int* e, cudaStream_t st) {
  SG_CUDA(cudaMemsetAsync(e, 0x80, sizeof(int) * cols, st));   // 0x80808080: no entry yet
  int64_t z = static_cast<int64_t>(device_sm_count()) * 8 / cols;
  const int64_t zmax = (n + 4095) / 4096;
  if (z > zmax) z = zmax;
  if (z < 1) z = 1;
  const int64_t rows = (n + z - 1) / z;
  col_exponent_kernel<<<dim3(cols, static_cast<unsigned>((n + rows - 1) / rows)), 256, 0, st>>>(
      n, X, ld, rows, e);
  SG_LAUNCH_CHECK();
}

__device__ int g_oz_err;

PFN_cuTensorMapEncodeTiled_v12000 oz_encode_fn() {
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

// FP64 column-major matrix (rows x cols, leading dimension ld), boxes of
// 16 rows x box_cols, 128-byte swizzle
bool make_map64(CUtensorMap* map, const double* ptr, int64_t rows, int64_t cols, int64_t ld,
                int box_cols) {
  auto fn = oz_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(cols)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * sizeof(double)};
  cuuint32_t box[2] = {16u, static_cast<cuuint32_t>(box_cols)};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(ptr), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// FP64 column-major matrix, boxes of 128 rows x 32 columns, no swizzle
bool make_map64_box(CUtensorMap* map, const double* ptr, int64_t rows, int64_t cols, int64_t ld) {
  auto fn = oz_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(cols)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * sizeof(double)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kUM), static_cast<cuuint32_t>(kUS)};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(ptr), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Launches of this file's tensor-core kernels since the last check: the
// check reads the device's error flag (a synchronising copy) only after
// one.  The flag stays set until read, so a timeout is reported by a later
// check even if another thread's check consumed the count.
std::atomic<int> oz_check_error_pending{0};

int* oz_err_flag() {
  static int* ptr[64] = {};
  static std::mutex mu;
  int dev = 0;
  SG_CUDA(cudaGetDevice(&dev));
  SG_REQUIRE(dev >= 0 && dev < 64, SG_ECUDA, "device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    SG_CUDA(cudaGetSymbolAddress(&p, g_oz_err));
    ptr[dev] = static_cast<int*>(p);
  }
  return ptr[dev];
}

int64_t oz_splits(int64_t n, int i, int s, int64_t* rows) {
  const int64_t tiles = static_cast<int64_t>((i + kOM - 1) / kOM) * ((s + kON - 1) / kON);
  int64_t S = static_cast<int64_t>(device_sm_count()) / tiles;
  const int64_t maxS = n / (4 * kOK);     // at least four stages per split
  if (S > maxS) S = maxS;
  // at most 2^12 level readouts per split keep the int64 halves exact
  const int64_t minS = (n + (int64_t(kOK) * kChunk << 12) - 1) / (int64_t(kOK) * kChunk << 12);
  if (S < minS) S = minS;
  if (S < 1) S = 1;
  int64_t r = (n + S - 1) / S;
  r = (r + kOK - 1) / kOK * kOK;
  if (rows) *rows = r;
  return (n + r - 1) / r;
}

// ------------------------------------------------------------- FP32 Gram
// G = X^T X of the FP32 basis (the CholQR Gram of Alg. 4) on the tensor
// cores, from exact digit slices as above.  A value x of column c is taken
// relative to the column's exponent e_c (|x| < 2^e_c) as u = x 2^(6 - e_c),
// |u| < 64, and cut in FP32 arithmetic into six balanced base-256 digits:
// d_t = u rounded to the nearest integer, then u <- 256 (u - d_t).  Every
// step is exact (u - d_t by Sterbenz, |u - d_t| <= 1/2, the scalings by
// powers of two), so |d_0| <= 64, |d_t| <= 128 and
//   x~ = 2^(e_c - 6) * sum_{t=0..5} d_t 256^-t,   |x~ - x| <= 2^(e_c - 47):
// every value within 2^23 of its column's largest is exact.  The digit
// pair (t, u) belongs to level t + u; levels 0..7 are formed (the pairs of
// levels 8..10 add less than 2^-58 max|x_m| max|x_n| to a product).  A level
// has at most six pairs, so its sum over 128 rows stays below
// 6 * 128 * 2^14 < 2^24 and is exact in the MMA's FP32 accumulator.  Every
// 128 rows the level sums are added into an exact integer per output
// (levels 0..3 and 4..7 in two int64 halves), which is rounded once:
//   G(m, n) = 2^(e_m + e_n - 68) * sum_l S_l 256^(7 - l)   (rounded to FP64).
// Against the exact Gram the error is at most
// 2^-46 (max|x_m| sum_k |x_kn| + max|x_n| sum_k |x_km|)
//   + n 2^-58 max|x_m| max|x_n| + the final rounding:
// the accuracy class of the exact-product SIMT kernel (about
// 2^-46 ||x_m|| ||x_n|| for vectors without extreme dynamic range).
//
// Tile: all s <= 128 columns of X as MMA M (operand A) against 32 of them as
// MMA N (operand B; quarter q = columns 32q .. 32q + 31), 32 rows per stage.
// Only the upper triangle is needed, so quarter q cuts and reads out the
// columns 0 .. 32q + 31 alone.  Both operands are digit slices in shared
// memory, 64-byte lines (the 32 rows of a stage of one column, 64-byte
// swizzled): A slice t holds the lines of columns 0..127, and the quarter's
// own 32 lines of each digit are stored once more, digit after digit, as
// the B slices (two more all-zero slices follow).  So one MMA of
// N = 32 (8 - t) multiplies A's digit t by B's digits 0 .. 7 - t and,
// written 32 t columns into the level sums, adds each pair (t, u) to level
// t + u: six MMAs per 16 rows.  One CTA per SM (224 KB of shared memory):
//   * warp 16 (one lane) loads each stage's columns 0 .. 32q + 31 (boxes of
//     32 rows x 32 columns, 128-byte swizzled) into a six-deep ring (a stage
//     is 4 to 16 KB, so the ring keeps enough bytes in flight to cover the
//     latency of HBM);
//   * warps 0-7 cut stage k into one of two sets of digit slices (one
//     16-byte store per digit: eight consecutive rows of one column, packed
//     two digits per conversion) while warp 17 (one lane) issues stage
//     k-1's MMAs;
//   * the level sums alternate between two sets of tensor-memory columns
//     (8 levels x 32 columns each); warps 8-15 read one set out while the
//     MMAs fill the other, so neither the cut nor the MMAs wait for them.
// Every wait is bounded, as in the kernels above.
constexpr int kGK = 32;                         // rows per stage
constexpr int kGN = 32;                         // output columns per CTA (MMA N)
constexpr int kGMaxS = 128;                     // columns of X (MMA M)
constexpr int kGDig = 6;                        // digit slices kept per value
constexpr int kGLev = 8;                        // levels 0..7
constexpr int kGChunk = 4;                      // stages per exact level sum
constexpr int kGBox = kGK * kGN * 4;            // one 32 x 32 FP32 box: 4 KB
constexpr int kGStageBytes = 4 * kGBox;         // columns 0..127 of a stage: 16 KB
constexpr int kGSliceA = kGMaxS * 64;           // A: 128 lines of 64 bytes, 8 KB
constexpr int kGSliceB = kGN * 64;              // B: 32 lines of 64 bytes, 2 KB
constexpr int kGBSlices = 8;                    // B digits 0..5 and two zero slices
constexpr int kGRing = 6;                       // staged stages in flight
constexpr int kGAOff = 0;
constexpr int kGBOff = kGAOff + kGDig * kGSliceA;
constexpr int kGBuf = kGBOff + kGBSlices * kGSliceB;   // 64 KB per set of slices
constexpr int kGSlicesOff = kGRing * kGStageBytes;     // after the staging ring
constexpr uint32_t kGSetCol = 256;              // accumulator set a at column 256 a
constexpr int kGNonFinite = 1 << 20;            // exponent of a column holding Inf or NaN
static_assert(kGLev * kGN <= static_cast<int>(kGSetCol), "a set of level sums fits its columns");

struct __align__(8) OzGShared {
  uint64_t full[kGRing], sfree[kGRing], afull[2], afree[2];
  uint64_t accfull[2], accfree[2], done;
  uint32_t tmem_base;
  int fail;
};

constexpr int kGSmem = kGSlicesOff + 2 * kGBuf + static_cast<int>(sizeof(OzGShared)) + 1024;
static_assert(kGBuf % 1024 == 0 && kGBOff % 1024 == 0 && kGSlicesOff % 1024 == 0,
              "staging boxes and slices start on 1024-byte boundaries");
static_assert(kGSmem <= 232448, "fits the 227 KB of shared memory per CTA");

__device__ __forceinline__ void mma_f16_ss(uint32_t dtmem, uint64_t a, uint64_t b,
                                           uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// This thread's lane, 8 consecutive 32-bit columns from taddr, without
// waiting for the load (tmem_wait_ld16 waits and orders the uses).
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr));
}

// Waits for this thread's tensor-memory loads; the 16 registers are operands
// so that no use of them is scheduled before the wait.
__device__ __forceinline__ void tmem_wait_ld16(uint32_t* v) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                 "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]),
                 "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
               :
               : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle (lines
// of 64 bytes, the 16-byte chunk c of line r stored at c ^ ((r >> 1) & 3)),
// 8-line groups 512 bytes apart (slice bases aligned to 1024 bytes).
__device__ __forceinline__ uint64_t sdesc64(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);  // start address
  d |= static_cast<uint64_t>(1) << 16;                 // leading byte offset (unused)
  d |= static_cast<uint64_t>(512 >> 4) << 32;          // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                 // descriptor version
  d |= static_cast<uint64_t>(4) << 61;                 // 64-byte swizzle
  return d;
}

// grid: (quarters of 32 output columns, splits of the rows)
__global__ void __launch_bounds__(kDThreads, 1)
oz_gram32_kernel(const __grid_constant__ CUtensorMap mapX, int64_t n, int s,
                 const int* __restrict__ ex, int64_t rows_per_split,
                 double* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsmem[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~static_cast<uintptr_t>(1023));
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int q = blockIdx.x;
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * rows_per_split;
  const int64_t k1 = (k0 + rows_per_split < n) ? k0 + rows_per_split : n;
  const int nk = static_cast<int>((k1 - k0 + kGK - 1) / kGK);
  auto stage = [&](int r) { return base + r * kGStageBytes; };
  auto sliceA = [&](int b, int t) { return base + kGSlicesOff + b * kGBuf + kGAOff + t * kGSliceA; };
  auto sliceB = [&](int b, int u) { return base + kGSlicesOff + b * kGBuf + kGBOff + u * kGSliceB; };
  OzGShared& sh = *reinterpret_cast<OzGShared*>(base + kGSlicesOff + 2 * kGBuf);
  auto failed = [&]() { return *reinterpret_cast<volatile int*>(&sh.fail) != 0; };
  auto group_end = [&](int k) { return (k % kGChunk) == kGChunk - 1 || k == nk - 1; };

  // warps 0-7 cut, warps 8-15 read out; of each, the two warps per group of
  // 32 tensor-memory lanes whose lanes hold columns 0 .. 32q + 31 take part
  // (the others wait at the end)
  const uint32_t nwork = static_cast<uint32_t>(64 * (q + 1));
  if (tid == 0) {
    for (int r = 0; r < kGRing; ++r) {
      mbar_init(&sh.full[r], 1);
      mbar_init(&sh.sfree[r], nwork);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.afull[b], nwork);
      mbar_init(&sh.afree[b], 1);
      mbar_init(&sh.accfull[b], 1);
      mbar_init(&sh.accfree[b], nwork);
    }
    mbar_init(&sh.done, 1);
    sh.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh.tmem_base)),
                 "r"(kOTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // never written: the A lines beyond column 32q + 31 (they feed MMA rows
  // whose outputs are not read) and B slices 6 and 7; zero them once
  if (warp < kDWarps) {
    const int l0 = kGN * (q + 1);
    const int per = (kGMaxS - l0) * 4;               // 16-byte words per A slice
    for (int e = tid; e < 2 * kGDig * per; e += kDSplit) {
      const int sl = e / per, w = e % per;
      *reinterpret_cast<uint4*>(sliceA(sl / kGDig, sl % kGDig) + l0 * 64 + w * 16) =
          make_uint4(0, 0, 0, 0);
    }
    constexpr int perB = (kGBSlices - kGDig) * kGSliceB / 16;
    for (int e = tid; e < 2 * perB; e += kDSplit)
      *reinterpret_cast<uint4*>(sliceB(e / perB, kGDig) + (e % perB) * 16) = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh.tmem_base;

  // Warp w (w < 16) covers the tensor-memory lanes, i.e. columns,
  // m = 32 (w % 4) + lane; half = (w / 4) % 2.  A cutting warp (w < 8) cuts
  // rows 16 half .. + 15 of each stage of column m; a reading warp (w >= 8)
  // owns the outputs (m, 32q + 16 half + c), c < 16, each as two int64
  // halves: ahi = sum of S_l 256^(3-l) over l = 0..3, alo = sum of
  // S_l 256^(7-l) over l = 4..7 (|S_l| < 2^24: each half grows by < 2^48.1
  // per readout and stays exact for 2^14 readouts); V = ahi 2^32 + alo
  const int m = (warp & 3) * 32 + lane;
  const int half = (warp >> 2) & 1;
  const bool mine = (warp & 3) <= q;   // columns 32 (w % 4) .. + 31 are within 0 .. 32q + 31
  const bool cutter = warp < kDWarps / 2;
  int64_t alo[16];
  int64_t ahi[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) { alo[c] = 0; ahi[c] = 0; }
  auto readout = [&](int g) -> bool {
    const int a = g & 1;
    if (!mbar_wait(&sh.accfull[a], static_cast<uint32_t>((g >> 1) & 1))) sh.fail = 1;
    if (__any_sync(0xffffffffu, failed())) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tl = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16) +
                        static_cast<uint32_t>(a) * kGSetCol + static_cast<uint32_t>(half * 16);
#pragma unroll
    for (int L = 0; L < kGLev; ++L) {
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        uint32_t v[8];
        tmem_ld8(tl + static_cast<uint32_t>(kGN * L + 8 * hh), v);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int64_t sv = level_int(v[c]);
          if (L < 4) ahi[8 * hh + c] += sv * (int64_t(1) << (8 * (3 - L)));
          else alo[8 * hh + c] += sv * (int64_t(1) << (8 * (7 - L)));
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    mbar_arrive(&sh.accfree[a]);
    return true;
  };

  if (warp == kDWarps) {
    // ------------------------------------------------ TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int k = 0; k < nk; ++k) {
        if (failed()) break;
        const int r = k % kGRing;
        if (k >= kGRing &&
            !mbar_wait(&sh.sfree[r], static_cast<uint32_t>((k / kGRing - 1) & 1))) {
          sh.fail = 1;
          break;
        }
        const int x = static_cast<int>(k0 + static_cast<int64_t>(k) * kGK);
        mbar_expect_tx(&sh.full[r], static_cast<uint32_t>((q + 1) * kGBox));
        for (int c = 0; c <= q; ++c)
          tma_load_2d(stage(r) + c * kGBox, &mapX, &sh.full[r], x, kGN * c);
        issued = k + 1;
      }
      if (failed()) {
        // drain this CTA's copies in flight: the last stage issued into each
        // slot (stages issued - kGRing .. issued - 1)
        for (int k = issued - kGRing > 0 ? issued - kGRing : 0; k < issued; ++k)
          mbar_wait(&sh.full[k % kGRing], static_cast<uint32_t>((k / kGRing) & 1));
      }
    }
  } else if (warp == kDWarps + 1) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      int grp = 0;
      for (int k = 0; k < nk; ++k) {
        if (failed()) break;
        const int b = k & 1;
        const uint32_t a = static_cast<uint32_t>(grp & 1);
        const bool fresh = (k % kGChunk) == 0;
        if (!mbar_wait(&sh.afull[b], static_cast<uint32_t>((k >> 1) & 1)) ||
            (fresh && grp >= 2 &&
             !mbar_wait(&sh.accfree[a], static_cast<uint32_t>(((grp >> 1) - 1) & 1)))) {
          sh.fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t bd0 = sdesc64(smem_u32(sliceB(b, 0)));
#pragma unroll 1
        for (int kk = 0; kk < kGK / 16; ++kk) {
#pragma unroll
          for (int t = 0; t < kGDig; ++t) {
            // A's digit t against B's digits 0 .. 7 - t: output column
            // 32 u + c holds the pair (t, u), level t + u at column
            // 32 (t + u) + c of the set; the first MMA of a group (t = 0,
            // all eight levels) starts the sums afresh
            const uint64_t ad = sdesc64(smem_u32(sliceA(b, t))) + static_cast<uint64_t>((kk * 32) >> 4);
            const uint32_t acc = (!fresh || kk > 0 || t > 0) ? 1u : 0u;
            mma_f16_ss(tmem + a * kGSetCol + static_cast<uint32_t>(kGN * t), ad,
                       bd0 + static_cast<uint64_t>((kk * 32) >> 4), idesc_f16(kGMaxS, kGN * (kGLev - t)),
                       acc);
          }
        }
        mma_commit(&sh.afree[b]);     // slices b reusable
        if (group_end(k)) {
          mma_commit(&sh.accfull[a]);
          ++grp;
        }
      }
      mma_commit(&sh.done);
    }
  } else if (mine && cutter) {
    // ------------------------------------------------ cut
    const int em = m < s ? ex[m] : -4000;
    // u = x 2^(6 - e) as two exact power-of-two scalings, both factors
    // normal; columns that are all zero, beyond s or hold an Inf or a NaN
    // are cut as zeros
    const bool live = em > -2000 && em < kGNonFinite;
    const int eb = (live && em < -50) ? 64 : 0;
    const float f1 = __int_as_float((127 + eb) << 23);
    const float f2 = live ? __int_as_float((127 + 6 - em - eb) << 23) : 0.0f;
    constexpr float kRound = 12582912.0f;   // 1.5 2^23: adding it rounds |v| < 2^22 to an integer
    for (int k = 0; k < nk; ++k) {
      const int b = k & 1;
      const int r = k % kGRing;
      bool bad = failed();
      if (!bad) {
        const bool ok = mbar_wait(&sh.full[r], static_cast<uint32_t>((k / kGRing) & 1)) &&
                        (k < 2 || mbar_wait(&sh.afree[b], static_cast<uint32_t>(((k >> 1) - 1) & 1)));
        if (!ok) {
          sh.fail = 1;
          bad = true;
        }
      }
      if (__any_sync(0xffffffffu, bad)) break;
#pragma unroll
      for (int gg = 0; gg < 2; ++gg) {
        // column m's rows 8 cg .. + 7 (cg = 2 half + gg): chunks 2 cg,
        // 2 cg + 1 of its 128-byte swizzled line in the staged boxes
        const int cg = 2 * half + gg;
        const unsigned char* line = stage(r) + m * 128;
        const uint4 r0 = *reinterpret_cast<const uint4*>(line + (((2 * cg) ^ (m & 7)) << 4));
        const uint4 r1 = *reinterpret_cast<const uint4*>(line + (((2 * cg + 1) ^ (m & 7)) << 4));
        const uint32_t v[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        uint32_t words[kGDig][4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          // rows 2p (low half) and 2p + 1 (high half) of the word
          float ua = live ? __fmul_rn(__fmul_rn(__uint_as_float(v[2 * p]), f1), f2) : 0.0f;
          float ub = live ? __fmul_rn(__fmul_rn(__uint_as_float(v[2 * p + 1]), f1), f2) : 0.0f;
#pragma unroll
          for (int t = 0; t < kGDig; ++t) {
            const float da = __fsub_rn(__fadd_rn(ua, kRound), kRound);
            const float db = __fsub_rn(__fadd_rn(ub, kRound), kRound);
            const __half2 h = __floats2half2_rn(da, db);
            words[t][p] = *reinterpret_cast<const uint32_t*>(&h);
            if (t + 1 < kGDig) {
              ua = __fmul_rn(__fsub_rn(ua, da), 256.0f);
              ub = __fmul_rn(__fsub_rn(ub, db), 256.0f);
            }
          }
        }
        // digit t of the eight rows: K chunk cg of line m of A slice t (and
        // of line m - 32q of B slice t for the quarter's own columns);
        // 64-byte swizzle: chunk cg of line r sits at cg ^ ((r >> 1) & 3)
        const int off = (cg ^ ((m >> 1) & 3)) << 4;
        unsigned char* dst = sliceA(b, 0) + m * 64 + off;
#pragma unroll
        for (int t = 0; t < kGDig; ++t)
          *reinterpret_cast<uint4*>(dst + t * kGSliceA) =
              make_uint4(words[t][0], words[t][1], words[t][2], words[t][3]);
        if ((warp & 3) == q) {
          unsigned char* dstb = sliceB(b, 0) + lane * 64 + off;
#pragma unroll
          for (int t = 0; t < kGDig; ++t)
            *reinterpret_cast<uint4*>(dstb + t * kGSliceB) =
                make_uint4(words[t][0], words[t][1], words[t][2], words[t][3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&sh.sfree[r]);
      mbar_arrive(&sh.afull[b]);
    }
  } else if (mine) {
    // ------------------------------------------------ readout
    const int ngroups = (nk + kGChunk - 1) / kGChunk;
    for (int g = 0; g < ngroups; ++g)
      if (!readout(g)) break;
  }
  // (twice the limit: after a failure the MMA warp may first spend one
  // limit on a step that never came)
  if (warp < 4 && !mbar_wait(&sh.done, 0, 2 * kWaitNs)) sh.fail = 1;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  const bool good = !sh.fail;
  if (!good) {
    if (tid == 0) atomicExch(err, 1);
  } else if (warp < kDWarps && !cutter && mine && m < s) {
    double* P = part + static_cast<int64_t>(blockIdx.y) * s * s;
    const int em = ex[m];
#pragma unroll
    for (int cc = 0; cc < 16; ++cc) {
      const int nn = kGN * q + 16 * half + cc;
      if (m <= nn && nn < s) {
        const int en = ex[nn];
        double val;
        if (em >= kGNonFinite || en >= kGNonFinite) {
          val = __longlong_as_double(0x7FF8000000000000ll);   // an Inf or NaN in either column
        } else if (em < -2000 || en < -2000) {
          val = 0.0;                                         // an all-zero column
        } else {
          // V = (ahi + carry) 2^32 + the low 32 bits of alo, rounded once
          const int64_t hi = ahi[cc] + (alo[cc] >> 32);
          const uint32_t lo = static_cast<uint32_t>(alo[cc]);
          val = int96_to_double(hi, lo, em + en - 68);
        }
        P[m + static_cast<int64_t>(nn) * s] = val;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kOTmemCols)
                 : "memory");
  }
}

// e[c] for FP32 columns: the exponent of the largest magnitude (|x| < 2^e),
// or kGNonFinite when the column holds an Inf or a NaN, merged with
// atomicMax like the FP64 kernel (all-zero columns keep the start value).
__global__ void __launch_bounds__(256)
col_exponent32_kernel(int64_t n, const float* __restrict__ X, int64_t ld, int64_t rows,
                      int* __restrict__ e) {
  const uint32_t* col = reinterpret_cast<const uint32_t*>(X + static_cast<int64_t>(blockIdx.x) * ld);
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * rows;
  const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
  // |x| orders like its bit pattern with the sign cleared; Inf and NaN
  // patterns lie above every finite one
  uint32_t mx = 0;
  auto take = [&](uint32_t b) {
    b &= 0x7FFFFFFFu;
    mx = b > mx ? b : mx;
  };
  int64_t r = r0;
  int64_t head = 0;   // elements before the first 16-byte boundary
  while (r + head < r1 && (reinterpret_cast<uintptr_t>(col + r + head) & 15)) ++head;
  if (threadIdx.x < head) take(__ldg(col + r + threadIdx.x));
  r += head;
  const uint4* p4 = reinterpret_cast<const uint4*>(col + r);
  const int64_t nq4 = (r1 - r) / 4;
  for (int64_t p = threadIdx.x; p < nq4; p += 4 * 256) {
    uint4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      v[u] = (p + u * 256 < nq4) ? __ldg(p4 + p + u * 256) : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      take(v[u].x);
      take(v[u].y);
      take(v[u].z);
      take(v[u].w);
    }
  }
  for (int64_t t = r + 4 * nq4 + threadIdx.x; t < r1; t += 256) take(__ldg(col + t));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const uint32_t o = __shfl_xor_sync(0xffffffffu, mx, off);
    mx = o > mx ? o : mx;
  }
  __shared__ uint32_t wm[8];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tb = 0;
    for (int w = 0; w < 8; ++w) tb = wm[w] > tb ? wm[w] : tb;
    if (tb >= 0x7F800000u) {
      atomicMax(e + blockIdx.x, kGNonFinite);
    } else if (tb != 0) {
      const int E = static_cast<int>(tb >> 23);   // |x| < 2^(E - 126); subnormals < 2^-126
      atomicMax(e + blockIdx.x, E == 0 ? -126 : E - 126);
    }
  }
}

void col_exponents32(int64_t n, const float* X, int64_t ld, int cols, int* e, cudaStream_t st) {
  SG_CUDA(cudaMemsetAsync(e, 0x80, sizeof(int) * cols, st));   // 0x80808080: no entry yet
  int64_t z = static_cast<int64_t>(device_sm_count()) * 8 / cols;
  const int64_t zmax = (n + 4095) / 4096;
  if (z > zmax) z = zmax;
  if (z < 1) z = 1;
  const int64_t rows = (n + z - 1) / z;
  col_exponent32_kernel<<<dim3(cols, static_cast<unsigned>((n + rows - 1) / rows)), 256, 0, st>>>(
      n, X, ld, rows, e);
  SG_LAUNCH_CHECK();
}

// FP32 column-major matrix (rows x cols, leading dimension ld), boxes of
// 32 rows x 32 columns, 128-byte swizzle
bool make_map32_gram(CUtensorMap* map, const float* ptr, int64_t rows, int64_t cols, int64_t ld) {
  auto fn = oz_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(rows), static_cast<cuuint64_t>(cols)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * sizeof(float)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kGK), static_cast<cuuint32_t>(kGN)};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

int64_t oz_gram32_splits(int64_t n, int s, int64_t* rows) {
  const int64_t nq = (s + kGN - 1) / kGN;
  int64_t S = static_cast<int64_t>(device_sm_count()) / nq;
  const int64_t maxS = n / (4 * kGK);     // at least four stages per split
  if (S > maxS) S = maxS;
  // at most 2^14 level readouts per split keep the int64 halves exact
  const int64_t span = int64_t(kGK) * kGChunk << 14;
  const int64_t minS = (n + span - 1) / span;
  if (S < minS) S = minS;
  if (S < 1) S = 1;
  int64_t r = (n + S - 1) / S;
  r = (r + kGK - 1) / kGK * kGK;
  if (rows) *rows = r;
  return (n + r - 1) / r;
}

}  // namespace

bool oz_dot_supported(int64_t n, const double* Q, int64_t ldq, int i, const double* X,
                      int64_t ldx, int s) {
  if (n < 8 * kOK || i < 1 || s < 1) return false;
  if ((reinterpret_cast<uintptr_t>(Q) | reinterpret_cast<uintptr_t>(X)) & 15) return false;
  if (((ldq * 8) & 15) || ((ldx * 8) & 15)) return false;
  if (n > (int64_t(1) << 31) - 1) return false;
  return oz_encode_fn() != nullptr;
}

// Whether the tensor-core form is expected to beat the FP64-pipe kernel:
// a tile of 128 x 32 outputs costs about kStageUs per 32 rows on one SM
// (measured 2.2 .. 2.4 us over i = 13 .. 240) plus kFixedUs of setup (the
// exponent and reduction launches, barriers, tensor memory), the FP64-pipe
// kernels about
// 1 TFLOP/s (2 n i s flops; the symmetric Gram n s (s+1)) plus their
// streams of Q and X at about 2 TB/s.
bool oz_dot_pays(int64_t n, int i, int s, bool sym) {
  constexpr double kStageUs = 2.4, kFixedUs = 15.0;
  const double tiles = static_cast<double>((i + kOM - 1) / kOM) * ((s + kON - 1) / kON);
  const double t_oz = (static_cast<double>((n + kOK - 1) / kOK) * tiles * kStageUs /
                           static_cast<double>(device_sm_count()) +
                       kFixedUs) * 1e-6;
  const double flops = sym ? static_cast<double>(n) * s * (s + 1.0)
                           : 2.0 * static_cast<double>(n) * i * s;
  const double bytes = static_cast<double>(n) * (sym ? s : i + s) * 8.0;
  return t_oz < 0.9 * (flops / 1.0e12 + bytes / 2.0e12);
}

int64_t oz_dot_part_size(int64_t n, int i, int s) {
  return oz_splits(n, i, s, nullptr) * i * s;
}

int64_t oz_exp_ints(int i, int s) { return static_cast<int64_t>(i) + s; }

bool oz_update_supported(int64_t n, const double* Q, int64_t ldq, int i, const double* X,
                         int64_t ldx, int s) {
  if (n < 4 * kUM || i < 1 || i > kUMaxK || s < 1) return false;
  if ((reinterpret_cast<uintptr_t>(Q) | reinterpret_cast<uintptr_t>(X)) & 15) return false;
  if (((ldq * 8) & 15) || ((ldx * 8) & 15)) return false;
  if (n > (int64_t(1) << 31) - 1) return false;
  return oz_encode_fn() != nullptr;
}

// Whether the tensor-core update is expected to beat the FP64-pipe kernel.
// One SM takes ceil(row tiles / row groups) tiles of 128 rows x 32 columns,
// each about kTileUs (readout, epilogue, pipeline fill) plus kStepUs per
// 16 columns of Q (measured: 7.7 us at 1 step, 14.6 us at 7, 23.4 us at 15),
// plus kFixedUs of setup (the exponent launch, W's digits, tensor memory).
// The FP64-pipe kernels sustain about 1.05 TFLOP/s (2 n i s flops, half
// for the triangle); the tiled one adds its streams of Q and X at about
// 2 TB/s, the narrow-Q one (i <= 16) overlaps them at about 5.5 TB/s.
bool oz_update_pays(int64_t n, int i, int s, bool upper) {
  constexpr double kTileUs = 6.6, kStepUs = 1.12, kFixedUs = 15.0;
  const int64_t ct = (s + kUN - 1) / kUN;
  const int64_t ntiles = (n + kUM - 1) / kUM;
  int64_t G = static_cast<int64_t>(device_sm_count()) / ct;
  if (G < 1) G = 1;
  if (G > ntiles) G = ntiles;
  const double per_sm = static_cast<double>((ntiles + G - 1) / G) *
                        ((ct + device_sm_count() - 1) / device_sm_count());
  const double t_oz = (per_sm * (kTileUs + kStepUs * ((i + 15) / 16)) + kFixedUs) * 1e-6;
  const double flops = (upper ? 1.0 : 2.0) * static_cast<double>(n) * i * s;
  const double bytes = static_cast<double>(n) * (i + 2.0 * s) * 8.0;
  const double t_fp64 = i <= 16 ? std::max(flops / 1.05e12, bytes / 5.5e12)
                                : flops / 1.05e12 + bytes / 2.0e12;
  return t_oz < 0.9 * t_fp64;
}

void oz_update(int64_t n, const double* Q, int64_t ldq, int i, const double* W, int ldw,
               double* X, int64_t ldx, int s, double alpha, double beta, bool upper, int* exps,
               cudaStream_t st) {
  int* err = oz_err_flag();
  col_exponents(n, Q, ldq, i, exps, st);
  CUtensorMap mq, mx;
  SG_REQUIRE(make_map64_box(&mq, Q, n, i, ldq) && make_map64_box(&mx, X, n, s, ldx), SG_ECUDA,
             "cuTensorMapEncodeTiled failed");
  ensure_dynamic_smem(reinterpret_cast<const void*>(oz_update_kernel), oz_update_smem(kUMaxK));
  const int ct = (s + kUN - 1) / kUN;
  const int64_t ntiles = (n + kUM - 1) / kUM;
  int64_t G = static_cast<int64_t>(device_sm_count()) / ct;
  if (G < 1) G = 1;
  if (G > ntiles) G = ntiles;
  dim3 grid(static_cast<unsigned>(ct), static_cast<unsigned>(G));
  oz_update_kernel<<<grid, kUThreads, oz_update_smem(i), st>>>(
      mq, mx, n, i, s, W, ldw, X, ldx, alpha, beta, upper ? 1 : 0, exps, err);
  SG_LAUNCH_CHECK();
  oz_check_error_pending.fetch_add(1);
}

void oz_check_error(cudaStream_t st) {
  if (oz_check_error_pending.exchange(0) == 0) return;
  int* f = oz_err_flag();
  int host = 0;
  SG_CUDA(cudaMemcpyAsync(&host, f, sizeof(int), cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  if (host) {
    SG_CUDA(cudaMemsetAsync(f, 0, sizeof(int), st));
    throw Error(SG_ECUDA, "tensor-core FP64 block dot: a bounded wait ran out");
  }
}

void oz_dot(int64_t n, const double* Q, int64_t ldq, int i, const double* X, int64_t ldx,
            int s, int* exps, double* part, int64_t part_cap, int* nsplit, cudaStream_t st) {
  int* err = oz_err_flag();
  int64_t rows = 0;
  const int64_t S = oz_splits(n, i, s, &rows);
  SG_REQUIRE(S * i * s <= part_cap, SG_EINVAL, "oz_dot: workspace too small");
  int* eq = exps;
  int* ex = exps + i;
  col_exponents(n, Q, ldq, i, eq, st);
  if (X == Q && s <= i)
    SG_CUDA(cudaMemcpyAsync(ex, eq, sizeof(int) * s, cudaMemcpyDeviceToDevice, st));
  else
    col_exponents(n, X, ldx, s, ex, st);
  CUtensorMap mq, mx;
  SG_REQUIRE(make_map64(&mq, Q, n, i, ldq, kOM) && make_map64(&mx, X, n, s, ldx, kON), SG_ECUDA,
             "cuTensorMapEncodeTiled failed");
  ensure_dynamic_smem(reinterpret_cast<const void*>(oz_dot_kernel), kOzSmem);
  dim3 grid((i + kOM - 1) / kOM, (s + kON - 1) / kON, static_cast<unsigned>(S));
  oz_dot_kernel<<<grid, kDThreads, kOzSmem, st>>>(mq, mx, n, i, s, eq, ex, rows, part, err);
  SG_LAUNCH_CHECK();
  oz_check_error_pending.fetch_add(1);
  *nsplit = static_cast<int>(S);
}

bool oz_gram32_supported(int64_t n, const float* X, int64_t ldx, int s) {
  if (n < 8 * kGK || s < 1 || s > kGMaxS) return false;
  if (reinterpret_cast<uintptr_t>(X) & 15) return false;
  if ((ldx * 4) & 15) return false;
  if (n > (int64_t(1) << 31) - 1) return false;
  return oz_encode_fn() != nullptr;
}

// Expected time of the tensor-core Gram: one CTA per SM takes a quarter of
// 32 output columns through stages of 32 rows at about kStageUs each
// (measured 1.6 us at n = 2^19 .. 2^21, s = 16 .. 128, whatever the
// quarter: a warp reaches the tensor-memory lanes of its own scheduler
// only, so each group of 32 columns is read out, and its columns cut, by
// one scheduler's warps, and their instruction issue, not the MMAs, sets
// the pace), plus kFixedUs of setup (the exponent and reduction launches,
// tensor memory).
double oz_gram32_seconds(int64_t n, int s) {
  constexpr double kStageUs = 1.6, kFixedUs = 15.0;
  const double nq = static_cast<double>((s + kGN - 1) / kGN);
  return (static_cast<double>((n + kGK - 1) / kGK) * nq * kStageUs /
              static_cast<double>(device_sm_count()) +
          kFixedUs) * 1e-6;
}

int64_t oz_gram32_part_size(int64_t n, int s) {
  return oz_gram32_splits(n, s, nullptr) * s * s;
}

void oz_gram32(int64_t n, const float* X, int64_t ldx, int s, int* exps, double* part,
               int64_t part_cap, int* nsplit, cudaStream_t st) {
  int* err = oz_err_flag();
  int64_t rows = 0;
  const int64_t S = oz_gram32_splits(n, s, &rows);
  SG_REQUIRE(S * s * s <= part_cap, SG_EINVAL, "oz_gram32: workspace too small");
  col_exponents32(n, X, ldx, s, exps, st);
  CUtensorMap mx;
  SG_REQUIRE(make_map32_gram(&mx, X, n, s, ldx), SG_ECUDA, "cuTensorMapEncodeTiled failed");
  ensure_dynamic_smem(reinterpret_cast<const void*>(oz_gram32_kernel), kGSmem);
  dim3 grid((s + kGN - 1) / kGN, static_cast<unsigned>(S));
  oz_gram32_kernel<<<grid, kDThreads, kGSmem, st>>>(mx, n, s, exps, rows, part, err);
  SG_LAUNCH_CHECK();
  oz_check_error_pending.fetch_add(1);
  *nsplit = static_cast<int>(S);
}

}  // namespace sg
