// Tall-skinny dense kernels of the block orthogonalisation (Alg. 4):
//   block_dot:    W = Q^T X   (BCGS projections and the CholQR Gram
//                 matrices), a reduction over the n rows split across
//                 CTAs with per-split partial tiles summed in fixed order;
//   block_update: X = beta X + alpha Q W (BCGS update; with an upper
//                 triangular W = Z^-1 it is the CholQR product V Z^-1).
//
// FP64 on this chip is bound by the FP64 pipe, not by HBM (the arithmetic
// intensity of W = Q^T X is ~i s / (4 (i+s)) flop/B), so the tiles are
// small (32 x 32 outputs per CTA, 2 x 2 per thread): the FP64 pipe stays
// saturated while padding waste and the Gram matrices' redundant lower
// tiles stay small.  Narrow shapes get their own tiles: for i <= 8 a
// warp-per-row layout lets whole warps skip padded rows, and for s <= 8 a
// 64 x 8 tile reads Q once without padding the columns.
//
// FP32 data: projections accumulate in FP32 per 32-row stage and fold the
// stage sums into a compensated total; Gram matrices (EXACT) form every
// product exactly (p = a b rounded plus its FMA remainder) and add it with
// a two-sum, so the Gram of FP32 vectors is accurate to about eps_32^2
// relative to the sum of |products| -- the accuracy the partial Cholesky
// bound of the FP32 basis relies on.
#include <atomic>
#include <cstdlib>

#include "sg_internal.h"

namespace sg {

namespace {

constexpr int kThreads = 256;
constexpr int BK = 32;  // rows of Q/X per shared-memory stage

// two-sum: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// C_part[z] (M x N, column-major) = A(k0:k1, :)^T B(k0:k1, :)
// Tile BM x BN, thread tile TM x TN; MW: thread rows vary across warps
// (whole warps idle on padded rows).
template <int BM, int BN, int TM, int TN, bool MW, bool EXACT, typename T>
__global__ void __launch_bounds__(kThreads)
dot_tile_kernel(int64_t K, int M, int N, const T* __restrict__ A,
                int64_t lda, const T* __restrict__ B, int64_t ldb,
                double* __restrict__ part, int64_t rows_per_split, int sym) {
  constexpr bool kF32 = sizeof(T) == 4;
  constexpr int TMN = BM / TM, TNN = BN / TN;
  static_assert(TMN * TNN == kThreads, "thread layout");
  if (sym && blockIdx.x > blockIdx.y) return;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int64_t k0 = blockIdx.z * rows_per_split;
  const int64_t k1 = (k0 + rows_per_split < K) ? k0 + rows_per_split : K;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = MW ? tid / TNN : tid % TMN;
  const int ty = MW ? tid % TNN : tid / TMN;
  const bool active = (m0 + tx * TM) < M;
  T acc[TM][TN], comp[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) { acc[a][b] = T(0); comp[a][b] = T(0); }
  for (int64_t kb = k0; kb < k1; kb += BK) {
    for (int e = tid; e < BK * BM; e += kThreads) {
      const int kk = e % BK, mm = e / BK;
      const int64_t k = kb + kk;
      const int m = m0 + mm;
      As[kk][mm] = (k < k1 && m < M) ? A[k + m * lda] : T(0);
    }
    for (int e = tid; e < BK * BN; e += kThreads) {
      const int kk = e % BK, nn = e / BK;
      const int64_t k = kb + kk;
      const int nc = n0 + nn;
      Bs[kk][nn] = (k < k1 && nc < N) ? B[k + nc * ldb] : T(0);
    }
    __syncthreads();
    if (active) {
      if (EXACT) {
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
          T av[TM], bv[TN];
#pragma unroll
          for (int a = 0; a < TM; ++a) av[a] = As[kk][tx * TM + a];
#pragma unroll
          for (int b = 0; b < TN; ++b) bv[b] = Bs[kk][ty * TN + b];
#pragma unroll
          for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TN; ++b) {
              const float p = av[a] * bv[b];
              const float pe = fmaf(av[a], bv[b], -p);  // exact remainder
              float s, e;
              two_sum(acc[a][b], p, s, e);
              acc[a][b] = s;
              comp[a][b] += e + pe;
            }
        }
      } else {
        T st[TM][TN];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TN; ++b) st[a][b] = kF32 ? T(0) : acc[a][b];
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
          T av[TM], bv[TN];
#pragma unroll
          for (int a = 0; a < TM; ++a) av[a] = As[kk][tx * TM + a];
#pragma unroll
          for (int b = 0; b < TN; ++b) bv[b] = Bs[kk][ty * TN + b];
#pragma unroll
          for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int b = 0; b < TN; ++b) st[a][b] = fma(av[a], bv[b], st[a][b]);
        }
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TN; ++b) {
            if (kF32) {  // compensated fold of the stage sum: acc - comp
              const T y = st[a][b] - comp[a][b];
              const T t = acc[a][b] + y;
              comp[a][b] = (t - acc[a][b]) - y;
              acc[a][b] = t;
            } else {
              acc[a][b] = st[a][b];
            }
          }
      }
    }
    __syncthreads();
  }
  double* P = part + static_cast<int64_t>(blockIdx.z) * M * N;
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int m = m0 + tx * TM + a, nc = n0 + ty * TN + b;
      if (m < M && nc < N) {
        double v;
        if (EXACT) v = static_cast<double>(acc[a][b]) + static_cast<double>(comp[a][b]);
        else v = static_cast<double>(acc[a][b]) - static_cast<double>(comp[a][b]);
        P[m + static_cast<int64_t>(nc) * M] = v;
      }
    }
}

// Small FP64 products (8 < i, i s <= 256, or the upper triangle of a Gram
// with s (s + 1) / 2 <= 256): one thread per needed output -- a padded tile
// would issue FP64 instructions for idle lanes, which cost the same pipe
// time on this chip -- and only as many warps as there are outputs.  Each
// block stages BK rows of Q and X in shared memory per step and adds its
// row split's products in row order; the splits are reduced in a fixed
// order afterwards (the lower triangle of a Gram is not written).
constexpr int kSmallOut = 256;
constexpr int kSmallCols = 160;   // M + N: the staged rows fit 48 KB of shared memory

__global__ void __launch_bounds__(kSmallOut)
dot_small_kernel(int64_t K, int M, int N, const double* __restrict__ A, int64_t lda,
                 const double* __restrict__ B, int64_t ldb, double* __restrict__ part,
                 int64_t rows_per_split, int sym) {
  extern __shared__ double small_smem[];
  double* As = small_smem;                     // BK x (M + 1)
  double* Bs = small_smem + BK * (M + 1);      // BK x (N + 1)
  const int64_t k0 = blockIdx.x * rows_per_split;
  const int64_t k1 = (k0 + rows_per_split < K) ? k0 + rows_per_split : K;
  const int tid = threadIdx.x;
  const int nout = sym ? N * (N + 1) / 2 : M * N;
  // this thread's output (a, b): row-major over (a, b) with b fastest;
  // for the Gram, the upper triangle a <= b row by row
  int a = 0, b = 0;
  if (sym) {
    int t = tid, row = 0;
    while (row < N && t >= N - row) { t -= N - row; ++row; }
    a = row;
    b = row + t;
  } else {
    a = tid / N;
    b = tid % N;
  }
  const bool live = tid < nout;
  double acc = 0.0;
  for (int64_t kb = k0; kb < k1; kb += BK) {
    for (int e = tid; e < BK * M; e += blockDim.x) {
      const int kk = e % BK, mm = e / BK;
      const int64_t k = kb + kk;
      As[kk * (M + 1) + mm] = k < k1 ? A[k + mm * lda] : 0.0;
    }
    for (int e = tid; e < BK * N; e += blockDim.x) {
      const int kk = e % BK, nn = e / BK;
      const int64_t k = kb + kk;
      Bs[kk * (N + 1) + nn] = k < k1 ? B[k + nn * ldb] : 0.0;
    }
    __syncthreads();
    if (live) {
#pragma unroll 8
      for (int kk = 0; kk < BK; ++kk) acc = fma(As[kk * (M + 1) + a], Bs[kk * (N + 1) + b], acc);
    }
    __syncthreads();
  }
  if (live) part[static_cast<int64_t>(blockIdx.x) * M * N + a + static_cast<int64_t>(b) * M] = acc;
}

// W(m, n) = sum_z part[z](m, n); sym reads the upper element for both
// (m, n) and (n, m).  One warp per output: lane l adds splits l, l+32, ...
// in order, then a fixed xor-shuffle tree combines the lanes, so the
// result is deterministic and the S loads are issued 32 at a time.
__global__ void reduce_parts_kernel(int M, int N, int S,
                                    const double* __restrict__ part,
                                    double* __restrict__ W, int ldw, int sym) {
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= static_cast<int64_t>(M) * N) return;
  const int m = static_cast<int>(gw % M), n = static_cast<int>(gw / M);
  int sm = m, sn = n;
  if (sym && m > n) { sm = n; sn = m; }
  double acc = 0.0;
  const int64_t MN = static_cast<int64_t>(M) * N;
  const double* p = part + sm + static_cast<int64_t>(sn) * M;
  for (int z = lane; z < S; z += 32) acc += p[z * MN];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) W[m + static_cast<int64_t>(n) * ldw] = acc;
}

void launch_reduce(int M, int N, int S, const double* part, double* W, int ldw,
                   bool sym, cudaStream_t st) {
  const int64_t threads = static_cast<int64_t>(M) * N * 32;
  reduce_parts_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, st>>>(
      M, N, S, part, W, ldw, sym ? 1 : 0);
  SG_LAUNCH_CHECK();
}

// Gram matrix of FP32 vectors, G = X^T X, with the products of the
// EXACT path (p = a b rounded plus its FMA remainder, two-sum accumulation)
// but without the square tiles' waste: a thread owns one 4 x 4 block
// (bi <= bj) of the upper triangle, the blocks numbered column by column
// (block t = bj (bj + 1) / 2 + bi), so only the diagonal blocks compute
// entries below the diagonal.  CTA (p, z) takes blocks p*T .. p*T+T-1
// (T = min(128, the triangle rounded up to whole warps) threads) over rows
// [z rows, (z+1) rows): it stages each 32-row slab of the
// columns its blocks touch in shared memory (rows padded to 16 bytes) and
// a thread forms 16 exact products per row from one float4 of each side.
// The triangle's parts of one split are adjacent in launch order, so they
// share the split's rows through L2.  The partial of split z holds the
// upper triangle (entry (m, n), m <= n, at m + n s).
constexpr int kGramMaxS = 128;
constexpr int kGramBK = 32;
constexpr int kGramThreads = 128;

__host__ __device__ constexpr int gram_blocks(int s) { return ((s + 3) / 4) * ((s + 3) / 4 + 1) / 2; }

template <int LDS>
__global__ void __launch_bounds__(kGramThreads)
gram_exact_kernel(int64_t K, int s, const float* __restrict__ X, int64_t ldx,
                  double* __restrict__ part, int64_t rows_per_split) {
  // the slab: kGramBK rows of LDS floats (at least the columns, padded to a
  // multiple of 4, plus 4; a compile-time stride keeps the addressing in the
  // instructions' offsets)
  constexpr int lds = LDS;
  extern __shared__ __align__(16) float Ss[];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // block of the triangle
  const int nb = gram_blocks(s);
  // block t -> (bi, bj), bi <= bj
  int bj = static_cast<int>((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while (bj > 0 && bj * (bj + 1) / 2 > t) --bj;
  while ((bj + 1) * (bj + 2) / 2 <= t) ++bj;
  const int bi = t - bj * (bj + 1) / 2;
  const bool active = t < nb;
  // columns this CTA reads: 0 .. 4 (last block's bj + 1)
  int tl = blockIdx.x * blockDim.x + blockDim.x - 1;
  if (tl > nb - 1) tl = nb - 1;
  int bjl = static_cast<int>((sqrtf(8.0f * tl + 1.0f) - 1.0f) * 0.5f);
  while (bjl > 0 && bjl * (bjl + 1) / 2 > tl) --bjl;
  while ((bjl + 1) * (bjl + 2) / 2 <= tl) ++bjl;
  const int ncol = 4 * (bjl + 1);
  const int64_t k0 = blockIdx.y * rows_per_split;
  const int64_t k1 = (k0 + rows_per_split < K) ? k0 + rows_per_split : K;
  const float* pa = Ss + 4 * bi;
  const float* pb = Ss + 4 * bj;
  float acc[4][4], comp[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b] = 0.0f; comp[a][b] = 0.0f; }
  for (int64_t kb = k0; kb < k1; kb += kGramBK) {
    __syncthreads();  // the previous slab has been read
    for (int e = threadIdx.x; e < kGramBK * ncol; e += blockDim.x) {
      const int kk = e % kGramBK, c = e / kGramBK;
      const int64_t k = kb + kk;
      Ss[kk * lds + c] = (k < k1 && c < s) ? X[k + c * ldx] : 0.0f;
    }
    __syncthreads();
    if (active) {
#pragma unroll 2
      for (int kk = 0; kk < kGramBK; ++kk) {
        const float4 a4 = *reinterpret_cast<const float4*>(pa + kk * lds);
        const float4 b4 = *reinterpret_cast<const float4*>(pb + kk * lds);
        const float av[4] = {a4.x, a4.y, a4.z, a4.w};
        const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const float p = av[a] * bv[b];
            const float pe = fmaf(av[a], bv[b], -p);  // exact remainder
            float sum, e;
            two_sum(acc[a][b], p, sum, e);
            acc[a][b] = sum;
            comp[a][b] += e + pe;
          }
      }
    }
  }
  if (!active) return;
  double* P = part + static_cast<int64_t>(blockIdx.y) * s * s;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int m = 4 * bi + a, n = 4 * bj + b;
      if (m <= n && n < s)
        P[m + static_cast<int64_t>(n) * s] =
            static_cast<double>(acc[a][b]) + static_cast<double>(comp[a][b]);
    }
}

// threads per Gram CTA: the triangle rounded up to whole warps, <= 128
int gram_cta_threads(int s) {
  const int t = (gram_blocks(s) + 31) / 32 * 32;
  return t < kGramThreads ? t : kGramThreads;
}

// Expected time of gram_exact_kernel: every thread slot of the triangle's
// parts (idle ones included) forms 16 exact products per row, about
// 2.66e12 slot-products per second on the whole GPU (measured at n = 2^21,
// s = 16 .. 128, within 10 % but for s = 16).
double gram_exact_seconds(int64_t n, int s) {
  const int T = gram_cta_threads(s);
  const int parts = (gram_blocks(s) + T - 1) / T;
  return static_cast<double>(n) * parts * T * 16.0 / 2.66e12;
}

// floats per slab row of the Gram kernel: the columns padded to a multiple
// of 4, plus 4 (rows stay 16-byte aligned), one of three compiled strides
int gram_lds(int s) { return s <= 32 ? 36 : (s <= 64 ? 68 : kGramMaxS + 4); }

// splits of the Gram kernel: as many CTAs as fit on the SMs at 80
// registers a thread and one slab of shared memory each (at most 32 per
// SM), >= 4 slabs per split
int64_t gram_splits(int64_t n, int s, int64_t* rows) {
  const int T = gram_cta_threads(s);
  const int parts = (gram_blocks(s) + T - 1) / T;
  int per_sm = 65536 / (80 * T);
  const int by_smem = (227 * 1024) / (kGramBK * gram_lds(s) * 4 + 1024);
  if (per_sm > by_smem) per_sm = by_smem;
  if (per_sm > 32) per_sm = 32;   // resident CTAs per SM
  if (per_sm < 1) per_sm = 1;
  int64_t S = (per_sm * static_cast<int64_t>(device_sm_count()) + parts - 1) / parts;
  const int64_t maxS = (n + 4 * kGramBK - 1) / (4 * kGramBK);
  if (S > maxS) S = maxS;
  if (S < 1) S = 1;
  int64_t r = (n + S - 1) / S;
  r = (r + kGramBK - 1) / kGramBK * kGramBK;
  S = (n + r - 1) / r;
  if (rows) *rows = r;
  return S < 1 ? 1 : S;
}

enum Cfg { CFG_SQ = 0, CFG_NARROW_M = 1, CFG_NARROW_N = 2, CFG_SQ16 = 3 };

struct DotPlan {
  int cfg, BM, BN, tm, tn, S;
  int64_t rows;
};

// FP64 (wide = false): 16 x 16 tiles, one output per thread -- the FP64
// pipe, not shared memory, is the limit, and 16-wide tiles pad i and s
// less.  FP32: 32 x 32 tiles with 2 x 2 outputs per thread.
// The split count S fills one wave of resident CTAs (8 of 256 threads per
// SM) as evenly as it can: S = floor(slots / working tiles), so every SM
// runs floor or ceil of the average and the last SM to finish is at most
// one CTA behind (a rounding-up rule left up to a seventh of the SMs idle
// for the last CTA's duration).  sym: only the upper tiles work.
DotPlan plan_dot(int64_t n, int i, int s, bool wide, bool sym) {
  DotPlan p;
  if (i <= 8) { p.cfg = CFG_NARROW_M; p.BM = 8; p.BN = 32; }
  else if (s <= 8) { p.cfg = CFG_NARROW_N; p.BM = 64; p.BN = 8; }
  else if (!wide) { p.cfg = CFG_SQ16; p.BM = 16; p.BN = 16; }
  else { p.cfg = CFG_SQ; p.BM = 32; p.BN = 32; }
  p.tm = (i + p.BM - 1) / p.BM;
  p.tn = (s + p.BN - 1) / p.BN;
  const bool sym_tiles = sym && i == s && (p.cfg == CFG_SQ || p.cfg == CFG_SQ16);
  const int64_t tiles = sym_tiles ? static_cast<int64_t>(p.tm) * (p.tm + 1) / 2
                                  : static_cast<int64_t>(p.tm) * p.tn;
  const int64_t slots = static_cast<int64_t>(device_sm_count()) * (2048 / kThreads);
  int64_t S = slots / tiles;
  const int64_t maxS = (n + 4 * BK - 1) / (4 * BK);  // >= 4 stages per split
  if (S > maxS) S = maxS;
  if (S < 1) S = 1;
  if (S > 4096) S = 4096;
  int64_t rows = (n + S - 1) / S;
  rows = (rows + BK - 1) / BK * BK;
  S = (n + rows - 1) / rows;
  if (S < 1) S = 1;
  p.S = static_cast<int>(S);
  p.rows = rows;
  return p;
}

template <bool EXACT, typename T>
void launch_dot(const DotPlan& p, cudaStream_t st, int64_t n, int i, int s,
                const T* Q, int64_t ldq, const T* X, int64_t ldx, double* part,
                bool sym) {
  dim3 grid(p.tm, p.tn, p.S);
  const int sy = sym ? 1 : 0;
  switch (p.cfg) {
    case CFG_NARROW_M:
      dot_tile_kernel<8, 32, 1, 1, true, EXACT, T><<<grid, kThreads, 0, st>>>(
          n, i, s, Q, ldq, X, ldx, part, p.rows, 0);
      break;
    case CFG_NARROW_N:
      dot_tile_kernel<64, 8, 2, 1, false, EXACT, T><<<grid, kThreads, 0, st>>>(
          n, i, s, Q, ldq, X, ldx, part, p.rows, 0);
      break;
    case CFG_SQ16:
      dot_tile_kernel<16, 16, 1, 1, false, EXACT, T><<<grid, kThreads, 0, st>>>(
          n, i, s, Q, ldq, X, ldx, part, p.rows, sy);
      break;
    default:
      dot_tile_kernel<32, 32, 2, 2, false, EXACT, T><<<grid, kThreads, 0, st>>>(
          n, i, s, Q, ldq, X, ldx, part, p.rows, sy);
  }
  SG_LAUNCH_CHECK();
}

// -1: not yet read from the environment; else SG_TC_AUTO / NEVER / ALWAYS
std::atomic<int> g_tc_policy{-1};

int policy_now() {
  int v = g_tc_policy.load();
  if (v < 0) {
    const char* e = std::getenv("SGMRES_NO_TC");
    const int env = (e && e[0] == '1') ? SG_TC_NEVER : SG_TC_AUTO;
    g_tc_policy.compare_exchange_strong(v, env);
    v = g_tc_policy.load();
  }
  return v;
}

bool tc_disabled() { return policy_now() == SG_TC_NEVER; }
bool tc_forced() { return policy_now() == SG_TC_ALWAYS; }

template <typename T>
void block_dot_impl(int64_t n, const T* Q, int64_t ldq, int i, const T* X,
                    int64_t ldx, int s, double* W, int ldw, bool sym,
                    double* part, int64_t part_cap, cudaStream_t st) {
  if (i <= 0 || s <= 0) return;
  if (n <= 0) {
    for (int c = 0; c < s; ++c)
      SG_CUDA(cudaMemsetAsync(W + static_cast<int64_t>(c) * ldw, 0,
                              sizeof(double) * i, st));
    return;
  }
  if (sizeof(T) == 8 && !tc_disabled() &&
      oz_dot_supported(n, reinterpret_cast<const double*>(Q), ldq, i,
                       reinterpret_cast<const double*>(X), ldx, s) &&
      (tc_forced() || oz_dot_pays(n, i, s, sym && i == s))) {
    // FP64 products on the tensor cores, exact digit slices; the column
    // exponents sit after the split partials.  A Gram comes out exactly
    // symmetric (both triangles are the same exact sums).
    const int64_t need = oz_dot_part_size(n, i, s);
    SG_REQUIRE(need + (oz_exp_ints(i, s) + 1) / 2 <= part_cap, SG_EINVAL,
               "block_dot: workspace too small");
    int S = 0;
    oz_dot(n, reinterpret_cast<const double*>(Q), ldq, i, reinterpret_cast<const double*>(X),
           ldx, s, reinterpret_cast<int*>(part + need), part, need, &S, st);
    launch_reduce(i, s, S, part, W, ldw, false, st);
    return;
  }
  if (sizeof(T) == 8 && i + s <= kSmallCols &&
      (sym && i == s ? s * (s + 1) / 2 <= kSmallOut : (i > 8 && i * s <= kSmallOut))) {
    // small FP64 products: one thread per needed output (a Q of at most
    // eight columns keeps the narrow tile, whose idle rows are whole warps)
    const bool tri = sym && i == s;
    const int nout = tri ? s * (s + 1) / 2 : i * s;
    const int threads = (nout + 31) / 32 * 32;
    int64_t S = static_cast<int64_t>(device_sm_count()) * (2048 / threads);
    const int64_t maxS = (n + 4 * BK - 1) / (4 * BK);
    if (S > maxS) S = maxS;
    if (S < 1) S = 1;
    if (S * i * s > part_cap) S = part_cap / (static_cast<int64_t>(i) * s);
    SG_REQUIRE(S >= 1, SG_EINVAL, "block_dot: workspace too small");
    int64_t rows = (n + S - 1) / S;
    rows = (rows + BK - 1) / BK * BK;
    S = (n + rows - 1) / rows;
    const size_t smem = sizeof(double) * BK * (i + 1 + s + 1);
    dot_small_kernel<<<static_cast<unsigned>(S), threads, smem, st>>>(
        n, i, s, reinterpret_cast<const double*>(Q), ldq, reinterpret_cast<const double*>(X),
        ldx, part, rows, tri ? 1 : 0);
    SG_LAUNCH_CHECK();
    launch_reduce(i, s, static_cast<int>(S), part, W, ldw, tri, st);
    return;
  }
  if (sizeof(T) == 4 && !sym && !tc_disabled() &&
      tc_dot_supported(n, reinterpret_cast<const float*>(Q), ldq, i,
                       reinterpret_cast<const float*>(X), ldx, s)) {
    // projections of the FP32 basis on the tensor cores
    int S = 0;
    tc_dot(n, reinterpret_cast<const float*>(Q), ldq, i,
           reinterpret_cast<const float*>(X), ldx, s, part, part_cap, &S, st);
    launch_reduce(i, s, S, part, W, ldw, false, st);
    return;
  }
  if (sizeof(T) == 4 && sym && i == s && !tc_disabled() &&
      reinterpret_cast<const void*>(Q) == reinterpret_cast<const void*>(X) &&
      oz_gram32_supported(n, reinterpret_cast<const float*>(X), ldx, s) &&
      (tc_forced() || oz_gram32_seconds(n, s) < 0.9 * gram_exact_seconds(n, s))) {
    // Gram of FP32 vectors on the tensor cores from exact digit slices; the
    // column exponents sit after the split partials
    const int64_t need = oz_gram32_part_size(n, s);
    SG_REQUIRE(need + (s + 1) / 2 <= part_cap, SG_EINVAL, "block_dot: workspace too small");
    int S = 0;
    oz_gram32(n, reinterpret_cast<const float*>(X), ldx, s, reinterpret_cast<int*>(part + need),
              part, need, &S, st);
    launch_reduce(s, s, S, part, W, ldw, true, st);
    return;
  }
  if (sizeof(T) == 4 && sym && i == s && s <= kGramMaxS &&
      reinterpret_cast<const void*>(Q) == reinterpret_cast<const void*>(X)) {
    // Gram of FP32 vectors: exact products over the upper triangle
    int64_t rows = 0;
    const int64_t S = gram_splits(n, s, &rows);
    SG_REQUIRE(S * s * s <= part_cap, SG_EINVAL, "block_dot: workspace too small");
    const int nt = gram_cta_threads(s);
    const int parts = (gram_blocks(s) + nt - 1) / nt;
    const int lds = gram_lds(s);
    const dim3 grid(parts, static_cast<unsigned>(S));
    const size_t smem = sizeof(float) * kGramBK * lds;
    const float* Xf = reinterpret_cast<const float*>(X);
    if (lds == 36)
      gram_exact_kernel<36><<<grid, nt, smem, st>>>(n, s, Xf, ldx, part, rows);
    else if (lds == 68)
      gram_exact_kernel<68><<<grid, nt, smem, st>>>(n, s, Xf, ldx, part, rows);
    else
      gram_exact_kernel<kGramMaxS + 4><<<grid, nt, smem, st>>>(n, s, Xf, ldx, part, rows);
    SG_LAUNCH_CHECK();
    launch_reduce(s, s, static_cast<int>(S), part, W, ldw, true, st);
    return;
  }
  DotPlan p = plan_dot(n, i, s, sizeof(T) == 4, sym);
  const bool exact = sym && sizeof(T) == 4;   // Gram of FP32 vectors
  if (sym && ((p.cfg != CFG_SQ && p.cfg != CFG_SQ16) || i != s)) sym = false;
  SG_REQUIRE(static_cast<int64_t>(p.S) * i * s <= part_cap, SG_EINVAL,
             "block_dot: workspace too small");
  if (exact) launch_dot<true, float>(p, st, n, i, s, reinterpret_cast<const float*>(Q), ldq,
                                     reinterpret_cast<const float*>(X), ldx, part, sym);
  else launch_dot<false, T>(p, st, n, i, s, Q, ldq, X, ldx, part, sym);
  launch_reduce(i, s, p.S, part, W, ldw, sym, st);
}

// --------------------------------------------------------- block_update
// C(r0:r0+UR, n0:n0+UN) = beta C + alpha A(rows, :) B(:, cols); thread
// tile TR rows x TN cols; the inner dimension M (= i) is staged UK at a
// time.
constexpr int UK = 16;

// FP32 wide form: one CTA owns 64 rows x 128 columns (Q is read once for
// s <= 128), 4 x 8 outputs per thread, shared rows padded to 16-byte
// multiples and read as float4.
constexpr int WR = 64, WN = 128, WK = 16;

__global__ void __launch_bounds__(kThreads)
update_wide_kernel(int64_t K, int M, int N, const float* __restrict__ A, int64_t lda,
                   const double* __restrict__ B, int ldb, float* __restrict__ C,
                   int64_t ldc, float alpha, float beta, int upper) {
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * WR;
  const int n0 = blockIdx.y * WN;
  __shared__ __align__(16) float As[WK][WR + 4];
  __shared__ __align__(16) float Bs[WK][WN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16;  // rows tx*4 .. +3
  const int ty = tid / 16;  // cols ty*8 .. +7
  float acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
  const int mend = upper ? ((n0 + WN < M) ? n0 + WN : M) : M;
  for (int mb = 0; mb < mend; mb += WK) {
    for (int e = tid; e < WK * WR; e += kThreads) {
      const int rr = e % WR, mm = e / WR;
      const int64_t r = r0 + rr;
      const int m = mb + mm;
      As[mm][rr] = (r < K && m < mend) ? A[r + m * lda] : 0.0f;
    }
    for (int e = tid; e < WK * WN; e += kThreads) {
      const int mm = e % WK, nn = e / WK;
      const int m = mb + mm, nc = n0 + nn;
      float v = 0.0f;
      if (m < mend && nc < N && !(upper && m > nc)) v = static_cast<float>(B[m + nc * ldb]);
      Bs[mm][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int mm = 0; mm < WK; ++mm) {
      const float4 av = *reinterpret_cast<const float4*>(&As[mm][tx * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[mm][ty * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[mm][ty * 8 + 4]);
      const float a4[4] = {av.x, av.y, av.z, av.w};
      const float b8[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(a4[a], b8[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int nc = n0 + ty * 8 + b;
    if (nc >= N) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t r = r0 + tx * 4 + a;
      if (r >= K) continue;
      float* cp = C + r + nc * ldc;
      float v = alpha * acc[a][b];
      if (beta != 0.0f) v = fmaf(beta, *cp, v);
      *cp = v;
    }
  }
}

template <int UR, int UN, int TR, int TN, typename T>
__global__ void __launch_bounds__(kThreads)
update_kernel(int64_t K, int M, int N, const T* __restrict__ A, int64_t lda,
              const double* __restrict__ B, int ldb, T* __restrict__ C,
              int64_t ldc, double alpha, double beta, int upper) {
  constexpr int TRN = UR / TR, TNN = UN / TN;
  static_assert(TRN * TNN == kThreads, "thread layout");
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * UR;
  const int n0 = blockIdx.y * UN;
  __shared__ T As[UK][UR + 2];
  __shared__ T Bs[UK][UN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % TRN, ty = tid / TRN;
  T acc[TR][TN];
#pragma unroll
  for (int a = 0; a < TR; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = T(0);
  const int mend = upper ? ((n0 + UN < M) ? n0 + UN : M) : M;
  for (int mb = 0; mb < mend; mb += UK) {
    for (int e = tid; e < UK * UR; e += kThreads) {
      const int rr = e % UR, mm = e / UR;
      const int64_t r = r0 + rr;
      const int m = mb + mm;
      As[mm][rr] = (r < K && m < mend) ? A[r + m * lda] : T(0);
    }
    for (int e = tid; e < UK * UN; e += kThreads) {
      const int mm = e % UK, nn = e / UK;
      const int m = mb + mm, nc = n0 + nn;
      T v = T(0);
      if (m < mend && nc < N && !(upper && m > nc)) v = static_cast<T>(B[m + nc * ldb]);
      Bs[mm][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int mm = 0; mm < UK; ++mm) {
      T av[TR], bv[TN];
#pragma unroll
      for (int a = 0; a < TR; ++a) av[a] = As[mm][tx * TR + a];
#pragma unroll
      for (int b = 0; b < TN; ++b) bv[b] = Bs[mm][ty * TN + b];
#pragma unroll
      for (int a = 0; a < TR; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < TN; ++b) {
    const int nc = n0 + ty * TN + b;
    if (nc >= N) continue;
#pragma unroll
    for (int a = 0; a < TR; ++a) {
      const int64_t r = r0 + tx * TR + a;
      if (r >= K) continue;
      T* cp = C + r + nc * ldc;
      T v = static_cast<T>(alpha) * acc[a][b];
      if (beta != 0.0) v = fma(static_cast<T>(beta), *cp, v);
      *cp = v;
    }
  }
}

// X = beta X + alpha Q W for a narrow Q (i <= MAXI): the tiled kernel
// above pads the inner dimension to UK, which for i = 1 would cost UK FMAs
// per output, and this product is bound by streaming X.  One row per
// thread: its i values of Q in registers, W's column chunk (zero below the
// diagonal for the triangular form) in shared memory, X read and written
// a column at a time (coalesced along rows), eight columns per pass so that
// their loads are in flight together.  FP64 operations per output are the
// limit next to the stream, so the two forms the solver uses get their own
// chains: MODE 1 (alpha = -1, beta = 1, the BCGS update) subtracts the
// products from X one FMA at a time, k in order; MODE 2 (beta = 0, the
// triangular products) forms the sum in k order and scales it unless
// alpha = 1; MODE 0 forms the sum and applies alpha and beta.
constexpr int kThinCols = 64;
constexpr int kThinPass = 8;

template <int MAXI, int MODE, typename T>
__global__ void __launch_bounds__(kThreads)
update_thin_kernel(int64_t n, int i, int s, const T* __restrict__ Q, int64_t ldq,
                   const double* __restrict__ W, int ldw, T* __restrict__ X, int64_t ldx,
                   double alpha, double beta, int upper) {
  __shared__ T Ws[MAXI][kThinCols];
  const int c0 = blockIdx.y * kThinCols;
  const int cn = (s - c0 < kThinCols) ? s - c0 : kThinCols;
  for (int e = threadIdx.x; e < MAXI * kThinCols; e += kThreads) {
    const int k = e / kThinCols, c = e % kThinCols;
    T v = T(0);
    if (k < i && c < cn && !(upper && k > c0 + c))
      v = static_cast<T>(W[k + static_cast<int64_t>(c0 + c) * ldw]);
    Ws[k][c] = v;
  }
  __syncthreads();
  const T a = static_cast<T>(alpha), b = static_cast<T>(beta);
  // the triangular form needs k <= c only; the bound is the same for a
  // whole warp, and the loops leave at it (predicated FP64 instructions
  // would still take their pipe time)
  auto kend = [&](int c) { return upper ? (c0 + c + 1 < i ? c0 + c + 1 : i) : i; };
  auto out = [&](const T* q, int c, T x) -> T {
    const int ke = kend(c);
    if (MODE == 1) {
      T v = x;
#pragma unroll
      for (int k = 0; k < MAXI; ++k) {
        if (k >= ke) break;
        v = fma(-q[k], Ws[k][c], v);
      }
      return v;
    }
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < MAXI; ++k) {
      if (k >= ke) break;
      acc = (k == 0) ? q[0] * Ws[0][c] : fma(q[k], Ws[k][c], acc);
    }
    if (MODE == 2) return alpha == 1.0 ? acc : a * acc;
    const T v = a * acc;
    return beta != 0.0 ? fma(b, x, v) : v;
  };
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; r < n;
       r += static_cast<int64_t>(gridDim.x) * kThreads) {
    T q[MAXI];
#pragma unroll
    for (int k = 0; k < MAXI; ++k) q[k] = k < i ? Q[r + k * ldq] : T(0);
    T* xr = X + r + static_cast<int64_t>(c0) * ldx;
    int c = 0;
    for (; c + kThinPass <= cn; c += kThinPass) {
      T xv[kThinPass];
#pragma unroll
      for (int u = 0; u < kThinPass; ++u)
        xv[u] = (MODE != 2 && beta != 0.0) ? xr[static_cast<int64_t>(c + u) * ldx] : T(0);
#pragma unroll
      for (int u = 0; u < kThinPass; ++u)
        xr[static_cast<int64_t>(c + u) * ldx] = out(q, c + u, xv[u]);
    }
    for (; c < cn; ++c) {
      const T x = (MODE != 2 && beta != 0.0) ? xr[static_cast<int64_t>(c) * ldx] : T(0);
      xr[static_cast<int64_t>(c) * ldx] = out(q, c, x);
    }
  }
}

template <int MAXI, typename T>
void launch_update_thin_i(dim3 grid, int64_t n, const T* Q, int64_t ldq, int i, const double* W,
                          int ldw, T* X, int64_t ldx, int s, double alpha, double beta, int up,
                          cudaStream_t st) {
  if (alpha == -1.0 && beta == 1.0)
    update_thin_kernel<MAXI, 1, T><<<grid, kThreads, 0, st>>>(n, i, s, Q, ldq, W, ldw, X, ldx,
                                                               alpha, beta, up);
  else if (beta == 0.0)
    update_thin_kernel<MAXI, 2, T><<<grid, kThreads, 0, st>>>(n, i, s, Q, ldq, W, ldw, X, ldx,
                                                               alpha, beta, up);
  else
    update_thin_kernel<MAXI, 0, T><<<grid, kThreads, 0, st>>>(n, i, s, Q, ldq, W, ldw, X, ldx,
                                                               alpha, beta, up);
}

template <typename T>
void launch_update_thin(int64_t n, const T* Q, int64_t ldq, int i, const double* W, int ldw,
                        T* X, int64_t ldx, int s, double alpha, double beta, bool upper,
                        cudaStream_t st) {
  const int cchunks = (s + kThinCols - 1) / kThinCols;
  int64_t rb = (n + kThreads - 1) / kThreads;
  const int64_t cap = static_cast<int64_t>(device_sm_count()) * 8 / cchunks + 1;
  if (rb > cap) rb = cap;
  dim3 grid(static_cast<unsigned>(rb), static_cast<unsigned>(cchunks));
  const int up = upper ? 1 : 0;
  if (i <= 4)
    launch_update_thin_i<4, T>(grid, n, Q, ldq, i, W, ldw, X, ldx, s, alpha, beta, up, st);
  else if (i <= 8)
    launch_update_thin_i<8, T>(grid, n, Q, ldq, i, W, ldw, X, ldx, s, alpha, beta, up, st);
  else if (i <= 12)
    launch_update_thin_i<12, T>(grid, n, Q, ldq, i, W, ldw, X, ldx, s, alpha, beta, up, st);
  else
    launch_update_thin_i<16, T>(grid, n, Q, ldq, i, W, ldw, X, ldx, s, alpha, beta, up, st);
  SG_LAUNCH_CHECK();
}

template <typename T>
void block_update_impl(int64_t n, const T* Q, int64_t ldq, int i,
                       const double* W, int ldw, T* X, int64_t ldx, int s,
                       double alpha, double beta, bool upper,
                       cudaStream_t st) {
  if (n <= 0 || s <= 0) return;
  if (i <= 0) {
    if (beta == 1.0) return;
    alpha = 0.0;  // X = beta X
  }
  const int ii = i > 0 ? i : 0;
  if (sizeof(T) == 8 && ii <= 16) {
    launch_update_thin<T>(n, Q, ldq, ii, W, ldw, X, ldx, s, alpha, beta, upper, st);
    return;
  }
  if (s <= 8) {
    dim3 grid(static_cast<unsigned>((n + 127) / 128), 1);
    update_kernel<128, 8, 4, 1, T><<<grid, kThreads, 0, st>>>(
        n, ii, s, Q, ldq, W, ldw, X, ldx, alpha, beta, upper ? 1 : 0);
  } else if (sizeof(T) == 8) {
    dim3 grid(static_cast<unsigned>((n + 63) / 64), (s + 15) / 16);
    update_kernel<64, 16, 4, 1, T><<<grid, kThreads, 0, st>>>(
        n, ii, s, Q, ldq, W, ldw, X, ldx, alpha, beta, upper ? 1 : 0);
  } else if (s <= 32) {
    // FP32, narrow blocks: 128 x 32 tiles, 4 x 4 outputs per thread
    dim3 grid(static_cast<unsigned>((n + 127) / 128), 1);
    update_kernel<128, 32, 4, 4, T><<<grid, kThreads, 0, st>>>(
        n, ii, s, Q, ldq, W, ldw, X, ldx, alpha, beta, upper ? 1 : 0);
  } else {
    dim3 grid(static_cast<unsigned>((n + WR - 1) / WR), (s + WN - 1) / WN);
    update_wide_kernel<<<grid, kThreads, 0, st>>>(
        n, ii, s, reinterpret_cast<const float*>(Q), ldq, W, ldw,
        reinterpret_cast<float*>(X), ldx, static_cast<float>(alpha),
        static_cast<float>(beta), upper ? 1 : 0);
  }
  SG_LAUNCH_CHECK();
}

}  // namespace

int tc_policy() { return policy_now(); }

int set_tc_policy(int policy) {
  if (policy != SG_TC_AUTO && policy != SG_TC_NEVER && policy != SG_TC_ALWAYS) return -1;
  const int old = policy_now();
  g_tc_policy.store(policy);
  return old;
}

void block_dot_capped(int64_t n, const double* Q, int64_t ldq, int i,
                      const double* X, int64_t ldx, int s, double* W, int ldw,
                      double* part, int64_t part_cap, cudaStream_t st) {
  // same kernels as block_dot, with the number of splits reduced so that
  // the split partials fit in `part_cap` doubles
  if (i <= 0 || s <= 0) return;
  SG_REQUIRE(static_cast<int64_t>(i) * s <= part_cap, SG_EINVAL,
             "block_dot_capped: i*s exceeds the scratch");
  if (n <= 0) {
    for (int c = 0; c < s; ++c)
      SG_CUDA(cudaMemsetAsync(W + static_cast<int64_t>(c) * ldw, 0,
                              sizeof(double) * i, st));
    return;
  }
  DotPlan p = plan_dot(n, i, s, false, false);
  const int64_t maxS = part_cap / (static_cast<int64_t>(i) * s);
  if (p.S > maxS) {
    int64_t rows = (n + maxS - 1) / maxS;
    rows = (rows + BK - 1) / BK * BK;
    p.rows = rows;
    p.S = static_cast<int>((n + rows - 1) / rows);
  }
  launch_dot<false, double>(p, st, n, i, s, Q, ldq, X, ldx, part, false);
  launch_reduce(i, s, p.S, part, W, ldw, false, st);
}

int64_t block_dot_part_size(int64_t n, int i, int s) {
  int64_t S = 1;
  for (int w = 0; w < 2; ++w)
    for (int y = 0; y < 2; ++y) {
      const DotPlan a = plan_dot(n, i, s, w == 1, y == 1);
      if (a.S > S) S = a.S;
    }
  int64_t need = S * i * s;
  if (i == s && s <= kGramMaxS) {
    int64_t g = gram_splits(n, s, nullptr) * s * s;
    const int64_t g32 = oz_gram32_part_size(n, s) + (s + 1) / 2;
    if (g32 > g) g = g32;
    if (g > need) need = g;
  }
  const int64_t tc = tc_dot_part_size(n, i, s);
  const int64_t oz = oz_dot_part_size(n, i, s) + (oz_exp_ints(i, s) + 1) / 2;
  need = need > tc ? need : tc;
  return need > oz ? need : oz;
}

void block_dot(int64_t n, const double* Q, int64_t ldq, int i,
               const double* X, int64_t ldx, int s, double* W, int ldw,
               bool sym, double* part, int64_t part_cap, cudaStream_t st) {
  block_dot_impl<double>(n, Q, ldq, i, X, ldx, s, W, ldw, sym, part, part_cap,
                         st);
}

void block_dot32(int64_t n, const float* Q, int64_t ldq, int i,
                 const float* X, int64_t ldx, int s, double* W, int ldw,
                 bool sym, double* part, int64_t part_cap, cudaStream_t st) {
  block_dot_impl<float>(n, Q, ldq, i, X, ldx, s, W, ldw, sym, part, part_cap,
                        st);
}

int64_t block_update_scratch(int i) { return (static_cast<int64_t>(i) + 1) / 2 + 1; }

void block_update(int64_t n, const double* Q, int64_t ldq, int i,
                  const double* W, int ldw, double* X, int64_t ldx, int s,
                  double alpha, double beta, bool upper, double* scratch,
                  int64_t scratch_doubles, cudaStream_t st) {
  if (n > 0 && i > 0 && s > 0 && scratch && scratch_doubles >= block_update_scratch(i) &&
      !tc_disabled() && oz_update_supported(n, Q, ldq, i, X, ldx, s) &&
      (tc_forced() || oz_update_pays(n, i, s, upper))) {
    // FP64 products on the tensor cores, exact digit slices
    oz_update(n, Q, ldq, i, W, ldw, X, ldx, s, alpha, beta, upper,
              reinterpret_cast<int*>(scratch), st);
    return;
  }
  block_update_impl<double>(n, Q, ldq, i, W, ldw, X, ldx, s, alpha, beta,
                            upper, st);
}

void block_update32(int64_t n, const float* Q, int64_t ldq, int i,
                    const double* W, int ldw, float* X, int64_t ldx, int s,
                    double alpha, double beta, bool upper, double* scratch,
                    int64_t scratch_doubles, cudaStream_t st) {
  if (i > 0 && s > 0 && scratch && !tc_disabled() &&
      tc_update_scratch(i, s) <= 2 * scratch_doubles &&
      tc_update_supported(n, Q, ldq, i, X, ldx, s)) {
    tc_update(n, Q, ldq, i, W, ldw, X, ldx, s, alpha, beta, upper,
              reinterpret_cast<float*>(scratch), 2 * scratch_doubles, st);
    return;
  }
  block_update_impl<float>(n, Q, ldq, i, W, ldw, X, ldx, s, alpha, beta,
                           upper, st);
}

}  // namespace sg
