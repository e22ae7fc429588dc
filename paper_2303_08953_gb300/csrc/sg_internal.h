// Internal declarations of the sm_103a s-step GMRES library: device
// matrix, workspace, error handling and the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>

#include "sgmres.h"

namespace sg {

struct Error : std::runtime_error {
  sg_status code;
  Error(sg_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define SG_CUDA(call)                                                      \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess)                                                 \
      throw ::sg::Error(SG_ECUDA, std::string(#call) + ": " +              \
                                      cudaGetErrorString(e_));             \
  } while (0)
// every kernel launch of the library goes through this check, which also
// counts it (sg_kernel_launches)
void count_launch();
void count_launches(long long k);
#define SG_LAUNCH_CHECK()                                                  \
  do {                                                                     \
    ::sg::count_launch();                                                  \
    SG_CUDA(cudaGetLastError());                                           \
  } while (0)
#define SG_REQUIRE(cond, code, msg)                                        \
  do {                                                                     \
    if (!(cond)) throw ::sg::Error(code, msg);                             \
  } while (0)

// CSR on the device (int32 indices, FP64 values, optional FP32 copy).
struct DevCsr {
  int32_t n = 0;
  int64_t nnz = 0;
  int32_t* rowptr = nullptr;
  int32_t* colind = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;
  double mean_row = 0;  // row-length statistics recorded at ingest
  int32_t max_row = 0;
  // SELL-32 copy (sliced ELLPACK, slices of 32 rows stored column-major,
  // padding marked by column -1), built at ingest when the padding is
  // small; null otherwise, and the SpMV then reads the CSR arrays.
  int32_t nslices = 0;
  int64_t sell_nnz = 0;
  int32_t* sptr = nullptr;  // nslices + 1 entry offsets
  int32_t* scol = nullptr;
  double* sval = nullptr;
  float* sval32 = nullptr;
  // The same columns as 16-bit offsets from each slice's smallest column
  // (0xFFFF marks padding), built when every slice spans fewer than 65535
  // columns: the SpMV then streams 10 bytes per stored entry instead of 12.
  int32_t* sbase = nullptr;  // nslices
  uint16_t* soff = nullptr;
};

// Build A's SELL-32 copy from its CSR arrays (kept when the padded size is
// at most 1.2 nnz + 32 per slice and fits int32 offsets); frees any old one.
void build_sell(DevCsr& A, cudaStream_t st);
// Copy A.val into the SELL value array after a value update.
void sell_refill_values(const DevCsr& A, cudaStream_t st);

// Column equilibration (Eq. equil): d[j] = 1 / ||A(:, j)||_2 from the rows
// of AT (1 for an empty column), summed in row order (deterministic).
void column_scale_factors(const DevCsr& AT, double* d, cudaStream_t st);
// E.val = A.val * d[col] (and the SELL values when A has them; E shares
// A's pattern arrays, its value arrays are allocated by the caller).
void scale_columns(const DevCsr& A, const double* d, DevCsr& E, cudaStream_t st);
// Failure-detection probes: a grid barrier / an mbarrier that cannot
// complete, waited on with the given limit; true when the kernel's bounded
// wait ran out and set its error flag.
bool probe_grid_barrier_timeout(uint64_t limit_ns, cudaStream_t st);
bool probe_mbarrier_timeout(uint64_t limit_ns, cudaStream_t st);
// y[i] = x[i] * d[i] (mul) or x[i] / d[i] (div), in place allowed.
void diag_apply(int64_t n, const double* d, const double* x, double* y, bool div,
                cudaStream_t st);

// ---------------------------------------------------------------- SpMV
// y = (A x - theta x + c z) / gamma      (z may be null when c == 0)
void spmv_newton(const DevCsr& A, const double* x, const double* z,
                 double* y, double theta, double c, double gamma,
                 cudaStream_t st);
void spmv_newton32(const DevCsr& A, const float* x, const float* z, float* y,
                   float theta, float c, float gamma, cudaStream_t st);
// One Arnoldi step of the Ritz pre-pass (cooperative launch): V[:, j+1] =
// normalised MGS projection of A V[:, j]; writes H(0..j+1, j) (ld ldh) and
// wn[j] = ||A v_j||.  red: >= 3 x SMs doubles (FP64); bar: 64 zeroed unsigned
// words (barrier state); err: set to 1 if a barrier wait ran out.
void arnoldi_step(const DevCsr& A, double* V, int64_t ld, int j, double* H,
                  int ldh, double* wn, double* red, int red_cap, unsigned* bar,
                  int* err, cudaStream_t st);
// FP32 form: while j + 1 <= 161 and red holds prepass_red_doubles() the
// step takes two grid barriers (the MGS coefficients from the basis's Gram
// matrix, whose rows it keeps in red across the steps of one pre-pass, so
// the steps 0..k-1 of a pre-pass run in order on one red buffer).
void arnoldi_step32(const DevCsr& A, float* V, int64_t ld, int j, double* H,
                    int ldh, double* wn, double* red, int red_cap, unsigned* bar,
                    int* err, cudaStream_t st);
int64_t prepass_red_doubles();
// r = b - A x
void residual(const DevCsr& A, const double* b, const double* x, double* r,
              cudaStream_t st);
// dval[k] = -lam[row(k)] * x[col(k)]
void sampled_outer(const DevCsr& A, const double* lam, const double* x,
                   double* dval, cudaStream_t st);
// CSR transpose (device to device), sorted columns.
void csr_transpose(const DevCsr& A, DevCsr& T, int32_t* work_counts,
                   cudaStream_t st);

// ------------------------------------------------------- vector kernels
// Deterministic two-stage reductions: stage 1 writes `nred` per-block
// partial sums, consumers add them in a fixed order.
int reduction_blocks();
void dot_partials(int64_t n, const double* x, const double* y,
                  double* partials, cudaStream_t st);
// out[0] = sum(partials) (or its square root when sqrt_out)
void finish_sum(const double* partials, double* out, bool sqrt_out,
                cudaStream_t st);
// y = x * (alpha_host)
void scale_copy(int64_t n, const double* x, double* y, double alpha,
                cudaStream_t st);
// x += Q(:, 0:k-1) y   (y: device, length k)
void gemv_n_add(int64_t n, int k, const double* Q, int64_t ldq,
                const double* y, double* x, cudaStream_t st);
void gemv_n_add32(int64_t n, int k, const float* Q, int64_t ldq,
                  const double* y, double* x, cudaStream_t st);
// precision conversions
void to_f32(int64_t n, const double* x, float* y, float scale,
            cudaStream_t st);
void axpy_f32_to_f64(int64_t n, double alpha, const float* d, double* x,
                     cudaStream_t st);
void fill_zero(int64_t n, double* x, cudaStream_t st);

// ------------------------------------------------------ dense kernels
// W = Q^T X through split-n partials (workspace `part`, `part_cap`
// doubles); sym: Q == X, only the upper tile triangle is computed.
void block_dot(int64_t n, const double* Q, int64_t ldq, int i,
               const double* X, int64_t ldx, int s, double* W, int ldw,
               bool sym, double* part, int64_t part_cap, cudaStream_t st);
void block_dot32(int64_t n, const float* Q, int64_t ldq, int i,
                 const float* X, int64_t ldx, int s, double* W, int ldw,
                 bool sym, double* part, int64_t part_cap, cudaStream_t st);
int64_t block_dot_part_size(int64_t n, int i, int s);
// block_dot without the symmetric option, splitting n into as many parts
// as fit in part_cap doubles (which must hold at least i*s)
void block_dot_capped(int64_t n, const double* Q, int64_t ldq, int i,
                      const double* X, int64_t ldx, int s, double* W, int ldw,
                      double* part, int64_t part_cap, cudaStream_t st);
// X = beta X + alpha Q W (W on the device, i x s, upper-triangular if
// `upper`, i == s)
// (on the tensor cores when it pays; scratch: >= block_update_scratch(i)
// doubles for Q's column exponents, may be null to force the FP64 pipe)
void block_update(int64_t n, const double* Q, int64_t ldq, int i,
                  const double* W, int ldw, double* X, int64_t ldx, int s,
                  double alpha, double beta, bool upper, double* scratch,
                  int64_t scratch_doubles, cudaStream_t st);
int64_t block_update_scratch(int i);

// process-wide tensor-core policy of the FP64 block products (SG_TC_*);
// set_tc_policy returns the previous one, or -1 for an unknown value
int tc_policy();
int set_tc_policy(int policy);
// FP32: runs on the tensor cores when supported (scratch: >= the
// tc_update_scratch floats, may be null to force the FFMA kernels)
void block_update32(int64_t n, const float* Q, int64_t ldq, int i,
                    const double* W, int ldw, float* X, int64_t ldx, int s,
                    double alpha, double beta, bool upper, double* scratch,
                    int64_t scratch_doubles, cudaStream_t st);

// Tensor-core (tcgen05, TMA) FP32 block dot W = Q^T X: split partials
// into `part`, number of splits in *nsplit; bounded waits record failure
// in a device flag that tc_check_error reads (and clears, then throws).
bool tc_dot_supported(int64_t n, const float* Q, int64_t ldq, int i,
                      const float* X, int64_t ldx, int s);
int64_t tc_dot_part_size(int64_t n, int i, int s);
void tc_dot(int64_t n, const float* Q, int64_t ldq, int i, const float* X,
            int64_t ldx, int s, double* part, int64_t part_cap, int* nsplit,
            cudaStream_t st);
void tc_check_error(cudaStream_t st);
// Tensor-core (tcgen05, TMA) FP64 block dot W = Q^T X from exact 8-bit
// digit slices of both operands: split partials into `part` (part_cap
// doubles), column exponents into `exps` (oz_exp_ints(i, s) ints), number of
// splits in *nsplit; a bounded wait that ran out sets a device flag that
// oz_check_error reads (and clears, then throws).
bool oz_dot_supported(int64_t n, const double* Q, int64_t ldq, int i, const double* X,
                      int64_t ldx, int s);
int64_t oz_dot_part_size(int64_t n, int i, int s);
int64_t oz_exp_ints(int i, int s);
bool oz_dot_pays(int64_t n, int i, int s, bool sym);
// Tensor-core FP64 block update X = beta X + alpha Q W (W on the device, i x s,
// upper-triangular if `upper`), from the same digit slices; exps: i ints.
bool oz_update_supported(int64_t n, const double* Q, int64_t ldq, int i, const double* X,
                         int64_t ldx, int s);
bool oz_update_pays(int64_t n, int i, int s, bool upper);
void oz_update(int64_t n, const double* Q, int64_t ldq, int i, const double* W, int ldw,
               double* X, int64_t ldx, int s, double alpha, double beta, bool upper, int* exps,
               cudaStream_t st);
void oz_dot(int64_t n, const double* Q, int64_t ldq, int i, const double* X, int64_t ldx,
            int s, int* exps, double* part, int64_t part_cap, int* nsplit, cudaStream_t st);
void oz_check_error(cudaStream_t st);
// Tensor-core FP32 Gram G = X^T X (s <= 128 columns) from exact digit
// slices: split partials of the upper triangle (entry (m, n), m <= n, at
// m + n s) into `part`, column exponents into `exps` (s ints); a bounded
// wait that ran out sets the flag oz_check_error reads.
bool oz_gram32_supported(int64_t n, const float* X, int64_t ldx, int s);
double oz_gram32_seconds(int64_t n, int s);
int64_t oz_gram32_part_size(int64_t n, int s);
void oz_gram32(int64_t n, const float* X, int64_t ldx, int s, int* exps, double* part,
               int64_t part_cap, int* nsplit, cudaStream_t st);
// Tensor-core (tcgen05, TMA) FP32 block update X = beta X + alpha Q W.
bool tc_update_supported(int64_t n, const float* Q, int64_t ldq, int i,
                         const float* X, int64_t ldx, int s);
int64_t tc_update_scratch(int i, int s);  // floats
void tc_update(int64_t n, const float* Q, int64_t ldq, int i, const double* W,
               int ldw, float* X, int64_t ldx, int s, double alpha, double beta,
               bool upper, float* scratch, int64_t scratch_floats,
               cudaStream_t st);
void tc_update_check_error(cudaStream_t st);

// dst[k] = src[idx[k]], k < count (device arrays).
// Structure checks of a square CSR matrix on the device (synchronises):
// returns the OR of 1 (rowptr does not run from 0 to nnz), 2 (a row's
// bounds are decreasing or outside [0, nnz]), 4 (a column outside
// [0, ncols)), 8 (columns not increasing within a row); *longest = the
// longest row.
int check_csr(const int32_t* rowptr, const int32_t* colind, int64_t n, int64_t nnz,
              int64_t ncols, int* flags, int* longest, cudaStream_t st);
void gather(const int32_t* idx, int64_t count, const double* src, double* dst,
            cudaStream_t st);

int device_sm_count();  // of the current device
int current_device();
// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) for kernel fn on the
// current device, once per (kernel, device) and size
void ensure_dynamic_smem(const void* fn, int bytes);

}  // namespace sg
