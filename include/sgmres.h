/*
 * sgmres.h -- C ABI of a single-GPU (sm_103a) adaptive s-step GMRES
 * after Xu, Alonso and Darve, "A numerically stable communication-avoiding
 * s-step GMRES algorithm" (arXiv 2303.08953).
 *
 * Problem statement (Alg. 4, REQUIRE/ENSURE): given a square sparse A
 * (CSR), a right-hand side b, an initial guess x0, a restart length m, an
 * initial step size s0 (or the estimator of Sec. 3.5), a polynomial basis
 * (Sec. 3.4) and the condition bound Omega (Sec. 3.2), return x with
 * ||b - A x||_2 / ||b - A x0||_2 <= tol.
 *
 * Conventions shared by every call:
 *  - Every call returns an sg_status; no exception crosses the ABI.
 *    On failure sg_last_error(h) gives a one-line message.
 *  - Dense vectors are FP64 arrays of length n.  Dense matrices are
 *    column-major with an explicit leading dimension (in elements).
 *  - The caller owns every array it passes; the library copies what it
 *    keeps (the matrix, on sg_analyze) and owns its own device workspace,
 *    sized on first use and kept until sg_destroy.
 *  - "stream" arguments are cudaStream_t values passed as void*; NULL
 *    selects the handle's own stream.  Solver calls are stream-ordered and
 *    return only after their results are complete (the small dense algebra
 *    runs on the host between kernels, as in the paper).
 *  - Indices are int32 (CSR requires nnz < 2^31).
 */
#ifndef SGMRES_H
#define SGMRES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SG_OK = 0,
  SG_EINVAL = 1,    /* bad argument (null pointer, size, unsorted CSR ...) */
  SG_ENOMEM = 2,    /* device or pinned-host allocation failed            */
  SG_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed         */
  SG_ENOCONV = 4,   /* iteration cap reached; x and the result are filled */
  SG_ENUMERIC = 5,  /* NaN/Inf met in the data or the small algebra        */
  SG_ESTATE = 6     /* call order violated (e.g. solve before analyze)     */
} sg_status;

/* Polynomial basis of the matrix powers kernel (Sec. 2 and Sec. 3.4):
 * scaled Newton, Eq. (scalednewton) with gamma from Eq. (scalingcoeff);
 * Newton, Eq. (newton) (gamma = 1); monomial, Eq. (monomial). */
typedef enum {
  SG_BASIS_SCALED_NEWTON = 0,
  SG_BASIS_NEWTON = 1,
  SG_BASIS_MONOMIAL = 2
} sg_basis;

/* Arithmetic of the Krylov basis.  FP64: everything in FP64.  FP32_IR:
 * FP32 matrix powers and block orthogonalisation inside an FP64
 * iterative-refinement loop (residual, Cholesky factors, Hessenberg least
 * squares and the estimator stay FP64).  Not in the paper. */
typedef enum { SG_PREC_FP64 = 0, SG_PREC_FP32_IR = 1 } sg_precision;

/* Matrix equilibration A' = D_r A D_c (Eq. equil, Sec. 4.3).
 * SCALAR: A' = A / alpha, alpha = max |theta| over the pre-pass Ritz
 *   values; for the monomial and standard Newton bases this is the
 *   constant scaling coefficient gamma = alpha, and it leaves the scaled
 *   Newton basis unchanged (its gamma is relative).
 * COLUMN: D_r = I, D_c = diag(1 / ||A(:, j)||_2): the solver runs on
 *   A' y = b and returns x = D_c y (forward solves only; D_c is built from
 *   the transpose, deterministically, on first use).
 * Residuals and tol refer to the original system in both cases. */
typedef enum {
  SG_EQUIL_NONE = 0,
  SG_EQUIL_SCALAR = 1,
  SG_EQUIL_COLUMN = 2
} sg_equil;

typedef struct sg_handle sg_handle;

/* Square CSR matrix, 0-based, columns sorted within each row. */
typedef struct {
  int32_t n;               /* rows = columns, >= 1                       */
  int64_t nnz;             /* rowptr[n]; < 2^31                          */
  const int32_t* rowptr;   /* n+1                                        */
  const int32_t* colind;   /* nnz                                        */
  const double* val;       /* nnz                                        */
  int32_t on_device;       /* 1: the three arrays are device pointers    */
} sg_csr;

/* Inputs of Alg. 4. */
typedef struct {
  int32_t m;           /* restart length: Krylov columns per cycle (>= 1)  */
  int32_t s;           /* > 0: initial step size s0; 0: estimator (Sec 3.5) */
  int32_t s_min;       /* clamp of the estimated s0 (estimator only)       */
  int32_t s_max;       /* Ritz values computed = s_max when s == 0         */
  double tol;          /* target ||b-Ax||/||b-Ax0||                        */
  int32_t max_iters;   /* cap on Krylov columns over all cycles (0: 50 m) */
  double omega;        /* partial CholQR bound Omega (Sec. 3.2), 1e7       */
  double omega_est;    /* estimator threshold (Sec. 3.5), 1e7              */
  int32_t basis;       /* sg_basis                                         */
  int32_t precision;   /* sg_precision                                     */
  double inner_tol;    /* FP32_IR: relative tolerance of each inner solve  */
  int32_t max_refine;  /* FP32_IR: cap on refinement steps                 */
  int32_t vectors_on_device; /* 1: b/x/g/lam of sg_solve* are device ptrs */
  void* stream;        /* cudaStream_t or NULL                             */
  int32_t equilibrate; /* an sg_equil value; default NONE                   */
  /* n_ritz > 0: use these Ritz values (host arrays of n_ritz entries, every
   * complex value with its conjugate) instead of running the pre-pass: they
   * are Leja-ordered and used as the pre-pass's would be (Sec. 3.4), and
   * with s == 0 the estimator runs on them.  A later solve with the same
   * matrix, or the adjoint solve (A^T has A's eigenvalues), can reuse the
   * Ritz values a solve reported in sg_result. */
  int32_t n_ritz;
  const double* ritz_re;
  const double* ritz_im;
} sg_opts;

/* Outputs.  The array members are caller-owned buffers that may be NULL;
 * each is filled up to its capacity, and the n_* counters give the true
 * number of entries (which may exceed the capacity). */
typedef struct {
  int32_t converged;       /* 1 when the true relres <= tol                */
  int32_t s0;              /* initial step size used (given or estimated)  */
  int32_t iters;           /* Krylov columns over all cycles               */
  int32_t restarts;        /* cycles - 1                                   */
  int32_t refinements;     /* FP32_IR outer steps (0 for FP64)             */
  double final_relres;     /* true ||b - A x|| / ||b - A x0||              */
  /* per Krylov column: implicit relative residual |g_{j+1}| / beta0     */
  int32_t hist_cap; double* relres_hist; int32_t n_hist;
  /* per block: columns generated, kept by CholQR #1, kept by CholQR #2   */
  int32_t blocks_cap; int32_t* s_eff_hist; int32_t* p1_hist;
  int32_t* s_hist; int32_t n_blocks;
  /* per cycle: true relative residual and columns used                   */
  int32_t cycles_cap; double* cycle_relres; int32_t* cycle_iters;
  int32_t n_cycles;
  /* Leja-ordered Ritz values and the scaling coefficients gamma          */
  int32_t ritz_cap; double* ritz_re; double* ritz_im; double* gamma;
  int32_t n_ritz;
  /* time spent per phase (ms, host wall clock around stream syncs)       */
  double t_prepass_ms, t_mpk_ms, t_ortho_ms, t_host_ms, t_total_ms;
  /* FP32_IR: Krylov columns run with the FP64 basis after the refinement
   * stalled (two refinement steps that did not halve the true residual,
   * the sign that kappa(A) eps_32 is near 1); 0 when it never did.
   * Included in iters; not in the paper. */
  int32_t fp64_iters;
} sg_result;

/* ----------------------------------------------------------- lifecycle */
/* Fill *o with the defaults (m=60, s=10, Omega=Omega_est=1e7, tol=1e-10,
 * scaled Newton, FP64). */
void sg_default_opts(sg_opts* o);

/* Create a handle on CUDA device `device`.  Errors: SG_EINVAL (null out),
 * SG_ECUDA (no such device / no driver). */
sg_status sg_create(int device, sg_handle** out);

/* Release the handle and all device memory it owns. NULL is a no-op. */
void sg_destroy(sg_handle* h);

/* Last error message of this handle ("" if none).  Valid until the next
 * call on the handle. */
const char* sg_last_error(const sg_handle* h);

/* Ingest A (Sec. 2 input; CSR as in the paper's implementation): checks
 * sizes, sorted in-range columns and int32 range, copies A to the device
 * (FP64 values, plus FP32 values for SG_PREC_FP32_IR) and picks the SpMV
 * variant from the row-length statistics.  Replaces any previous matrix.
 * Errors: SG_EINVAL, SG_ENOMEM, SG_ECUDA. */
sg_status sg_analyze(sg_handle* h, const sg_csr* A);

/* Ingest one process's row block of a row-partitioned matrix (Sec. 5:
 * rows are distributed over the processes): A->n local rows whose columns
 * are local indices in [0, ncols), ncols >= n, as sg_host_halo_plan
 * numbers them (owned columns first, then the halo), distinct within a
 * row and kept in the given order.  Only the kernel-level calls run on
 * such a handle: sg_spmv_newton and sg_residual read x (and the shift term
 * x[row]) as the length-ncols vector [own entries; halo entries]; the
 * solve-level calls return SG_ESTATE.  Errors as sg_analyze. */
sg_status sg_analyze_rows(sg_handle* h, const sg_csr* A, int32_t ncols);

/* dst[k] = src[idx[k]] for k < count (device arrays, idx int32): packs the
 * entries a neighbouring process needs from this one before a halo
 * exchange.  Runs on `stream`.  Errors: SG_EINVAL, SG_ECUDA. */
sg_status sg_gather(const int32_t* idx, int64_t count, const double* src, double* dst,
                    void* stream);

/* Replace the values of the analysed matrix, keeping its pattern: val
 * has nnz entries (device pointer when on_device, else host).  The FP32
 * copy is refreshed and the transpose is rebuilt on the next adjoint
 * call.  Errors: SG_ESTATE (no matrix), SG_EINVAL, SG_ECUDA. */
sg_status sg_update_values(sg_handle* h, const double* val,
                           int32_t on_device);

/* Storage the SpMV kernels use for the analysed matrix: *sell = 1 when
 * the SELL-32 copy (slices of 32 rows, column-major within a slice) was
 * built at ingest, 0 when the CSR arrays are walked directly (the padding
 * to each slice's longest row would exceed 20% of nnz); *stored = the
 * entries the SpMV reads per product (padded count for SELL-32, nnz for
 * CSR).  Either pointer may be NULL.  Not in the paper: a layout report.
 * Errors: SG_EINVAL (NULL handle), SG_ESTATE (no matrix). */
sg_status sg_matrix_info(const sg_handle* h, int32_t* sell, int64_t* stored);

/* ------------------------------------------------------------- solvers */
/* Adaptive s-step GMRES(m) (Alg. 4 with restarts): solves A x = b.
 * x holds x0 on entry and the solution on exit.  res may be NULL.
 * Returns SG_OK when converged, SG_ENOCONV when max_iters was reached
 * (x and res are still filled), SG_ENUMERIC on NaN/Inf. */
sg_status sg_solve(sg_handle* h, const double* b, double* x,
                   const sg_opts* opts, sg_result* res);

/* Adjoint solve A^T lam = g with the same method on the transposed CSR,
 * built on first use (not in the paper; gradient of a loss through
 * x = A^-1 b).  lam holds the initial guess on entry. */
sg_status sg_solve_adjoint(sg_handle* h, const double* g, double* lam,
                           const sg_opts* opts, sg_result* res);

/* Sampled outer product on A's pattern: dval[k] = -lam[row(k)] * x[col(k)]
 * for every stored entry k, i.e. dL/dA_ij when x = A^-1 b and
 * lam = A^-T dL/dx.  All three are device arrays (dval has nnz entries).
 * Not in the paper. */
sg_status sg_grad_values(sg_handle* h, const double* lam, const double* x,
                         double* dval, void* stream);

/* -------------------------------------------------- kernel-level calls
 * Device-pointer entry points of the individual steps, with the layouts
 * the solver uses.  They run on `stream` and return after enqueueing
 * (no synchronisation) unless stated. */

/* One Newton step of the matrix powers kernel (Eq. newtonrecurrence,
 * plus the conjugate-pair form): y = (A x - theta x + c z) / gamma.
 * z may be NULL when c == 0.  x, y, z: length-n device vectors; y must not
 * alias x or z. */
sg_status sg_spmv_newton(sg_handle* h, const double* x, const double* z,
                         double* y, double theta, double c, double gamma,
                         void* stream);

/* r = b - A x (Alg. 4, first line). */
sg_status sg_residual(sg_handle* h, const double* b, const double* x,
                      double* r, void* stream);

/* Matrix powers kernel (Sec. 2): V[:,0] = q, then s steps of the basis
 * given by theta (Leja-ordered shifts; a conjugate pair appears as
 * (a+ib, a-ib) in consecutive entries) and gamma.  V is n x (s+1),
 * column-major with leading dimension ldv >= n. */
sg_status sg_mpk(sg_handle* h, const double* q, double* V, int64_t ldv,
                 int32_t s, const double* theta_re, const double* theta_im,
                 const double* gamma, void* stream);

/* Ritz pre-pass alone (Sec. 3.4: Ritz values from k steps of Arnoldi):
 * k steps of modified Gram-Schmidt Arnoldi with the analysed matrix from
 * the unit vector q (device, n doubles), in the handle's workspace, one
 * cooperative kernel per step (the launches of a k are captured once in a
 * CUDA graph and replayed).  precision: SG_PREC_FP64, or SG_PREC_FP32_IR
 * for the FP32 basis (q rounded to FP32).  H (host, ldh >= k+1, k columns,
 * column-major) receives the (k+1) x k Hessenberg matrix, *steps the steps
 * completed (fewer than k after an invariant subspace: h_{j+1,j} <= 1e-12
 * of ||A v_j||).  Synchronises `stream`.  Errors: SG_EINVAL (k < 1, null
 * pointers, ldh), SG_ESTATE (no matrix), SG_ECUDA (a barrier wait ran
 * out). */
sg_status sg_arnoldi(sg_handle* h, const double* q, int32_t k, int32_t precision,
                     double* H, int32_t ldh, int32_t* steps, void* stream);

/* Block dot product of BCGS (Alg. 4 'First BCGS'): W = Q^T X, with Q
 * n x i (ldq), X n x s (ldx) and W i x s (ldw), all device memory.
 * Deterministic split-n reduction through the handle's workspace.
 * sym != 0 requires Q == X and fills W from its upper triangle. */
sg_status sg_block_dot(sg_handle* h, int64_t n, const double* Q, int64_t ldq,
                       int32_t i, const double* X, int64_t ldx, int32_t s,
                       double* W, int32_t ldw, int32_t sym, void* stream);

/* Block update of BCGS (Alg. 4): X <- beta X + alpha Q W, Q n x i,
 * W i x s (device), X n x s.  X must not alias Q.  With upper != 0, W is
 * upper triangular (i == s) and only its upper triangle is read: this is
 * the triangular product Q_k = V Z^-1 of CholQR with W = Z^-1. */
sg_status sg_block_update(sg_handle* h, int64_t n, const double* Q,
                          int64_t ldq, int32_t i, const double* W,
                          int32_t ldw, double* X, int64_t ldx, int32_t s,
                          double alpha, double beta, int32_t upper,
                          void* stream);

/* FP32 forms of the two block kernels, as used by the FP32 basis of
 * SG_PREC_FP32_IR: Q and X are FP32 (column-major), W is FP64.  With sym,
 * sg_block_dot_f32 forms the Gram matrix X^T X (the CholQR Gram of Alg. 4)
 * without rounding its products in FP32: for s <= 128, n >= 256, X 16-byte
 * aligned and ldx a multiple of 4, on the tensor cores when a cost model
 * says so, from six 8-bit digit slices of each value relative to its
 * column's largest magnitude (every value within 2^23 of it exact; entry
 * (a, b) within 2^-46 (max|x_a| sum|x_b| + max|x_b| sum|x_a|)
 * + n 2^-58 max|x_a| max|x_b| of the exact Gram, plus one rounding); else
 * from exact FP32 products accumulated with compensated sums (accurate to
 * ~eps_32^2 relative to sum |x_k y_k|).  An Inf or a NaN in a column makes
 * that column's row and column of the Gram non-finite (NaN on the tensor
 * cores).  Otherwise, when the
 * leading dimensions are multiples of
 * 4, the pointers 16-byte aligned, n >= 512 and s <= 128, it runs on the
 * tensor cores (TMA + tcgen05, TF32 hi/lo split: hi*hi + lo*hi + hi*lo,
 * FP32 accumulation, Q's split parts in tensor memory), else in FP32 FFMA.
 * sg_block_update_f32 likewise runs on the tensor cores when Q is 16-byte
 * aligned with a leading dimension that is a multiple of 4, n >= 128 and
 * s <= 128 (the Q tile's split parts in tensor memory, W split into TF32
 * hi + FP32 remainder in shared memory).  Both calls
 * synchronise the stream before returning (a tensor-core wait timeout is
 * reported as SG_ECUDA). */
sg_status sg_block_dot_f32(sg_handle* h, int64_t n, const float* Q,
                           int64_t ldq, int32_t i, const float* X,
                           int64_t ldx, int32_t s, double* W, int32_t ldw,
                           int32_t sym, void* stream);
sg_status sg_block_update_f32(sg_handle* h, int64_t n, const float* Q,
                              int64_t ldq, int32_t i, const double* W,
                              int32_t ldw, float* X, int64_t ldx, int32_t s,
                              double alpha, double beta, int32_t upper,
                              void* stream);

/* Two-norm of a device vector, returned on the host (synchronises). */
sg_status sg_nrm2(sg_handle* h, int64_t n, const double* x, double* out,
                  void* stream);

/* Allocation-free block dot product W = Q^T X (same layouts and result as
 * sg_block_dot without `sym`).  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- frameworks and
 * services that give out all device memory through their own pool
 * allocator, programs with a device-memory budget fixed at start-up, and
 * code that must not add the device-wide synchronisation of cudaFree.
 *  - No handle and no allocation: the split partial sums live in a
 *    file-scope device array of SG_NOALLOC_SCRATCH_DOUBLES doubles (4 MiB)
 *    that every GPU loading the library holds until the process exits.
 *  - Runs on the calling thread's current device and on `stream` (NULL is
 *    the legacy default stream).  The first call on a device looks up the
 *    array's device address (cudaGetSymbolAddress) and keeps it for the
 *    life of the process; make that first call before any stream capture.
 *    A cudaDeviceReset unloads the array with the module, so make no
 *    further calls on a device after resetting it.
 *  - Requires i*s <= SG_NOALLOC_SCRATCH_DOUBLES; larger shapes return
 *    SG_EINVAL with the limit in the message.  Q, X, W: device memory.
 *  - Every call shares the one array, so calls that overlap on the GPU
 *    (other streams, other host threads) race and corrupt each other;
 *    serialise them.  Each call overwrites the partials it reads, so
 *    nothing needs clearing between calls.
 *  - err (may be NULL) receives a message of at most err_cap bytes. */
#define SG_NOALLOC_SCRATCH_DOUBLES (1 << 19)
sg_status sg_block_dot_noalloc(int64_t n, const double* Q, int64_t ldq,
                               int32_t i, const double* X, int64_t ldx,
                               int32_t s, double* W, int32_t ldw,
                               void* stream, char* err, int32_t err_cap);

/* Failure-detection probe (a diagnostic; the paper has no counterpart).
 * Every wait inside the library's kernels (the grid barrier of the
 * cooperative Arnoldi step, the mbarriers of the tensor-core kernels) is
 * time-bounded: when it runs out the kernel sets an error flag, finishes
 * without the missing data and the call returns SG_ECUDA.  This call runs
 * two tiny kernels on `device` whose waits cannot complete -- a grid
 * barrier expecting one block more than is launched, and an mbarrier that
 * nothing arrives on -- with a limit of limit_ms (clamped to 1..2000 ms),
 * and reports in *grid_barrier_timed_out / *mbarrier_timed_out (1/0)
 * whether each wait ran out and was reported.  The device stays usable.
 * Errors: SG_EINVAL (NULL output), SG_ECUDA. */
sg_status sg_probe_bounded_waits(int32_t device, double limit_ms,
                                 int32_t* grid_barrier_timed_out,
                                 int32_t* mbarrier_timed_out);

/* Number of kernels this library has launched in the process so far (a
 * diagnostic for benchmarks: every launch goes through one counter). */
int64_t sg_kernel_launches(void);

/* Tensor-core policy of the FP64 block products (not in the paper; the
 * paper's BCGS kernels run on CPUs).  SG_TC_AUTO (0, the default): the
 * tensor-core form of sg_block_dot / sg_block_update (and of the solver's
 * own block products) runs where a per-shape cost model expects it to beat
 * the FP64 pipe; SG_TC_NEVER (1): always the FP64-pipe kernels (also what
 * the environment variable SGMRES_NO_TC=1 selects at the first call);
 * SG_TC_ALWAYS (2): the tensor-core form wherever its layout requirements
 * hold.  Both forms give the same products to FP64 rounding, so this only
 * chooses speed.  Process-wide; returns the previous policy, or -1 for an
 * unknown value (nothing changed). */
#define SG_TC_AUTO 0
#define SG_TC_NEVER 1
#define SG_TC_ALWAYS 2
int32_t sg_set_tc_policy(int32_t policy);

/* ------------------------------------------- host small dense algebra
 * Pure host functions (no handle, no GPU) used between kernels; exposed
 * so they can be checked on their own. */

/* Partial Cholesky with the ICE condition stop (Alg. 3, Sec. 3.2): G is
 * s x s (ldg), R receives the p x p factor (column-major, ld = s), kappa
 * the estimates kappa_1..kappa_p (and the rejected one, if any).  Returns
 * p (0 when the first pivot is not positive). */
int32_t sg_host_partial_cholesky(const double* G, int32_t ldg, int32_t s,
                                 double omega, double* R, double* kappa);

/* Eigenvalues of an upper Hessenberg k x k matrix (ldh) by the implicit
 * double-shift QR iteration: the Ritz values of the Arnoldi pre-pass
 * (Sec. 3.4).  Complex pairs are returned as exact conjugates.  Returns 0,
 * or -1 when the iteration does not converge. */
int32_t sg_host_hessenberg_eigvals(const double* H, int32_t ldh, int32_t k,
                                   double* re, double* im);

/* Leja order of k values with conjugate pairs adjacent (Sec. 3.4). */
void sg_host_leja_order(int32_t k, const double* re, const double* im,
                        double* out_re, double* out_im);

/* gamma_i = |mean(theta) - theta_i| (Eq. scalingcoeff), degenerate
 * values replaced by the mean of the others (1 if none). */
void sg_host_scaling_coefficients(int32_t k, const double* re,
                                  const double* im, double* gamma);

/* Initial step size estimator (Sec. 3.5, Eq. auxiliarymatrix): column
 * norms of E into norms (length k, may be NULL) and s0* = number of
 * leading columns with ||E_j|| < omega_est, clamped to [s_min, s_max]. */
int32_t sg_host_estimate_step(int32_t k, const double* re, const double* im,
                              double eps, double omega_est, int32_t s_min,
                              int32_t s_max, double* norms);

/* Inverse of the leading p x p block of the upper-triangular R (the
 * triangular factor of a partial CholQR, Alg. 4 'Q_k = X Z^-1').  Returns 0,
 * or -1 on bad arguments. */
int32_t sg_host_upper_inverse(const double* R, int32_t ldr, int32_t p, double* Ri,
                              int32_t ldri);

/* Basis parameters of s steps of the matrix powers kernel from the
 * Leja-ordered shifts (re, im; a conjugate pair in consecutive entries)
 * and scaling coefficients gamma (Eq. newtonrecurrence and its pair form):
 * per step the real shift theta[j], the coefficient c[j] of V_{j-1} (b^2 /
 * gamma_{j-1} on a pair's second step, else 0) and the scale g[j], and the
 * (s+1) x s change-of-basis matrix B with A V(:, 1:s) = V B (ldb >= s+1).
 * Any output may be NULL.  Returns 0, or -1 on bad arguments. */
int32_t sg_host_basis(int32_t s, const double* re, const double* im,
                      const double* gamma, double* theta, double* c, double* g,
                      double* B, int32_t ldb);

/* The two BCGS passes combined (Alg. 4 'Combine both steps'):
 * R_top = W(:, 1:q) + R'(:, 1:q) Z(1:q, 1:q) (i x q) and
 * R_kk = Z~(1:q, 1:q) Z(1:q, 1:q) (q x q), Z and Z~ upper triangular.
 * Returns 0, or -1 on bad arguments. */
int32_t sg_host_combine_r(int32_t i, int32_t q, const double* W, int32_t ldw,
                          const double* Rp, int32_t ldrp, const double* Z1,
                          int32_t ldz1, const double* R2, int32_t ldr2,
                          double* R_top, int32_t ldt, double* R_kk, int32_t ldk);

/* New columns i..i+q-1 (1-based i) of the unrotated Hessenberg matrix H
 * (ld >= i+q) from V = Q Rbar and A V(:, 1:q) = V B (Alg. 4 'Assemble upper
 * Hessenberg'): H(:, new) = (Rbar B - [H_old Rbar_top; 0]) T^-1, with Rbar's
 * first column e_i and the rest [R_top; R_kk].  Uses H's earlier columns.
 * Returns 0, or -1 on bad arguments. */
int32_t sg_host_assemble_hessenberg(double* H, int32_t ldh, int32_t i, int32_t q,
                                    const double* R_top, int32_t ldt,
                                    const double* R_kk, int32_t ldk, const double* B,
                                    int32_t ldb);

/* Least-squares update of GMRES for column j (0-based) of the unrotated
 * H (Alg. 1 'Apply Givens'): copies rows 0..j+1 of it into Hr, applies the
 * rotations cs/sn[0..j-1], makes rotation j, updates g (length >= j+2) and
 * returns |g[j+1]|, the residual norm of the least-squares problem (-1 on
 * bad arguments). */
double sg_host_givens_column(double* Hr, int32_t ldhr, double* cs, double* sn,
                             double* g, const double* H, int32_t ldh, int32_t j);

/* y (length jj) of the triangular system Hr(0:jj, 0:jj) y = g(0:jj). */
int32_t sg_host_givens_solve(const double* Hr, int32_t ldhr, const double* g,
                             int32_t jj, double* y);

/* Halo of a row block for the row-partitioned solve (Sec. 5: rows are
 * distributed over processes, and every SpMV needs the entries of x that
 * other processes own).  rows = hi - lo consecutive rows [lo, hi) in CSR
 * with global column indices (rowptr starts at 0).  Writes the sorted
 * distinct columns outside [lo, hi) to halo_cols (capacity >= rowptr[rows];
 * may be NULL) and each entry's local column to local_colind (may be NULL):
 * c - lo for an owned column, rows + its position in halo_cols otherwise,
 * so the block is a rows x (rows + halo) matrix over [own x; halo x].
 * Entry order is kept.  Returns the number of halo columns, -1 on bad
 * arguments. */
int64_t sg_host_halo_plan(int32_t rows, const int32_t* rowptr, const int32_t* colind,
                          int32_t lo, int32_t hi, int32_t* local_colind,
                          int32_t* halo_cols);

#ifdef __cplusplus
}
#endif

#endif /* SGMRES_H */
