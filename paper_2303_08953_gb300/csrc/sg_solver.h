// Handle, device workspace and the host driver of the solver.
#pragma once
#include <string>
#include <vector>

#include "sg_dense.h"
#include "sg_internal.h"

struct sg_handle {
  int device = 0;
  cudaStream_t own = nullptr;
  sg::DevCsr A;      // the analysed matrix
  sg::DevCsr AT;     // its transpose (built on the first adjoint call)
  bool have_A = false, have_AT = false;
  bool rows_only = false;  // A is a row block (sg_analyze_rows): kernel-level calls only
  int64_t ncols = 0;       // columns of A (n for a square matrix)
  std::string err;

  // workspace (sized on demand, kept until destroy)
  int64_t ws_n = 0, ld = 0;
  int ws_m = 0, ws_k = 0;
  double* Q = nullptr;      // ld x (m+1)
  double* V = nullptr;      // ld x (k+1)
  double* Y = nullptr;      // ld x k
  double* bvec = nullptr;   // n
  double* xvec = nullptr;   // n
  double* rvec = nullptr;   // n
  double* part = nullptr;   // block_dot partials
  int64_t part_cap = 0;
  double* red = nullptr;    // 3 x reduction_blocks partial sums
  double* small = nullptr;  // device small matrices
  unsigned* sync = nullptr;  // 256 B: grid-barrier words + error flag
  int64_t small_cap = 0;
  double* hbuf = nullptr;   // pinned host mirror of `small`
  // FP32 basis workspace (precision FP32_IR)
  float* Q32 = nullptr;
  float* V32 = nullptr;
  float* Y32 = nullptr;
  float* r32 = nullptr;
  int64_t ws32_n = 0;
  int ws32_m = 0, ws32_k = 0;
  double* dvec = nullptr;   // n, FP64 correction accumulator
  double* x0vec = nullptr;  // n, the initial guess kept by the FP32-basis solve
  int64_t x0_n = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // captured Ritz pre-pass graphs, keyed by everything their kernels read
  struct PrepassGraph {
    const void* key[6];
    int k = 0;
    int64_t n = 0;
    long long kernels = 0;
    cudaGraphExec_t exec = nullptr;
  };
  std::vector<PrepassGraph> graphs;
  // column equilibration: A' = A D_c shares A's pattern arrays and owns
  // its scaled values; dcol = diag(D_c)
  sg::DevCsr AE;
  bool have_AE = false;
  double* dcol = nullptr;
  void drop_graphs() {
    for (auto& g : graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    graphs.clear();
  }
};

namespace sg {

struct SolveOpts {
  int m, s, s_min, s_max, max_iters, basis;
  int equil = 0;  // sg_equil: SCALAR acts here (gamma = max |theta|)
  double tol, omega, omega_est, eps;
  int n_ritz = 0;                  // > 0: Ritz values given, no pre-pass
  const double* ritz_re = nullptr;
  const double* ritz_im = nullptr;
};

// Record of one solve (mirrors sg_result, without caller buffers).
struct SolveLog {
  bool converged = false;
  int s0 = 0, iters = 0, restarts = 0, refinements = 0;
  double final_relres = 0.0;
  std::vector<double> relres_hist, cycle_relres, ritz_re, ritz_im, gamma;
  std::vector<int> s_eff_hist, p1_hist, s_hist, cycle_iters;
  double t_prepass = 0, t_mpk = 0, t_ortho = 0, t_host = 0, t_total = 0;
  bool stalled = false;  // a refinement stall ended the FP32-basis solve
  int fp64_iters = 0;    // columns run with the FP64 basis after a stall
};

void ensure_workspace(sg_handle* h, int64_t n, int m, int k);
void count_launches(long long k);
long long launches_so_far();
void ensure_workspace32(sg_handle* h, int64_t n, int m, int k);

// Ritz pre-pass alone (Sec. 3.4): k steps of MGS-Arnoldi with M from the
// unit vector q (device, FP64; rounded to FP32 for the FP32 basis) in the
// workspace basis.  Fills H ((k+1) x k, ld k+1, host) and returns the
// steps completed.
int ritz_prepass(sg_handle* h, const DevCsr& M, const double* q, int k, bool fp32,
                 cudaStream_t st, std::vector<double>& H);

// FP64 adaptive s-step GMRES on matrix M (A or A^T): b, x device vectors
// of the workspace (x in: x0, out: solution).
void solve_fp64(sg_handle* h, const DevCsr& M, const SolveOpts& o,
                cudaStream_t st, SolveLog& log);
// FP32 basis + FP64 iterative refinement.
void solve_fp32_ir(sg_handle* h, const DevCsr& M, const SolveOpts& o,
                   double inner_tol, int max_refine, cudaStream_t st,
                   SolveLog& log);

}  // namespace sg
