// Host-side small dense FP64 algebra of the adaptive s-step GMRES: the
// parts the paper keeps "local to each processor" (Sec. 2): partial
// Cholesky with the incremental condition estimator (Alg. 3), triangular
// inverses, Ritz values, Leja ordering, scaling coefficients, the step-size
// estimator (Sec. 3.5), Hessenberg assembly and Givens rotations (Alg. 4).
#pragma once
#include <cstdint>
#include <vector>

namespace sg {

// Column-major helper: element (r, c) of a matrix with leading dim ld.
inline double& at(double* a, int64_t ld, int64_t r, int64_t c) {
  return a[r + c * ld];
}
inline double at(const double* a, int64_t ld, int64_t r, int64_t c) {
  return a[r + c * ld];
}

// Alg. 3 with the ICE stop.  Returns p; R (s x s, ld = ldr) holds the
// p x p factor in its leading block (rest zero).
int partial_cholesky(const double* G, int ldg, int s, double omega,
                     double* R, int ldr, double* kappa);

// Inverse of the leading p x p block of an upper-triangular R.
void upper_inverse(const double* R, int ldr, int p, double* Ri, int ldri);

// Eigenvalues of an upper Hessenberg matrix (implicit double shift QR).
int hessenberg_eigvals(const double* H, int ldh, int k, double* re,
                       double* im);

void leja_order(int k, const double* re, const double* im, double* ore,
                double* oim);
void scaling_coefficients(int k, const double* re, const double* im,
                          double* gamma);
int estimate_step(int k, const double* re, const double* im, double eps,
                  double omega_est, int s_min, int s_max, double* norms);

// Per-step basis parameters and the change-of-basis matrix B, (s+1) x s.
struct BasisStep {
  double theta;   // real shift a (Re theta)
  double c;       // coefficient of V_{j-1} (b^2/gamma_{j-1} on a pair's
                  // second step, else 0)
  double gamma;   // scale
};
void basis_steps(int s, const double* re, const double* im,
                 const double* gamma, std::vector<BasisStep>& out);
void change_of_basis(const std::vector<BasisStep>& st, int s, double* B,
                     int ldb);

// New Hessenberg columns i..i+q-1 (1-based i) of the unrotated H
// ((m+1) x m, ld = ldh) from R_top (i x q, ld), R_kk (q x q, ld) and the
// change-of-basis B ((q+1) x q, ld).  Uses H's previous columns.
void assemble_hessenberg(double* H, int ldh, int i, int q,
                         const double* R_top, int ldt, const double* R_kk,
                         int ldk, const double* B, int ldb);

// R_top = W(:, 1:q) + R'(:, 1:q) Z(1:q, 1:q) (i x q) and R_kk = Z~ Z(1:q, 1:q)
// (q x q, upper triangular): the two BCGS passes combined (Alg. 4
// 'Combine both steps').  Z and Z~ are upper triangular.
void combine_r(int i, int q, const double* W, int ldw, const double* Rp, int ldrp,
               const double* Z1, int ldz1, const double* R2, int ldr2, double* R_top,
               int ldt, double* R_kk, int ldk);

// Column j of the unrotated H (rows 0..j+1) into Hr, rotated by the
// previous rotations; a new rotation annihilates Hr(j+1, j) and updates g.
// Returns |g[j+1]| (Alg. 1 'Apply Givens').
double givens_column(double* Hr, int ldhr, double* cs, double* sn, double* g,
                     const double* H, int ldh, int j);
// y of the leading jj x jj triangular system Hr y = g.
void givens_solve(const double* Hr, int ldhr, const double* g, int jj, double* y);

// Halo of a block of consecutive rows [lo, hi) of a row-partitioned CSR
// (columns global): the sorted distinct columns outside [lo, hi) into
// halo_cols (may be NULL), and each entry's local column into
// local_colind (may be NULL): c - lo for an owned column, rows + its
// position in halo_cols otherwise.  Returns the number of halo columns.
int64_t halo_plan(int rows, const int32_t* rowptr, const int32_t* colind, int32_t lo,
                  int32_t hi, int32_t* local_colind, int32_t* halo_cols);

// Least-squares state of GMRES: rotated Hessenberg, rotations, g.
struct Givens {
  int m = 0;
  std::vector<double> Hr, cs, sn, g;
  void reset(int m_, double beta);
  // copies column j (rows 0..j+1) from H, rotates it, updates g; returns
  // |g[j+1]|.
  double add_column(const double* H, int ldh, int j);
  // y of the leading jj x jj triangular system Hr y = g.
  void solve(int jj, double* y) const;
};

}  // namespace sg
