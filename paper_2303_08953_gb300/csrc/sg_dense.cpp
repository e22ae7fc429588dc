// Host FP64 small dense algebra (see sg_dense.h).
#include "sg_dense.h"

#include <algorithm>
#include <cmath>
#include <limits>
#include <numeric>

namespace sg {

namespace {

// Largest eigenvalue of the symmetric 2x2 [[a, b], [b, d]] and a unit
// eigenvector (u0, u1).
void sym2_top(double a, double b, double d, double* lam, double* u0,
              double* u1) {
  const double half = 0.5 * (a - d);
  const double rad = std::hypot(half, b);
  *lam = 0.5 * (a + d) + rad;
  if (b == 0.0) {
    *u0 = (a >= d) ? 1.0 : 0.0;
    *u1 = (a >= d) ? 0.0 : 1.0;
    return;
  }
  // two algebraically equal eigenvector forms; keep the longer one
  double x1 = b, y1 = *lam - a, x2 = *lam - d, y2 = b;
  double n1 = std::hypot(x1, y1), n2 = std::hypot(x2, y2);
  if (n1 >= n2) { *u0 = x1 / n1; *u1 = y1 / n1; }
  else          { *u0 = x2 / n2; *u1 = y2 / n2; }
}

// Incremental condition estimate of an upper-triangular factor grown by
// columns (Sec. 3.2, after Bischof's ICE).  xmax: unit vector whose image
// x^T R has norm Dmax (lower bound of sigma_max); wmin = R^-T y for a unit
// y, with ||wmin|| = 1/dmin (dmin an upper bound of sigma_min).
struct IncCond {
  std::vector<double> xmax, wmin;
  double Dmax = 0, dmin = 0;
  void start(double r11) {
    xmax.assign(1, 1.0);
    wmin.assign(1, 1.0 / r11);
    Dmax = std::fabs(r11);
    dmin = std::fabs(r11);
  }
  // new column: v = R(0:j-1, j), gam = R(j, j)
  double grow(const double* v, int j, double gam) {
    double al = 0.0, al2 = 0.0;
    for (int t = 0; t < j; ++t) { al += xmax[t] * v[t]; al2 += wmin[t] * v[t]; }
    double nu, s1, c1;
    sym2_top(Dmax * Dmax + al * al, al * gam, gam * gam, &nu, &s1, &c1);
    for (int t = 0; t < j; ++t) xmax[t] *= s1;
    xmax.push_back(c1);
    Dmax = std::sqrt(nu);
    const double ig2 = 1.0 / (gam * gam);
    double mu, s2, c2;
    sym2_top(1.0 / (dmin * dmin) + al2 * al2 * ig2, -al2 * ig2, ig2, &mu, &s2,
             &c2);
    for (int t = 0; t < j; ++t) wmin[t] *= s2;
    wmin.push_back((c2 - s2 * al2) / gam);
    dmin = 1.0 / std::sqrt(mu);
    return Dmax / dmin;
  }
};

}  // namespace

int partial_cholesky(const double* G, int ldg, int s, double omega,
                     double* R, int ldr, double* kappa) {
  for (int c = 0; c < s; ++c)
    for (int r = 0; r < s; ++r) at(R, ldr, r, c) = 0.0;
  IncCond ice;
  std::vector<double> col(s);
  for (int j = 0; j < s; ++j) {
    // off-diagonal entries of column j: forward substitution with R^T
    for (int i = 0; i < j; ++i) {
      double acc = at(G, ldg, i, j);
      for (int k = 0; k < i; ++k) acc -= at(R, ldr, k, i) * at(R, ldr, k, j);
      at(R, ldr, i, j) = acc / at(R, ldr, i, i);
    }
    double piv = at(G, ldg, j, j);
    for (int k = 0; k < j; ++k) piv -= at(R, ldr, k, j) * at(R, ldr, k, j);
    if (!(piv > 0.0) || !std::isfinite(piv)) {
      for (int i = 0; i < j; ++i) at(R, ldr, i, j) = 0.0;
      return j;
    }
    const double rjj = std::sqrt(piv);
    at(R, ldr, j, j) = rjj;
    double kap;
    if (j == 0) {
      ice.start(rjj);
      kap = 1.0;
    } else {
      for (int i = 0; i < j; ++i) col[i] = at(R, ldr, i, j);
      kap = ice.grow(col.data(), j, rjj);
    }
    if (kappa) kappa[j] = kap;
    if (kap > omega) {
      for (int i = 0; i <= j; ++i) at(R, ldr, i, j) = 0.0;
      return j;
    }
  }
  return s;
}

void upper_inverse(const double* R, int ldr, int p, double* Ri, int ldri) {
  for (int c = 0; c < p; ++c)
    for (int r = 0; r < p; ++r) at(Ri, ldri, r, c) = 0.0;
  // column c of R^-1 solves R x = e_c by back substitution
  for (int c = 0; c < p; ++c) {
    at(Ri, ldri, c, c) = 1.0 / at(R, ldr, c, c);
    for (int r = c - 1; r >= 0; --r) {
      double acc = 0.0;
      for (int k = r + 1; k <= c; ++k) acc += at(R, ldr, r, k) * at(Ri, ldri, k, c);
      at(Ri, ldri, r, c) = -acc / at(R, ldr, r, r);
    }
  }
}

// ------------------------------------------------------------ eigenvalues
namespace {

void eig2(double a, double b, double c, double d, double* re, double* im) {
  // eigenvalues of [[a, b], [c, d]]
  const double p = 0.5 * (a - d);
  const double disc = p * p + b * c;
  const double mid = 0.5 * (a + d);
  if (disc >= 0.0) {
    const double sq = std::sqrt(disc);
    const double l1 = mid + (p >= 0.0 ? sq : -sq);
    const double det = a * d - b * c;
    const double l2 = (l1 != 0.0) ? det / l1 : mid - (p >= 0.0 ? sq : -sq);
    re[0] = l1; im[0] = 0.0;
    re[1] = l2; im[1] = 0.0;
  } else {
    const double sq = std::sqrt(-disc);
    re[0] = mid; im[0] = sq;
    re[1] = mid; im[1] = -sq;
  }
}

// Householder reflector for (x0, x1[, x2]): P = I - tau v v^T with v0 = 1,
// P x = beta e1.  Returns tau (0 when x is already e1-aligned).
double house(int len, double* x, double* v) {
  double sig = 0.0;
  for (int t = 1; t < len; ++t) sig += x[t] * x[t];
  v[0] = 1.0;
  for (int t = 1; t < len; ++t) v[t] = x[t];
  if (sig == 0.0) return 0.0;
  const double nx = std::sqrt(x[0] * x[0] + sig);
  const double v0 = (x[0] <= 0.0) ? x[0] - nx : -sig / (x[0] + nx);
  const double tau = 2.0 * v0 * v0 / (sig + v0 * v0);
  for (int t = 1; t < len; ++t) v[t] /= v0;
  return tau;
}

}  // namespace

int hessenberg_eigvals(const double* Hin, int ldh, int k, double* re,
                       double* im) {
  if (k <= 0) return 0;
  std::vector<double> a(static_cast<size_t>(k) * k);
  auto A = [&](int r, int c) -> double& { return a[r + static_cast<size_t>(c) * k]; };
  double hnorm = 0.0;
  for (int c = 0; c < k; ++c)
    for (int r = 0; r < k; ++r) {
      A(r, c) = (r <= c + 1) ? at(Hin, ldh, r, c) : 0.0;
      hnorm = std::max(hnorm, std::fabs(A(r, c)));
    }
  const double eps = std::numeric_limits<double>::epsilon();
  int hi = k - 1;
  int its = 0, total_its = 0;
  while (hi >= 0) {
    // find the start l of the unreduced active block ending at hi
    int l = hi;
    while (l > 0) {
      double sc = std::fabs(A(l - 1, l - 1)) + std::fabs(A(l, l));
      if (sc == 0.0) sc = hnorm;
      if (std::fabs(A(l, l - 1)) <= eps * sc) {
        A(l, l - 1) = 0.0;
        break;
      }
      --l;
    }
    if (l == hi) {                       // 1x1 block converged
      re[hi] = A(hi, hi);
      im[hi] = 0.0;
      --hi;
      its = 0;
      continue;
    }
    if (l == hi - 1) {                   // 2x2 block converged
      double r2[2], i2[2];
      eig2(A(hi - 1, hi - 1), A(hi - 1, hi), A(hi, hi - 1), A(hi, hi), r2, i2);
      re[hi - 1] = r2[0]; im[hi - 1] = i2[0];
      re[hi] = r2[1];     im[hi] = i2[1];
      hi -= 2;
      its = 0;
      continue;
    }
    if (++total_its > 100 * k) return -1;
    ++its;
    // Francis double shift from the trailing 2x2 (sum s, product t);
    // an ad hoc shift every 10 stalled iterations breaks cycles.
    double s, t;
    if (its % 10 == 0) {
      // exceptional shifts A(hi,hi) +- w, w the size of the last two
      // subdiagonal entries
      const double w = std::fabs(A(hi, hi - 1)) + std::fabs(A(hi - 1, hi - 2));
      s = 2.0 * A(hi, hi);
      t = A(hi, hi) * A(hi, hi) - w * w;
    } else {
      s = A(hi - 1, hi - 1) + A(hi, hi);
      t = A(hi - 1, hi - 1) * A(hi, hi) - A(hi - 1, hi) * A(hi, hi - 1);
    }
    // first column of (H^2 - s H + t I) restricted to the block
    double x[3];
    x[0] = A(l, l) * A(l, l) + A(l, l + 1) * A(l + 1, l) - s * A(l, l) + t;
    x[1] = A(l + 1, l) * (A(l, l) + A(l + 1, l + 1) - s);
    x[2] = A(l + 1, l) * A(l + 2, l + 1);
    for (int q = l; q <= hi - 2; ++q) {
      double v[3];
      const double tau = house(3, x, v);
      if (tau != 0.0) {
        const int c0 = std::max(l, q - 1);
        for (int c = c0; c <= hi; ++c) {      // from the left, rows q..q+2
          const double dot = A(q, c) + v[1] * A(q + 1, c) + v[2] * A(q + 2, c);
          const double f = tau * dot;
          A(q, c) -= f;
          A(q + 1, c) -= f * v[1];
          A(q + 2, c) -= f * v[2];
        }
        const int r1 = std::min(q + 3, hi);
        for (int r = l; r <= r1; ++r) {       // from the right, cols q..q+2
          const double dot = A(r, q) + v[1] * A(r, q + 1) + v[2] * A(r, q + 2);
          const double f = tau * dot;
          A(r, q) -= f;
          A(r, q + 1) -= f * v[1];
          A(r, q + 2) -= f * v[2];
        }
      }
      x[0] = A(q + 1, q);
      x[1] = A(q + 2, q);
      if (q < hi - 2) x[2] = A(q + 3, q);
    }
    {  // final 2-element reflector on rows/cols hi-1, hi
      const int q = hi - 1;
      double v[2];
      const double tau = house(2, x, v);
      if (tau != 0.0) {
        for (int c = std::max(l, q - 1); c <= hi; ++c) {
          const double f = tau * (A(q, c) + v[1] * A(q + 1, c));
          A(q, c) -= f;
          A(q + 1, c) -= f * v[1];
        }
        for (int r = l; r <= hi; ++r) {
          const double f = tau * (A(r, q) + v[1] * A(r, q + 1));
          A(r, q) -= f;
          A(r, q + 1) -= f * v[1];
        }
      }
    }
    // clean the bulge remnants below the subdiagonal
    for (int c = l; c <= hi; ++c)
      for (int r = c + 2; r <= hi; ++r) A(r, c) = 0.0;
  }
  return 0;
}

// ---------------------------------------------------------------- Leja
namespace {
bool is_tie(double a, double b) {
  if (std::isinf(a) || std::isinf(b)) return a == b;
  return std::fabs(a - b) <= 1e-9 * std::max({1.0, std::fabs(a), std::fabs(b)});
}
// candidate (score sc, value (cr, ci), index ic) beats the best so far?
bool beats(double sc, double cr, double ci, int ic, double sb, double br,
           double bi, int ib) {
  if (!is_tie(sc, sb)) return sc > sb;
  if (cr != br) return cr > br;
  if (ci != bi) return ci > bi;
  return ic < ib;
}
}  // namespace

void leja_order(int k, const double* re, const double* im, double* ore,
                double* oim) {
  std::vector<char> used(k, 0);
  std::vector<int> order;
  order.reserve(k);
  auto take = [&](int i) {
    order.push_back(i);
    used[i] = 1;
    if (im[i] > 0.0) {  // its conjugate follows at once
      int best = -1;
      double bd = 0.0;
      for (int j = 0; j < k; ++j) {
        if (used[j] || !(im[j] < 0.0)) continue;
        const double d = std::hypot(re[j] - re[i], im[j] + im[i]);
        if (best < 0 || d < bd) { best = j; bd = d; }
      }
      if (best >= 0) { order.push_back(best); used[best] = 1; }
    }
  };
  int first = -1;
  double fs = 0.0;
  for (int i = 0; i < k; ++i) {
    if (im[i] < 0.0) continue;
    const double sc = std::hypot(re[i], im[i]);
    if (first < 0 || beats(sc, re[i], im[i], i, fs, re[first], im[first], first)) {
      first = i;
      fs = sc;
    }
  }
  if (first >= 0) take(first);
  while (static_cast<int>(order.size()) < k) {
    int best = -1;
    double bs = 0.0;
    for (int i = 0; i < k; ++i) {
      if (used[i] || im[i] < 0.0) continue;
      double sc = 0.0;
      for (int j : order) {
        const double d = std::hypot(re[i] - re[j], im[i] - im[j]);
        if (d == 0.0) { sc = -std::numeric_limits<double>::infinity(); break; }
        sc += std::log(d);
      }
      if (best < 0 || beats(sc, re[i], im[i], i, bs, re[best], im[best], best)) {
        best = i;
        bs = sc;
      }
    }
    if (best < 0) {  // only unmatched negative-imaginary values remain
      for (int i = 0; i < k; ++i) if (!used[i]) { best = i; break; }
      order.push_back(best);
      used[best] = 1;
      continue;
    }
    take(best);
  }
  for (int t = 0; t < k; ++t) { ore[t] = re[order[t]]; oim[t] = im[order[t]]; }
}

void scaling_coefficients(int k, const double* re, const double* im,
                          double* gamma) {
  if (k <= 0) return;
  double mean = 0.0, amax = 0.0;
  for (int t = 0; t < k; ++t) {
    mean += re[t];
    amax = std::max(amax, std::hypot(re[t], im[t]));
  }
  mean /= k;
  double good_sum = 0.0;
  int good = 0;
  std::vector<char> bad(k, 0);
  for (int t = 0; t < k; ++t) {
    gamma[t] = std::hypot(mean - re[t], im[t]);
    if (gamma[t] <= 1e-14 * amax) bad[t] = 1;
    else { good_sum += gamma[t]; ++good; }
  }
  const double fill = good ? good_sum / good : 1.0;
  for (int t = 0; t < k; ++t) if (bad[t]) gamma[t] = fill;
}

int estimate_step(int k, const double* re, const double* im, double eps,
                  double omega_est, int s_min, int s_max, double* norms) {
  // log2 E (Eq. auxiliarymatrix), one column at a time; row i carries
  // the running log-product over k < j (skipping k = i once j > i).
  double mean = 0.0;
  for (int t = 0; t < k; ++t) mean += re[t];
  mean = k ? mean / k : 0.0;
  std::vector<double> den(k);
  for (int t = 0; t < k; ++t) den[t] = std::log2(std::hypot(mean - re[t], im[t]));
  const double le = std::log2(eps);
  std::vector<double> run(k, 0.0), col(k);
  int s0 = k;
  bool crossed = false;
  for (int j = 0; j < k; ++j) {
    double mx = -std::numeric_limits<double>::infinity();
    for (int i = 0; i < k; ++i) {
      col[i] = (j < i) ? run[i] : run[i] + le;
      mx = std::max(mx, col[i]);
    }
    double acc = 0.0;
    if (std::isfinite(mx))
      for (int i = 0; i < k; ++i) acc += std::exp2(2.0 * (col[i] - mx));
    const double nrm = std::isfinite(mx) ? std::exp2(mx) * std::sqrt(acc) : 0.0;
    if (norms) norms[j] = nrm;
    if (!crossed && !(nrm < omega_est)) { s0 = j; crossed = true; }
    // advance the running products with factor k = j (skipped in row j)
    for (int i = 0; i < k; ++i) {
      if (i == j) continue;
      const double d = std::hypot(re[i] - re[j], im[i] - im[j]);
      run[i] += (d == 0.0) ? -std::numeric_limits<double>::infinity()
                           : std::log2(d) - den[j];
    }
  }
  if (s_max > 0) s0 = std::min(s0, s_max);
  return std::max(s0, s_min);
}

// ---------------------------------------------------------------- basis
void basis_steps(int s, const double* re, const double* im,
                 const double* gamma, std::vector<BasisStep>& out) {
  out.assign(s, BasisStep{0.0, 0.0, 1.0});
  for (int j = 0; j < s; ++j) {
    out[j].theta = re[j];
    out[j].gamma = gamma[j];
    if (j > 0 && im[j] < 0.0 && im[j - 1] > 0.0)
      out[j].c = im[j] * im[j] / gamma[j - 1];
  }
}

void change_of_basis(const std::vector<BasisStep>& st, int s, double* B,
                     int ldb) {
  for (int c = 0; c < s; ++c)
    for (int r = 0; r <= s; ++r) at(B, ldb, r, c) = 0.0;
  for (int j = 0; j < s; ++j) {
    at(B, ldb, j, j) = st[j].theta;
    at(B, ldb, j + 1, j) = st[j].gamma;
    if (st[j].c != 0.0) at(B, ldb, j - 1, j) = -st[j].c;
  }
}

void assemble_hessenberg(double* H, int ldh, int i, int q,
                         const double* R_top, int ldt, const double* R_kk,
                         int ldk, const double* B, int ldb) {
  // Rbar ((i+q) x (q+1)): column 0 = e_i, then [R_top; R_kk].
  const int nr = i + q;
  std::vector<double> Rb(static_cast<size_t>(nr) * (q + 1), 0.0);
  auto RB = [&](int r, int c) -> double& { return Rb[r + static_cast<size_t>(c) * nr]; };
  RB(i - 1, 0) = 1.0;
  for (int c = 0; c < q; ++c) {
    for (int r = 0; r < i; ++r) RB(r, c + 1) = at(R_top, ldt, r, c);
    for (int r = 0; r < q; ++r) RB(i + r, c + 1) = at(R_kk, ldk, r, c);
  }
  // M = Rbar * B(0:q, 0:q-1) - [H(0:i-1, 0:i-2) Rbar(0:i-2, 0:q-1); 0]
  std::vector<double> M(static_cast<size_t>(nr) * q, 0.0);
  auto MM = [&](int r, int c) -> double& { return M[r + static_cast<size_t>(c) * nr]; };
  for (int c = 0; c < q; ++c)
    for (int t = 0; t <= q; ++t) {
      const double bv = at(B, ldb, t, c);
      if (bv == 0.0) continue;
      for (int r = 0; r < nr; ++r) MM(r, c) += RB(r, t) * bv;
    }
  if (i > 1)
    for (int c = 0; c < q; ++c)
      for (int t = 0; t < i - 1; ++t) {
        const double rv = RB(t, c);
        if (rv == 0.0) continue;
        for (int r = 0; r < i; ++r) MM(r, c) -= at(H, ldh, r, t) * rv;
      }
  // H_new T = M with T = Rbar(i-1 : i+q-2, 0:q-1), upper triangular
  for (int r = 0; r < nr; ++r) {
    for (int c = 0; c < q; ++c) {
      double acc = MM(r, c);
      for (int t = 0; t < c; ++t) acc -= at(H, ldh, r, i - 1 + t) * RB(i - 1 + t, c);
      at(H, ldh, r, i - 1 + c) = acc / RB(i - 1 + c, c);
    }
  }
  for (int c = 0; c < q; ++c)
    for (int r = nr; r < ldh; ++r) at(H, ldh, r, i - 1 + c) = 0.0;
}

void Givens::reset(int m_, double beta) {
  m = m_;
  Hr.assign(static_cast<size_t>(m + 1) * m, 0.0);
  cs.assign(m, 0.0);
  sn.assign(m, 0.0);
  g.assign(m + 1, 0.0);
  g[0] = beta;
}

double givens_column(double* Hr, int ldhr, double* cs, double* sn, double* g,
                     const double* H, int ldh, int j) {
  double* h = Hr + static_cast<size_t>(j) * ldhr;
  for (int r = 0; r <= j + 1; ++r) h[r] = at(H, ldh, r, j);
  for (int l = 0; l < j; ++l) {
    const double t = cs[l] * h[l] + sn[l] * h[l + 1];
    h[l + 1] = -sn[l] * h[l] + cs[l] * h[l + 1];
    h[l] = t;
  }
  const double a = h[j], b = h[j + 1];
  const double r = std::hypot(a, b);
  if (r == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
  else { cs[j] = a / r; sn[j] = b / r; }
  h[j] = r;
  h[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  return std::fabs(g[j + 1]);
}

void givens_solve(const double* Hr, int ldhr, const double* g, int jj, double* y) {
  for (int r = jj - 1; r >= 0; --r) {
    double acc = g[r];
    for (int c = r + 1; c < jj; ++c) acc -= Hr[r + static_cast<size_t>(c) * ldhr] * y[c];
    y[r] = acc / Hr[r + static_cast<size_t>(r) * ldhr];
  }
}

double Givens::add_column(const double* H, int ldh, int j) {
  return givens_column(Hr.data(), m + 1, cs.data(), sn.data(), g.data(), H, ldh, j);
}

void Givens::solve(int jj, double* y) const {
  givens_solve(Hr.data(), m + 1, g.data(), jj, y);
}

void combine_r(int i, int q, const double* W, int ldw, const double* Rp, int ldrp,
               const double* Z1, int ldz1, const double* R2, int ldr2, double* R_top,
               int ldt, double* R_kk, int ldk) {
  for (int c = 0; c < q; ++c) {
    for (int r = 0; r < i; ++r) {
      double acc = W[r + static_cast<int64_t>(c) * ldw];
      for (int t = 0; t <= c; ++t)
        acc += Rp[r + static_cast<int64_t>(t) * ldrp] * Z1[t + static_cast<int64_t>(c) * ldz1];
      R_top[r + static_cast<int64_t>(c) * ldt] = acc;
    }
    for (int r = 0; r < q; ++r) {
      double acc = 0.0;
      for (int t = r; t <= c; ++t)
        acc += R2[r + static_cast<int64_t>(t) * ldr2] * Z1[t + static_cast<int64_t>(c) * ldz1];
      R_kk[r + static_cast<int64_t>(c) * ldk] = acc;
    }
  }
}

int64_t halo_plan(int rows, const int32_t* rowptr, const int32_t* colind, int32_t lo,
                  int32_t hi, int32_t* local_colind, int32_t* halo_cols) {
  const int64_t nnz = rowptr[rows];
  std::vector<int32_t> halo;
  for (int64_t k = 0; k < nnz; ++k)
    if (colind[k] < lo || colind[k] >= hi) halo.push_back(colind[k]);
  std::sort(halo.begin(), halo.end());
  halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
  if (halo_cols) std::copy(halo.begin(), halo.end(), halo_cols);
  if (local_colind) {
    for (int64_t k = 0; k < nnz; ++k) {
      const int32_t c = colind[k];
      if (c >= lo && c < hi) {
        local_colind[k] = c - lo;
      } else {
        const auto it = std::lower_bound(halo.begin(), halo.end(), c);
        local_colind[k] = rows + static_cast<int32_t>(it - halo.begin());
      }
    }
  }
  return static_cast<int64_t>(halo.size());
}

}  // namespace sg
