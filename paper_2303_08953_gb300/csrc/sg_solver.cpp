// Host driver of the adaptive s-step GMRES (Alg. 4 with restarts): the
// kernels run on one stream; the s x s Cholesky factors, the Hessenberg
// matrix and the Givens rotations live on the host, as in the paper where
// they are "local to each processor" (Sec. 2).  Control crosses to the
// host twice per block (after each Gram matrix), carrying (i+s) x s
// values.
#include "sg_solver.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

namespace sg {

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

template <typename T>
void dev_alloc(T** p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (count == 0) return;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count);
  if (e != cudaSuccess) {
    *p = nullptr;
    throw Error(SG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
}

// Small-matrix slots inside h->small / h->hbuf (offsets in doubles).
struct Slots {
  int64_t W, G, Z, Y, scal, H, wn, total;
};
Slots slots_for(int m, int k) {
  Slots s{};
  const int64_t mm = m + 1, kk = k + 1;
  int64_t o = 0;
  s.W = o;    o += mm * kk;   // i x s block products (W, R')
  s.G = o;    o += kk * kk;   // Gram matrices
  s.Z = o;    o += kk * kk;   // inverse Cholesky factors
  s.Y = o;    o += mm;        // least-squares solution
  s.scal = o; o += 16;        // scalars (norms)
  s.H = o;    o += kk * kk;   // Arnoldi pre-pass Hessenberg ((k+1) x k)
  s.wn = o;   o += kk;        // pre-pass norms before projection
  s.total = o;
  return s;
}

// Partial sums of the streaming reductions (3 x reduction_blocks) and of
// the cooperative pre-pass (the larger of the grouped step's 24 per SM and
// the two-barrier step's partials plus its Gram rows).
int red_doubles() {
  return 3 * reduction_blocks() +
         static_cast<int>(std::max<int64_t>(24 * device_sm_count(), prepass_red_doubles()));
}

// Largest split-partials buffer over every block shape the solver uses
// (i <= imax rows of Q^T, s <= smax columns).
int64_t max_part_size(int64_t n, int imax, int smax) {
  int64_t best = 1;
  for (int i = 1; i <= std::max(imax, smax); ++i)
    for (int s = 1; s <= smax; ++s)
      best = std::max(best, block_dot_part_size(n, i, s));
  return best;
}

}  // namespace

void ensure_workspace(sg_handle* h, int64_t n, int m, int k) {
  if (h->ws_n == n && h->ws_m >= m && h->ws_k >= k && h->Q) return;
  m = std::max(m, h->ws_n == n ? h->ws_m : 0);
  k = std::max(k, h->ws_n == n ? h->ws_k : 0);
  const int64_t ld = (n + 31) / 32 * 32;  // 256-byte aligned columns
  h->drop_graphs();
  dev_alloc(&h->Q, static_cast<size_t>(ld) * (m + 1));
  dev_alloc(&h->V, static_cast<size_t>(ld) * (k + 1));
  dev_alloc(&h->Y, static_cast<size_t>(ld) * k);
  dev_alloc(&h->bvec, n);
  dev_alloc(&h->xvec, n);
  dev_alloc(&h->rvec, n);
  const int64_t part = max_part_size(n, m + 1, k);
  dev_alloc(&h->part, part);
  h->part_cap = part;
  dev_alloc(&h->red, static_cast<size_t>(red_doubles()));
  Slots sl = slots_for(m, k);
  dev_alloc(&h->small, sl.total);
  h->small_cap = sl.total;
  if (h->hbuf) cudaFreeHost(h->hbuf);
  h->hbuf = nullptr;
  SG_CUDA(cudaMallocHost(reinterpret_cast<void**>(&h->hbuf), sizeof(double) * sl.total));
  for (auto& e : h->ev)
    if (!e) SG_CUDA(cudaEventCreate(&e));
  h->ws_n = n;
  h->ld = ld;
  h->ws_m = m;
  h->ws_k = k;
}

void ensure_workspace32(sg_handle* h, int64_t n, int m, int k) {
  // FP64 vectors, partials and small slots come from the FP64 workspace
  // with empty basis blocks; the FP32 basis is allocated here.
  if (!(h->ws_n == n && h->ws_m >= m && h->ws_k >= k)) {
    h->drop_graphs();
    if (h->Q) cudaFree(h->Q);
    if (h->V) cudaFree(h->V);
    if (h->Y) cudaFree(h->Y);
    h->Q = h->V = h->Y = nullptr;
    const int mm = std::max(m, h->ws_n == n ? h->ws_m : 0);
    const int kk = std::max(k, h->ws_n == n ? h->ws_k : 0);
    const int64_t ld = (n + 31) / 32 * 32;
    dev_alloc(&h->bvec, n);
    dev_alloc(&h->xvec, n);
    dev_alloc(&h->rvec, n);
    const int64_t part = max_part_size(n, mm + 1, kk);
    dev_alloc(&h->part, part);
    h->part_cap = part;
    dev_alloc(&h->red, static_cast<size_t>(red_doubles()));
    Slots sl = slots_for(mm, kk);
    dev_alloc(&h->small, sl.total);
    h->small_cap = sl.total;
    if (h->hbuf) cudaFreeHost(h->hbuf);
    h->hbuf = nullptr;
    SG_CUDA(cudaMallocHost(reinterpret_cast<void**>(&h->hbuf), sizeof(double) * sl.total));
    for (auto& e : h->ev)
      if (!e) SG_CUDA(cudaEventCreate(&e));
    h->ws_n = n;
    h->ld = ld;
    h->ws_m = mm;
    h->ws_k = kk;
  }
  if (h->ws32_n == n && h->ws32_m >= m && h->ws32_k >= k) return;
  const int64_t ld = h->ld;
  const int mm = std::max(m, h->ws_m), kk = std::max(k, h->ws_k);
  h->drop_graphs();
  dev_alloc(&h->Q32, static_cast<size_t>(ld) * (mm + 1));
  dev_alloc(&h->V32, static_cast<size_t>(ld) * (kk + 1));
  dev_alloc(&h->Y32, static_cast<size_t>(ld) * kk);
  h->ws32_n = n;
  h->ws32_m = mm;
  h->ws32_k = kk;
}

namespace {

// Kernel set of one basis precision: FP64 (T = double) or FP32 (float).
template <typename T> struct Basis;

template <> struct Basis<double> {
  static double* Q(sg_handle* h) { return h->Q; }
  static double* V(sg_handle* h) { return h->V; }
  static double* Y(sg_handle* h) { return h->Y; }
  static void spmv(const DevCsr& M, const double* x, const double* z, double* y,
                   double th, double c, double g, cudaStream_t st) {
    spmv_newton(M, x, z, y, th, c, g, st);
  }
  static void from_f64(int64_t n, const double* r, double* q, double a, cudaStream_t st) {
    scale_copy(n, r, q, a, st);
  }
  static void bdot(int64_t n, const double* Q, int64_t ldq, int i, const double* X,
                   int64_t ldx, int s, double* W, int ldw, bool sym, double* part,
                   int64_t cap, cudaStream_t st) {
    block_dot(n, Q, ldq, i, X, ldx, s, W, ldw, sym, part, cap, st);
  }
  static void bupd(sg_handle* h, int64_t n, const double* Q, int64_t ldq, int i,
                   const double* W, int ldw, double* X, int64_t ldx, int s, double al,
                   double be, bool up, cudaStream_t st) {
    // Q's column exponents of the tensor-core form go to the (then idle)
    // split-partials buffer
    block_update(n, Q, ldq, i, W, ldw, X, ldx, s, al, be, up, h->part, h->part_cap, st);
  }
  static void gemv(int64_t n, int k, const double* Q, int64_t ldq, const double* y,
                   double* x, cudaStream_t st) {
    gemv_n_add(n, k, Q, ldq, y, x, st);
  }
};

template <> struct Basis<float> {
  static float* Q(sg_handle* h) { return h->Q32; }
  static float* V(sg_handle* h) { return h->V32; }
  static float* Y(sg_handle* h) { return h->Y32; }
  static void spmv(const DevCsr& M, const float* x, const float* z, float* y,
                   double th, double c, double g, cudaStream_t st) {
    spmv_newton32(M, x, z, y, static_cast<float>(th), static_cast<float>(c),
                  static_cast<float>(g), st);
  }
  static void from_f64(int64_t n, const double* r, float* q, double a, cudaStream_t st) {
    to_f32(n, r, q, static_cast<float>(a), st);
  }
  static void bdot(int64_t n, const float* Q, int64_t ldq, int i, const float* X,
                   int64_t ldx, int s, double* W, int ldw, bool sym, double* part,
                   int64_t cap, cudaStream_t st) {
    block_dot32(n, Q, ldq, i, X, ldx, s, W, ldw, sym, part, cap, st);
  }
  // the tensor-core update stages W's TF32 split in the (then idle)
  // split-partials buffer of the workspace
  static void bupd(sg_handle* h, int64_t n, const float* Q, int64_t ldq, int i,
                   const double* W, int ldw, float* X, int64_t ldx, int s, double al,
                   double be, bool up, cudaStream_t st) {
    block_update32(n, Q, ldq, i, W, ldw, X, ldx, s, al, be, up, h->part, h->part_cap, st);
  }
  static void gemv(int64_t n, int k, const float* Q, int64_t ldq, const double* y,
                   double* x, cudaStream_t st) {
    gemv_n_add32(n, k, Q, ldq, y, x, st);
  }
};

// ---------------------------------------------------------------------
// Ritz pre-pass: k steps of MGS-Arnoldi from q (device, unit norm) with
// the basis in V's columns (Sec. 3.4).  Returns the steps completed and
// fills Hh ((k+1) x k, host, ld k+1).
template <typename T>
void step_kernel(const DevCsr& M, T* V, int64_t ld, int j, double* H, int ldh,
                 double* wn, double* red, int red_cap, unsigned* bar, int* err,
                 cudaStream_t st);
template <>
void step_kernel<double>(const DevCsr& M, double* V, int64_t ld, int j, double* H,
                         int ldh, double* wn, double* red, int red_cap, unsigned* bar,
                         int* err, cudaStream_t st) {
  arnoldi_step(M, V, ld, j, H, ldh, wn, red, red_cap, bar, err, st);
}
template <>
void step_kernel<float>(const DevCsr& M, float* V, int64_t ld, int j, double* H,
                        int ldh, double* wn, double* red, int red_cap, unsigned* bar,
                        int* err, cudaStream_t st) {
  arnoldi_step32(M, V, ld, j, H, ldh, wn, red, red_cap, bar, err, st);
}

// Barrier words (words 0 and 32) and error flag (word 48) of the
// cooperative pre-pass kernels: a 256-byte device block of the handle.
unsigned* prepass_barrier(sg_handle* h) {
  if (!h->sync) {
    SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->sync), 256));
    SG_CUDA(cudaMemset(h->sync, 0, 256));
  }
  return h->sync;
}
int* prepass_error(sg_handle* h) { return reinterpret_cast<int*>(prepass_barrier(h) + 48); }

template <typename T>
void enqueue_prepass(sg_handle* h, const DevCsr& M, const T* q, int k,
                     cudaStream_t st) {
  using B = Basis<T>;
  const int64_t n = M.n, ld = h->ld;
  T* V = B::V(h);
  Slots sl = slots_for(h->ws_m, h->ws_k);
  double* Hd = h->small + sl.H;
  double* wn = h->small + sl.wn;
  const int ldh = k + 1;
  SG_CUDA(cudaMemsetAsync(Hd, 0, sizeof(double) * ldh * k, st));
  SG_CUDA(cudaMemsetAsync(prepass_barrier(h), 0, 256, st));
  SG_CUDA(cudaMemcpyAsync(V, q, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
  for (int j = 0; j < k; ++j)
    step_kernel<T>(M, V, ld, j, Hd, ldh, wn, h->red, red_doubles(),
                   prepass_barrier(h), prepass_error(h), st);
}

// Ritz pre-pass: k steps of MGS-Arnoldi from q (device, unit norm) with
// the basis in V's columns (Sec. 3.4), one cooperative kernel per step.
// The k launches are captured once into a CUDA graph on the handle's own
// stream and replayed (ordered after/before `st` with events); if capture
// is not possible the kernels are launched directly.  Returns the steps completed and fills
// Hh ((k+1) x k, host, ld k+1).
template <typename T>
int arnoldi_prepass(sg_handle* h, const DevCsr& M, const T* q, int k,
                    cudaStream_t st, std::vector<double>& Hh) {
  using B = Basis<T>;
  const void* vals = sizeof(T) == 8 ? static_cast<const void*>(M.sptr ? M.sval : M.val)
                                     : static_cast<const void*>(M.sptr ? M.sval32 : M.val32);
  const void* key[6] = {M.sptr ? static_cast<const void*>(M.sptr) : M.rowptr, vals, q,
                        B::V(h), h->small, h->red};
  prepass_barrier(h);  // allocate the barrier block before any capture
  sg_handle::PrepassGraph* g = nullptr;
  for (auto& c : h->graphs)
    if (c.k == k && c.n == M.n && std::equal(key, key + 6, c.key)) g = &c;
  if (!g) {
    sg_handle::PrepassGraph ng;
    std::copy(key, key + 6, ng.key);
    ng.k = k;
    ng.n = M.n;
    cudaGraph_t graph = nullptr;
    const long long before = launches_so_far();
    bool ok = cudaStreamBeginCapture(h->own, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      try {
        enqueue_prepass<T>(h, M, q, k, h->own);
      } catch (...) {
        ok = false;
      }
      ok = (cudaStreamEndCapture(h->own, &graph) == cudaSuccess) && ok && graph;
    }
    ng.kernels = launches_so_far() - before;
    count_launches(-ng.kernels);  // captured, not launched
    if (ok && cudaGraphInstantiate(&ng.exec, graph, 0) != cudaSuccess) ok = false;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();  // clear the error a failed capture leaves behind
    if (ok) {
      h->graphs.push_back(ng);
      g = &h->graphs.back();
    }
  }
  if (g) {
    SG_CUDA(cudaEventRecord(h->ev[3], st));
    SG_CUDA(cudaStreamWaitEvent(h->own, h->ev[3], 0));
    SG_CUDA(cudaGraphLaunch(g->exec, h->own));
    count_launches(g->kernels);
    SG_CUDA(cudaEventRecord(h->ev[3], h->own));
    SG_CUDA(cudaStreamWaitEvent(st, h->ev[3], 0));
  } else {
    enqueue_prepass<T>(h, M, q, k, st);
  }
  Slots sl = slots_for(h->ws_m, h->ws_k);
  const int ldh = k + 1;
  Hh.assign(static_cast<size_t>(ldh) * k, 0.0);
  std::vector<double> wnh(k);
  SG_CUDA(cudaMemcpyAsync(h->hbuf, h->small + sl.H, sizeof(double) * ldh * k,
                          cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaMemcpyAsync(h->hbuf + ldh * k, h->small + sl.wn, sizeof(double) * k,
                          cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaMemcpyAsync(h->hbuf + ldh * k + k, prepass_error(h), sizeof(int),
                          cudaMemcpyDeviceToHost, st));
  SG_CUDA(cudaStreamSynchronize(st));
  int flag = 0;
  std::memcpy(&flag, h->hbuf + ldh * k + k, sizeof(int));
  if (flag != 0)
    throw Error(SG_ECUDA, "Ritz pre-pass: a grid barrier wait ran out");
  std::memcpy(Hh.data(), h->hbuf, sizeof(double) * ldh * k);
  std::memcpy(wnh.data(), h->hbuf + ldh * k, sizeof(double) * k);
  for (int j = 0; j < k; ++j) {
    const double sub = Hh[(j + 1) + static_cast<size_t>(j) * ldh];
    if (!(sub > 1e-12 * wnh[j]) || !std::isfinite(sub)) return j + 1;
  }
  return k;
}

struct Shifts {
  std::vector<double> re, im, gamma;
  std::vector<BasisStep> steps;
};

Shifts shifts_from_values(const std::vector<double>& re, const std::vector<double>& im,
                          int steps, int basis, int equil);

Shifts make_shifts(const std::vector<double>& Hh, int ldh, int steps,
                   int basis, int equil) {
  std::vector<double> re(steps), im(steps);
  if (hessenberg_eigvals(Hh.data(), ldh, steps, re.data(), im.data()) != 0)
    throw Error(SG_ENUMERIC, "Ritz values: QR iteration did not converge");
  for (int t = 0; t < steps; ++t)
    if (!std::isfinite(re[t]) || !std::isfinite(im[t]))
      throw Error(SG_ENUMERIC, "Ritz values: non-finite");
  return shifts_from_values(re, im, steps, basis, equil);
}

// Leja order, scaling coefficients and basis parameters of the Ritz values
// (Sec. 3.4), from the pre-pass or supplied by the caller.
Shifts shifts_from_values(const std::vector<double>& re, const std::vector<double>& im,
                          int steps, int basis, int equil) {
  Shifts sh;
  sh.re.resize(steps);
  sh.im.resize(steps);
  leja_order(steps, re.data(), im.data(), sh.re.data(), sh.im.data());
  sh.gamma.resize(steps);
  scaling_coefficients(steps, sh.re.data(), sh.im.data(), sh.gamma.data());
  std::vector<double> th_re(sh.re), th_im(sh.im), gm(sh.gamma);
  if (basis == SG_BASIS_MONOMIAL) {
    std::fill(th_re.begin(), th_re.end(), 0.0);
    std::fill(th_im.begin(), th_im.end(), 0.0);
    std::fill(gm.begin(), gm.end(), 1.0);
  } else if (basis == SG_BASIS_NEWTON) {
    std::fill(gm.begin(), gm.end(), 1.0);
  }
  if (equil == SG_EQUIL_SCALAR && basis != SG_BASIS_SCALED_NEWTON) {
    // A' = A / alpha (Eq. equil): the basis of A' is the basis of A with
    // the constant scaling coefficient alpha = max |theta| (Sec. 4.3);
    // the scaled Newton coefficients are relative and do not change
    double alpha = 0.0;
    for (int t = 0; t < steps; ++t) alpha = std::max(alpha, std::hypot(sh.re[t], sh.im[t]));
    if (alpha > 0.0) std::fill(gm.begin(), gm.end(), alpha);
  }
  basis_steps(steps, th_re.data(), th_im.data(), gm.data(), sh.steps);
  return sh;
}

// -------------------------------------------------------------------------
// Alg. 4 with restarts.  T is the storage/arithmetic of the Krylov basis;
// x, r and b are always FP64 (xvec, rvec, bvec), so with T = float every
// cycle restarts from an FP64 residual: one iterative-refinement step per
// cycle.  cycle_tol > 0 ends a cycle once the implicit residual has
// dropped by that factor relative to the cycle's own start.
// cycle_tol > 0: a cycle also ends once its implicit residual has dropped
// by that factor (the inner solve of a refinement step).  stall > 0: the
// solve stops (log.stalled) when a cycle's true residual is above `stall`
// times the one two cycles earlier.  first_max > 0: the solve also stops
// (log.stalled) when the first cycle leaves a true residual above
// first_max times the initial one.
template <typename T>
void solve_impl(sg_handle* h, const DevCsr& M, const SolveOpts& o,
                double cycle_tol, double stall, cudaStream_t st, SolveLog& log,
                double first_max = 0.0) {
  using B = Basis<T>;
  const double t0 = now_ms();
  const int64_t n = M.n;
  const int m = o.m;
  const int kritz = std::min(o.s > 0 ? o.s : o.s_max, m);
  const int64_t ld = h->ld;
  T* Qb = B::Q(h);
  T* Vb = B::V(h);
  T* Yb = B::Y(h);
  Slots sl = slots_for(h->ws_m, h->ws_k);
  double* Wd = h->small + sl.W;
  double* Gd = h->small + sl.G;
  double* Zd = h->small + sl.Z;
  double* yd = h->small + sl.Y;
  double* sc = h->small + sl.scal;
  double* hb = h->hbuf;
  const int max_iters = o.max_iters > 0 ? o.max_iters : 50 * m;

  auto device_norm = [&](const double* v, double* slot) {
    dot_partials(n, v, v, h->red, st);
    finish_sum(h->red, slot, true, st);
  };
  auto fetch = [&](const double* src, int64_t count, double* dst) {
    SG_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
  };

  // r = b - A x0, beta0 (Alg. 4, first line)
  residual(M, h->bvec, h->xvec, h->rvec, st);
  device_norm(h->rvec, sc);
  fetch(sc, 1, hb);
  SG_CUDA(cudaStreamSynchronize(st));
  const double beta0 = hb[0];
  log = SolveLog();
  if (!std::isfinite(beta0)) throw Error(SG_ENUMERIC, "non-finite initial residual");
  if (beta0 == 0.0) {
    log.converged = true;
    log.t_total = now_ms() - t0;
    return;
  }
  double beta = beta0;
  Shifts sh;
  bool have_shifts = false;
  int cur_s = 0;
  int total = 0;
  std::vector<double> Hh(static_cast<size_t>(m + 1) * m);
  const int ldH = m + 1;
  Givens gv;
  const size_t kk2 = static_cast<size_t>(h->ws_k + 1) * (h->ws_k + 1);
  std::vector<double> Wh, Gh, Zinv(kk2), Z1(kk2), Rph, R2(kk2), Rtop, Rkk, Bm, yv;

  for (;;) {
    // Q_1 = r / beta
    B::from_f64(n, h->rvec, Qb, 1.0 / beta, st);
    if (!have_shifts) {
      const double tp = now_ms();
      int steps = 0;
      if (o.n_ritz > 0) {
        steps = o.n_ritz;
        sh = shifts_from_values(std::vector<double>(o.ritz_re, o.ritz_re + steps),
                                std::vector<double>(o.ritz_im, o.ritz_im + steps), steps,
                                o.basis, o.equil);
      } else {
        std::vector<double> Hp;
        steps = arnoldi_prepass<T>(h, M, Qb, kritz, st, Hp);
        sh = make_shifts(Hp, kritz + 1, steps, o.basis, o.equil);
      }
      if (o.s > 0) {
        cur_s = std::min(o.s, steps);
      } else {
        cur_s = estimate_step(steps, sh.re.data(), sh.im.data(), o.eps,
                              o.omega_est, o.s_min, std::min(o.s_max, steps),
                              nullptr);
        cur_s = std::min(cur_s, steps);
      }
      cur_s = std::max(cur_s, 1);
      log.s0 = cur_s;
      log.ritz_re = sh.re;
      log.ritz_im = sh.im;
      log.gamma = sh.gamma;
      have_shifts = true;
      log.t_prepass += now_ms() - tp;
    }
    std::fill(Hh.begin(), Hh.end(), 0.0);
    gv.reset(m, beta);
    int i = 1, jdone = 0;
    bool stop_cycle = false;
    while (i <= m && !stop_cycle) {
      const int s_eff = std::min(cur_s, m + 1 - i);
      const T* qi = Qb + static_cast<int64_t>(i - 1) * ld;
      SG_CUDA(cudaEventRecord(h->ev[0], st));
      // matrix powers kernel (Sec. 2): V[:, j+1] from V[:, j] (V[:,0] = Q_i)
      for (int j = 0; j < s_eff; ++j) {
        const T* src = (j == 0) ? qi : Vb + static_cast<int64_t>(j) * ld;
        const T* zsrc = nullptr;
        if (sh.steps[j].c != 0.0)
          zsrc = (j == 1) ? qi : Vb + static_cast<int64_t>(j - 1) * ld;
        B::spmv(M, src, zsrc, Vb + static_cast<int64_t>(j + 1) * ld,
                sh.steps[j].theta, sh.steps[j].c, sh.steps[j].gamma, st);
      }
      SG_CUDA(cudaEventRecord(h->ev[1], st));
      T* X = Vb + ld;
      // first BCGS: W = Q^T X; X -= Q W; G = X^T X
      B::bdot(n, Qb, ld, i, X, ld, s_eff, Wd, i, false, h->part, h->part_cap, st);
      B::bupd(h, n, Qb, ld, i, Wd, i, X, ld, s_eff, -1.0, 1.0, false, st);
      B::bdot(n, X, ld, s_eff, X, ld, s_eff, Gd, s_eff, true, h->part, h->part_cap, st);
      fetch(Wd, static_cast<int64_t>(i) * s_eff, hb);
      fetch(Gd, static_cast<int64_t>(s_eff) * s_eff, hb + static_cast<int64_t>(i) * s_eff);
      SG_CUDA(cudaEventRecord(h->ev[2], st));
      SG_CUDA(cudaStreamSynchronize(st));
      if (sizeof(T) == 4) { tc_check_error(st); tc_update_check_error(st); oz_check_error(st); }
      else oz_check_error(st);
      {
        float a = 0, b = 0;
        cudaEventElapsedTime(&a, h->ev[0], h->ev[1]);
        cudaEventElapsedTime(&b, h->ev[1], h->ev[2]);
        log.t_mpk += a;
        log.t_ortho += b;
      }
      const double th0 = now_ms();
      Wh.assign(hb, hb + static_cast<int64_t>(i) * s_eff);
      Gh.assign(hb + static_cast<int64_t>(i) * s_eff,
                hb + static_cast<int64_t>(i) * s_eff + static_cast<int64_t>(s_eff) * s_eff);
      for (double v : Gh)
        if (!std::isfinite(v)) throw Error(SG_ENUMERIC, "non-finite Gram matrix");
      // first partial CholQR (Alg. 3)
      const int ldr = s_eff;
      Z1.assign(static_cast<size_t>(s_eff) * s_eff, 0.0);
      const int p1 = partial_cholesky(Gh.data(), s_eff, s_eff, o.omega, Z1.data(), ldr, nullptr);
      int q = 0;
      bool breakdown = false;
      Rtop.clear();
      Rkk.clear();
      log.s_eff_hist.push_back(s_eff);
      log.p1_hist.push_back(p1);
      log.t_host += now_ms() - th0;
      if (p1 == 0) {
        breakdown = true;
        q = 1;
        Rtop.assign(Wh.begin(), Wh.begin() + i);
        Rkk.assign(1, 0.0);
      } else {
        upper_inverse(Z1.data(), ldr, p1, Zinv.data(), p1);
        // H2D staging uses its own pinned slot: the D2H slots may be
        // refilled before this copy has run
        std::memcpy(hb + sl.Z, Zinv.data(), sizeof(double) * p1 * p1);
        SG_CUDA(cudaMemcpyAsync(Zd, hb + sl.Z, sizeof(double) * p1 * p1, cudaMemcpyHostToDevice, st));
        SG_CUDA(cudaEventRecord(h->ev[1], st));
        // Q_k = X(:, 1:p) Z^-1, then second BCGS and the second Gram
        B::bupd(h, n, X, ld, p1, Zd, p1, Yb, ld, p1, 1.0, 0.0, true, st);
        B::bdot(n, Qb, ld, i, Yb, ld, p1, Wd, i, false, h->part, h->part_cap, st);
        B::bupd(h, n, Qb, ld, i, Wd, i, Yb, ld, p1, -1.0, 1.0, false, st);
        // Gram of the block the first pass already orthonormalised: FP64
        // uses the symmetric kernel; the FP32 basis needs only FP32-level
        // accuracy here (its condition number is ~1), so it goes to the
        // tensor-core kernel like the projections
        B::bdot(n, Yb, ld, p1, Yb, ld, p1, Gd, p1, sizeof(T) == 8, h->part, h->part_cap, st);
        fetch(Wd, static_cast<int64_t>(i) * p1, hb);
        fetch(Gd, static_cast<int64_t>(p1) * p1, hb + static_cast<int64_t>(i) * p1);
        SG_CUDA(cudaEventRecord(h->ev[2], st));
        SG_CUDA(cudaStreamSynchronize(st));
        if (sizeof(T) == 4) { tc_check_error(st); tc_update_check_error(st); oz_check_error(st); }
        else oz_check_error(st);
        {
          float b = 0;
          cudaEventElapsedTime(&b, h->ev[1], h->ev[2]);
          log.t_ortho += b;
        }
        const double th1 = now_ms();
        Rph.assign(hb, hb + static_cast<int64_t>(i) * p1);
        Gh.assign(hb + static_cast<int64_t>(i) * p1,
                  hb + static_cast<int64_t>(i) * p1 + static_cast<int64_t>(p1) * p1);
        for (double v : Gh)
          if (!std::isfinite(v)) throw Error(SG_ENUMERIC, "non-finite Gram matrix");
        R2.assign(static_cast<size_t>(p1) * p1, 0.0);
        const int p2 = partial_cholesky(Gh.data(), p1, p1, o.omega, R2.data(), p1, nullptr);
        if (p2 == 0) {
          breakdown = true;
          q = 1;
          Rtop.resize(i);
          for (int r = 0; r < i; ++r) Rtop[r] = Wh[r] + Rph[r] * Z1[0];
          Rkk.assign(1, 0.0);
          log.t_host += now_ms() - th1;
        } else {
          q = p2;
          // R_top = W(:, 1:q) + R'(:, 1:q) Z(1:q, 1:q); R_kk = Z~ Z(1:q, 1:q)
          Rtop.assign(static_cast<size_t>(i) * q, 0.0);
          Rkk.assign(static_cast<size_t>(q) * q, 0.0);
          combine_r(i, q, Wh.data(), i, Rph.data(), i, Z1.data(), ldr, R2.data(), p1,
                    Rtop.data(), i, Rkk.data(), q);
          upper_inverse(R2.data(), p1, q, Zinv.data(), q);
          std::memcpy(hb + sl.Z, Zinv.data(), sizeof(double) * q * q);
          log.t_host += now_ms() - th1;
          SG_CUDA(cudaMemcpyAsync(Zd, hb + sl.Z, sizeof(double) * q * q, cudaMemcpyHostToDevice, st));
          // Q_k = Q_k(:, 1:q) Z~^-1 into Q's next columns
          B::bupd(h, n, Yb, ld, q, Zd, q, Qb + static_cast<int64_t>(i) * ld, ld, q,
                  1.0, 0.0, true, st);
        }
      }
      const double th2 = now_ms();
      // Hessenberg columns, Givens rotations, convergence check
      Bm.assign(static_cast<size_t>(q + 1) * q, 0.0);
      {
        std::vector<BasisStep> stq(sh.steps.begin(), sh.steps.begin() + q);
        change_of_basis(stq, q, Bm.data(), q + 1);
      }
      assemble_hessenberg(Hh.data(), ldH, i, q, Rtop.data(), i, Rkk.data(), q, Bm.data(), q + 1);
      log.s_hist.push_back(breakdown ? 0 : q);
      for (int c = 0; c < q; ++c) {
        const int j = i - 1 + c;
        const double gj = gv.add_column(Hh.data(), ldH, j);
        const double rel = gj / beta0;
        if (!std::isfinite(rel)) throw Error(SG_ENUMERIC, "non-finite residual estimate");
        log.relres_hist.push_back(rel);
        jdone = j + 1;
        if (rel <= o.tol || breakdown || (cycle_tol > 0.0 && gj <= cycle_tol * beta)) {
          stop_cycle = true;
          break;
        }
      }
      if (!breakdown && q < s_eff) cur_s = q;  // Alg. 4: s = p
      i += q;
      if (total + jdone >= max_iters) stop_cycle = true;
      log.t_host += now_ms() - th2;
    }
    // end of cycle: y from the triangular least-squares problem, x += Q y
    yv.assign(jdone, 0.0);
    gv.solve(jdone, yv.data());
    std::memcpy(hb + sl.Y, yv.data(), sizeof(double) * jdone);
    SG_CUDA(cudaMemcpyAsync(yd, hb + sl.Y, sizeof(double) * jdone, cudaMemcpyHostToDevice, st));
    B::gemv(n, jdone, Qb, ld, yd, h->xvec, st);
    residual(M, h->bvec, h->xvec, h->rvec, st);
    device_norm(h->rvec, sc);
    fetch(sc, 1, hb);
    SG_CUDA(cudaStreamSynchronize(st));
    beta = hb[0];
    total += jdone;
    const double rel_true = beta / beta0;
    log.cycle_relres.push_back(rel_true);
    log.cycle_iters.push_back(jdone);
    if (!std::isfinite(rel_true)) throw Error(SG_ENUMERIC, "non-finite residual");
    if (rel_true <= o.tol) {
      log.converged = true;
      break;
    }
    if (total >= max_iters) break;
    if (beta == 0.0) { log.converged = true; break; }
    const size_t nc = log.cycle_relres.size();
    if (stall > 0.0 && nc >= 3 && rel_true > stall * log.cycle_relres[nc - 3]) {
      log.stalled = true;
      break;
    }
    if (first_max > 0.0 && nc == 1 && rel_true > first_max) {
      log.stalled = true;
      break;
    }
  }
  log.iters = total;
  log.restarts = static_cast<int>(log.cycle_relres.size()) - 1;
  log.final_relres = log.cycle_relres.back();
  log.t_total = now_ms() - t0;
}

}  // namespace

int ritz_prepass(sg_handle* h, const DevCsr& M, const double* q, int k, bool fp32,
                 cudaStream_t st, std::vector<double>& H) {
  const int64_t n = M.n;
  if (fp32) {
    ensure_workspace32(h, n, k, k);
    to_f32(n, q, h->Q32, 1.0f, st);
    return arnoldi_prepass<float>(h, M, h->Q32, k, st, H);
  }
  ensure_workspace(h, n, k, k);
  SG_CUDA(cudaMemcpyAsync(h->Q, q, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  return arnoldi_prepass<double>(h, M, h->Q, k, st, H);
}

void solve_fp64(sg_handle* h, const DevCsr& M, const SolveOpts& o,
                cudaStream_t st, SolveLog& log) {
  const int kritz = std::min(o.s > 0 ? o.s : o.s_max, o.m);
  ensure_workspace(h, M.n, o.m, std::max(kritz, 1));
  solve_impl<double>(h, M, o, 0.0, 0.0, st, log);
}

void solve_fp32_ir(sg_handle* h, const DevCsr& M, const SolveOpts& o,
                   double inner_tol, int max_refine, cudaStream_t st,
                   SolveLog& log) {
  const int kritz = std::min(o.s > 0 ? o.s : o.s_max, o.m);
  ensure_workspace32(h, M.n, o.m, std::max(kritz, 1));
  SolveOpts o32 = o;
  // Bounds of the FP32 basis.  The paper's rule Omega ~ 0.1 eps^-1/2
  // (Sec. 3.2) is set by the accuracy of the Gram matrix the Cholesky
  // factor comes from; the FP32 Gram matrices here are formed from exact
  // products with compensated sums (relative accuracy ~2^-40 after the
  // split reduction), so Omega_32 = 0.1 (2^-40)^-1/2 = 0.1 2^20.  That also
  // keeps the FP32 triangular product's orthogonality loss eps_32 Omega
  // below 1e-2, which the second CholQR pass removes.  The estimator uses
  // the basis round-off eps_32 = 2^-24 and the same threshold.
  const double omega32 = 0.1 * std::ldexp(1.0, 20);
  o32.eps = std::ldexp(1.0, -24);
  o32.omega = std::min(o.omega, omega32);
  o32.omega_est = std::min(o.omega_est, omega32);
  o32.max_iters = o.max_iters > 0 ? o.max_iters : max_refine * o.m;
  // Refinement with an FP32 inner solve contracts the residual by about
  // max(inner_tol, kappa(A) eps_32) per step, and only while kappa(A)
  // eps_32 < 1.  So the remaining iterations run with the FP64 basis (same
  // method, the FP32 pre-pass's Ritz values) when
  //  - the first refinement step leaves more than 10 inner_tol of the
  //    initial residual: kappa(A) eps_32 is what limits it, and the FP64
  //    solve starts afresh from x0 (on the 192^3 diffusion system it needs
  //    8,891 columns from the FP32 iterate, 7,603 from x0), or
  //  - two refinement steps together fail to halve the true residual: the
  //    FP64 solve continues from the current x;
  // the solve then still reaches tol whenever the FP64 solve does.
  const int64_t n = M.n;
  if (!h->x0vec || h->x0_n != n) {
    dev_alloc(&h->x0vec, static_cast<size_t>(n));
    h->x0_n = n;
  }
  SG_CUDA(cudaMemcpyAsync(h->x0vec, h->xvec, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  solve_impl<float>(h, M, o32, inner_tol, 0.5, st, log, 10.0 * inner_tol);
  log.refinements = static_cast<int>(log.cycle_relres.size());
  const int left = o32.max_iters - log.iters;
  if (log.converged || !log.stalled || left <= 0) return;
  const bool afresh = log.refinements == 1;
  const double scale = afresh ? 1.0 : log.final_relres;  // residual now / initial residual
  if (!(scale > 0.0)) return;
  if (afresh)
    SG_CUDA(cudaMemcpyAsync(h->xvec, h->x0vec, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  const int kritz64 = std::min(o.s > 0 ? o.s : o.s_max, o.m);
  ensure_workspace(h, M.n, o.m, std::max(kritz64, 1));
  SolveOpts o64 = o;
  o64.tol = o.tol / scale;
  o64.max_iters = left;
  if (o64.n_ritz == 0 && !log.ritz_re.empty()) {   // no second pre-pass
    o64.n_ritz = static_cast<int>(log.ritz_re.size());
    o64.ritz_re = log.ritz_re.data();
    o64.ritz_im = log.ritz_im.data();
  }
  SolveLog l64;
  solve_impl<double>(h, M, o64, 0.0, 0.0, st, l64);
  for (double r : l64.relres_hist) log.relres_hist.push_back(r * scale);
  for (double r : l64.cycle_relres) log.cycle_relres.push_back(r * scale);
  log.cycle_iters.insert(log.cycle_iters.end(), l64.cycle_iters.begin(), l64.cycle_iters.end());
  log.s_eff_hist.insert(log.s_eff_hist.end(), l64.s_eff_hist.begin(), l64.s_eff_hist.end());
  log.p1_hist.insert(log.p1_hist.end(), l64.p1_hist.begin(), l64.p1_hist.end());
  log.s_hist.insert(log.s_hist.end(), l64.s_hist.begin(), l64.s_hist.end());
  log.iters += l64.iters;
  log.fp64_iters = l64.iters;
  log.restarts = static_cast<int>(log.cycle_relres.size()) - 1;
  log.converged = l64.converged;
  log.final_relres = l64.final_relres * scale;
  log.t_prepass += l64.t_prepass;
  log.t_mpk += l64.t_mpk;
  log.t_ortho += l64.t_ortho;
  log.t_host += l64.t_host;
  log.t_total += l64.t_total;
}

}  // namespace sg
