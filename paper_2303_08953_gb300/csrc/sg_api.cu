// extern "C" boundary of the library (declared in include/sgmres.h).
// Every entry point catches the internal sg::Error / CUDA failures and
// returns a status; the message is kept in the handle.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "sg_solver.h"

using sg::Error;

namespace sg {
namespace {
std::atomic<long long> g_launches{0};
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(); }
}  // namespace sg

namespace {

sg_status fail(sg_handle* h, sg_status code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

template <typename F>
sg_status guarded(sg_handle* h, F&& f) {
  try {
    if (h) h->err.clear();
    f();
    return SG_OK;
  } catch (const Error& e) {
    return fail(h, e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(h, SG_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(h, SG_EINVAL, e.what());
  }
}

cudaStream_t pick(sg_handle* h, void* s) {
  return s ? static_cast<cudaStream_t>(s) : h->own;
}

void free_csr(sg::DevCsr& A) {
  if (A.rowptr) cudaFree(A.rowptr);
  if (A.colind) cudaFree(A.colind);
  if (A.val) cudaFree(A.val);
  if (A.val32) cudaFree(A.val32);
  if (A.sptr) cudaFree(A.sptr);
  if (A.scol) cudaFree(A.scol);
  if (A.sval) cudaFree(A.sval);
  if (A.sval32) cudaFree(A.sval32);
  if (A.sbase) cudaFree(A.sbase);
  if (A.soff) cudaFree(A.soff);
  A = sg::DevCsr();
}

__global__ void f64_to_f32_kernel(int64_t n, const double* x, float* y) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    y[i] = static_cast<float>(x[i]);
}

// FP32 copies of the values (CSR and, when present, SELL-32)
void make_val32(sg::DevCsr& A, cudaStream_t st) {
  if (A.val32) cudaFree(A.val32);
  A.val32 = nullptr;
  if (A.sval32) cudaFree(A.sval32);
  A.sval32 = nullptr;
  SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&A.val32), sizeof(float) * std::max<int64_t>(A.nnz, 1)));
  f64_to_f32_kernel<<<sg::device_sm_count() * 8, 256, 0, st>>>(A.nnz, A.val, A.val32);
  SG_LAUNCH_CHECK();
  if (A.sptr) {
    SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&A.sval32), sizeof(float) * A.sell_nnz));
    f64_to_f32_kernel<<<sg::device_sm_count() * 8, 256, 0, st>>>(A.sell_nnz, A.sval, A.sval32);
    SG_LAUNCH_CHECK();
  }
}

sg::SolveOpts to_internal(const sg_opts* o) {
  sg::SolveOpts s;
  s.m = o->m;
  s.s = o->s;
  s.s_min = std::max(1, o->s_min);
  s.s_max = o->s_max > 0 ? o->s_max : o->m;
  s.max_iters = o->max_iters;
  s.basis = o->basis;
  s.tol = o->tol;
  s.omega = o->omega;
  s.omega_est = o->omega_est;
  s.eps = std::ldexp(1.0, -53);
  s.equil = o->equilibrate;
  s.n_ritz = o->n_ritz;
  s.ritz_re = o->ritz_re;
  s.ritz_im = o->ritz_im;
  return s;
}

void check_opts(const sg_opts* o) {
  SG_REQUIRE(o, SG_EINVAL, "opts is NULL");
  SG_REQUIRE(o->m >= 1, SG_EINVAL, "m must be >= 1");
  SG_REQUIRE(o->s >= 0, SG_EINVAL, "s must be >= 0");
  SG_REQUIRE(o->s > 0 || o->s_max >= 1 || o->m >= 1, SG_EINVAL, "bad s_max");
  SG_REQUIRE(o->tol >= 0.0, SG_EINVAL, "tol must be >= 0");
  SG_REQUIRE(o->omega > 1.0 && o->omega_est > 0.0, SG_EINVAL, "bad omega");
  SG_REQUIRE(o->basis >= 0 && o->basis <= 2, SG_EINVAL, "bad basis");
  SG_REQUIRE(o->precision == SG_PREC_FP64 || o->precision == SG_PREC_FP32_IR,
             SG_EINVAL, "bad precision");
  SG_REQUIRE(o->equilibrate >= SG_EQUIL_NONE && o->equilibrate <= SG_EQUIL_COLUMN,
             SG_EINVAL, "bad equilibrate");
  SG_REQUIRE(o->n_ritz >= 0, SG_EINVAL, "n_ritz must be >= 0");
  if (o->n_ritz > 0) {
    SG_REQUIRE(o->ritz_re && o->ritz_im, SG_EINVAL, "n_ritz > 0 needs ritz_re and ritz_im");
    int pos = 0, neg = 0;
    for (int t = 0; t < o->n_ritz; ++t) {
      SG_REQUIRE(std::isfinite(o->ritz_re[t]) && std::isfinite(o->ritz_im[t]), SG_EINVAL,
                 "non-finite Ritz value");
      if (o->ritz_im[t] > 0.0) {
        ++pos;
        bool found = false;
        for (int u = 0; u < o->n_ritz && !found; ++u)
          found = o->ritz_re[u] == o->ritz_re[t] && o->ritz_im[u] == -o->ritz_im[t];
        SG_REQUIRE(found, SG_EINVAL, "a complex Ritz value without its conjugate");
      } else if (o->ritz_im[t] < 0.0) {
        ++neg;
      }
    }
    SG_REQUIRE(pos == neg, SG_EINVAL, "unpaired complex Ritz values");
  }
}

template <typename T>
void copy_in(T* dst, const T* src, int64_t n, bool on_device, cudaStream_t st) {
  SG_CUDA(cudaMemcpyAsync(dst, src, sizeof(T) * n,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
}

void fill_result(const sg::SolveLog& L, sg_result* r) {
  if (!r) return;
  r->converged = L.converged ? 1 : 0;
  r->s0 = L.s0;
  r->iters = L.iters;
  r->restarts = L.restarts;
  r->refinements = L.refinements;
  r->final_relres = L.final_relres;
  auto put = [](auto* dst, int cap, const auto& v) {
    if (!dst) return;
    const int k = std::min<int>(cap, static_cast<int>(v.size()));
    for (int t = 0; t < k; ++t) dst[t] = v[t];
  };
  r->n_hist = static_cast<int32_t>(L.relres_hist.size());
  put(r->relres_hist, r->hist_cap, L.relres_hist);
  r->n_blocks = static_cast<int32_t>(L.s_hist.size());
  put(r->s_eff_hist, r->blocks_cap, L.s_eff_hist);
  put(r->p1_hist, r->blocks_cap, L.p1_hist);
  put(r->s_hist, r->blocks_cap, L.s_hist);
  r->n_cycles = static_cast<int32_t>(L.cycle_relres.size());
  put(r->cycle_relres, r->cycles_cap, L.cycle_relres);
  put(r->cycle_iters, r->cycles_cap, L.cycle_iters);
  r->n_ritz = static_cast<int32_t>(L.ritz_re.size());
  put(r->ritz_re, r->ritz_cap, L.ritz_re);
  put(r->ritz_im, r->ritz_cap, L.ritz_im);
  put(r->gamma, r->ritz_cap, L.gamma);
  r->t_prepass_ms = L.t_prepass;
  r->t_mpk_ms = L.t_mpk;
  r->t_ortho_ms = L.t_ortho;
  r->t_host_ms = L.t_host;
  r->t_total_ms = L.t_total;
  r->fp64_iters = L.fp64_iters;
}

// A^T on the device (built on first use; values follow A's)
void ensure_transpose(sg_handle* h, cudaStream_t st) {
  if (h->have_AT) return;
  h->AT.n = h->A.n;
  h->AT.nnz = h->A.nnz;
  SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->AT.rowptr), sizeof(int32_t) * (h->A.n + 1)));
  SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->AT.colind), sizeof(int32_t) * std::max<int64_t>(h->A.nnz, 1)));
  SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->AT.val), sizeof(double) * std::max<int64_t>(h->A.nnz, 1)));
  int32_t* counts = nullptr;
  SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&counts), sizeof(int32_t) * (h->A.n + 1)));
  try {
    sg::csr_transpose(h->A, h->AT, counts, st);
    SG_CUDA(cudaStreamSynchronize(st));
  } catch (...) {
    cudaFree(counts);
    throw;
  }
  cudaFree(counts);
  h->AT.mean_row = h->A.mean_row;
  sg::build_sell(h->AT, st);
  if (h->A.val32) make_val32(h->AT, st);
  h->have_AT = true;
}

// the column-equilibrated matrix A D_c (its own value arrays only)
void free_equil(sg_handle* h) {
  if (!h->have_AE && !h->dcol) return;
  h->drop_graphs();
  sg::DevCsr& E = h->AE;
  if (E.val) cudaFree(E.val);
  if (E.sval) cudaFree(E.sval);
  if (E.val32) cudaFree(E.val32);
  if (E.sval32) cudaFree(E.sval32);
  if (h->dcol) cudaFree(h->dcol);
  h->dcol = nullptr;
  E = sg::DevCsr();
  h->have_AE = false;
}

void ensure_equil(sg_handle* h, cudaStream_t st) {
  if (h->have_AE) return;
  ensure_transpose(h, st);
  try {
    SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->dcol), sizeof(double) * h->A.n));
    sg::column_scale_factors(h->AT, h->dcol, st);
    sg::DevCsr& E = h->AE;
    E = h->A;  // pattern arrays are shared with A
    E.val = E.sval = nullptr;
    E.val32 = E.sval32 = nullptr;
    SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&E.val), sizeof(double) * std::max<int64_t>(h->A.nnz, 1)));
    if (h->A.sptr)
      SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&E.sval), sizeof(double) * h->A.sell_nnz));
    sg::scale_columns(h->A, h->dcol, E, st);
    SG_CUDA(cudaStreamSynchronize(st));
    h->have_AE = true;
  } catch (...) {
    h->have_AE = true;  // let free_equil release what was allocated
    free_equil(h);
    throw;
  }
}

sg_status run_solve(sg_handle* h, bool adjoint, const double* b, double* x,
                    const sg_opts* opts, sg_result* res) {
  sg_status st_code = SG_OK;
  sg::SolveLog log;
  sg_status rc = guarded(h, [&] {
    SG_REQUIRE(h->have_A, SG_ESTATE, "no matrix: call sg_analyze first");
    SG_REQUIRE(!h->rows_only, SG_ESTATE, "a row block supports the kernel-level calls only");
    check_opts(opts);
    SG_REQUIRE(b && x, SG_EINVAL, "b/x is NULL");
    SG_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = pick(h, opts->stream);
    const sg::DevCsr* M = &h->A;
    const bool colscale = opts->equilibrate == SG_EQUIL_COLUMN;
    SG_REQUIRE(!(adjoint && colscale), SG_EINVAL,
               "column equilibration applies to forward solves only");
    if (adjoint) {
      ensure_transpose(h, st);
      M = &h->AT;
    } else if (colscale) {
      ensure_equil(h, st);
      M = &h->AE;
    }
    const int64_t n = M->n;
    sg::SolveOpts o = to_internal(opts);
    const int kritz = std::min(o.s > 0 ? o.s : o.s_max, o.m);
    sg::ensure_workspace(h, n, o.m, std::max(kritz, 1));
    const bool dev = opts->vectors_on_device != 0;
    copy_in(h->bvec, b, n, dev, st);
    copy_in(h->xvec, static_cast<const double*>(x), n, dev, st);
    if (colscale) sg::diag_apply(n, h->dcol, h->xvec, h->xvec, true, st);  // y0 = D_c^-1 x0
    if (opts->precision == SG_PREC_FP32_IR) {
      if (!M->val32) make_val32(*const_cast<sg::DevCsr*>(M), st);
      sg::solve_fp32_ir(h, *M, o, opts->inner_tol > 0 ? opts->inner_tol : 1e-4,
                        opts->max_refine > 0 ? opts->max_refine : 20, st, log);
    } else {
      sg::solve_fp64(h, *M, o, st, log);
    }
    if (colscale) sg::diag_apply(n, h->dcol, h->xvec, h->xvec, false, st);  // x = D_c y
    SG_CUDA(cudaMemcpyAsync(x, h->xvec, sizeof(double) * n,
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
    fill_result(log, res);
    if (!log.converged) st_code = SG_ENOCONV;
  });
  if (rc != SG_OK) return rc;
  if (st_code == SG_ENOCONV)
    return fail(h, SG_ENOCONV, "iteration cap reached before tol");
  return SG_OK;
}

}  // namespace

extern "C" {

int64_t sg_kernel_launches(void) { return sg::g_launches.load(); }

int32_t sg_set_tc_policy(int32_t policy) { return sg::set_tc_policy(policy); }

void sg_default_opts(sg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->m = 60;
  o->s = 10;
  o->s_min = 1;
  o->s_max = 0;
  o->tol = 1e-10;
  o->max_iters = 0;
  o->omega = 1e7;
  o->omega_est = 1e7;
  o->basis = SG_BASIS_SCALED_NEWTON;
  o->precision = SG_PREC_FP64;
  o->inner_tol = 1e-4;
  o->max_refine = 20;
  o->vectors_on_device = 0;
  o->stream = nullptr;
}

sg_status sg_create(int device, sg_handle** out) {
  if (!out) return SG_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return SG_ECUDA;
  sg_handle* h = new (std::nothrow) sg_handle();
  if (!h) return SG_ENOMEM;
  h->device = device;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return SG_ECUDA;
  }
  *out = h;
  return SG_OK;
}

void sg_destroy(sg_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->own) cudaStreamSynchronize(h->own);
  h->drop_graphs();
  free_equil(h);
  free_csr(h->A);
  free_csr(h->AT);
  double* d[] = {h->Q, h->V, h->Y, h->bvec, h->xvec, h->rvec, h->part, h->red, h->small, h->dvec,
                 h->x0vec};
  for (double* p : d) if (p) cudaFree(p);
  if (h->sync) cudaFree(h->sync);
  float* f[] = {h->Q32, h->V32, h->Y32, h->r32};
  for (float* p : f) if (p) cudaFree(p);
  if (h->hbuf) cudaFreeHost(h->hbuf);
  for (auto e : h->ev) if (e) cudaEventDestroy(e);
  if (h->own) cudaStreamDestroy(h->own);
  delete h;
}

const char* sg_last_error(const sg_handle* h) { return h ? h->err.c_str() : "null handle"; }

// Ingest of a square matrix (ncols = n, columns sorted in each row) or of
// a row block of a partitioned matrix (ncols >= n, columns distinct in each
// row but in the caller's order: local numbering of a halo block).
static sg_status analyze_impl(sg_handle* h, const sg_csr* A, int64_t ncols, bool block) {
  return guarded(h, [&] {
    SG_REQUIRE(A && A->rowptr && A->colind && A->val, SG_EINVAL, "null CSR array");
    SG_REQUIRE(A->n >= 1, SG_EINVAL, "n must be >= 1");
    SG_REQUIRE(A->nnz >= 0 && A->nnz < (int64_t(1) << 31), SG_EINVAL, "nnz out of int32 range");
    SG_REQUIRE(ncols >= A->n && ncols < (int64_t(1) << 31), SG_EINVAL,
               "ncols must be in [n, 2^31)");
    SG_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = h->own;
    const int64_t n = A->n, nnz = A->nnz;
    const bool dev = A->on_device != 0;
    int32_t maxrow = 0;
    if (block) {
      // a row block: columns distinct but unsorted (local numbering), checked
      // on the host (from a host copy when A is on the device)
      std::vector<int32_t> rp(n + 1), ci(nnz);
      const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
      SG_CUDA(cudaMemcpy(rp.data(), A->rowptr, sizeof(int32_t) * (n + 1), kind));
      if (nnz) SG_CUDA(cudaMemcpy(ci.data(), A->colind, sizeof(int32_t) * nnz, kind));
      SG_REQUIRE(rp[0] == 0 && rp[n] == nnz, SG_EINVAL, "rowptr must start at 0 and end at nnz");
      std::vector<int32_t> row;
      for (int64_t r = 0; r < n; ++r) {
        SG_REQUIRE(rp[r + 1] >= rp[r], SG_EINVAL, "rowptr not non-decreasing");
        maxrow = std::max(maxrow, rp[r + 1] - rp[r]);
        for (int32_t k = rp[r]; k < rp[r + 1]; ++k)
          SG_REQUIRE(ci[k] >= 0 && ci[k] < ncols, SG_EINVAL, "column index out of range");
        row.assign(ci.begin() + rp[r], ci.begin() + rp[r + 1]);
        std::sort(row.begin(), row.end());
        SG_REQUIRE(std::adjacent_find(row.begin(), row.end()) == row.end(), SG_EINVAL,
                   "repeated column in a row");
      }
    }
    // the device copy, installed only once it has passed its checks (a
    // rejected matrix leaves the handle's previous one in place)
    sg::DevCsr T;
    T.n = A->n;
    T.nnz = nnz;
    try {
      SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&T.rowptr), sizeof(int32_t) * (n + 1)));
      SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&T.colind), sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
      SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&T.val), sizeof(double) * std::max<int64_t>(nnz, 1)));
      copy_in(T.rowptr, A->rowptr, n + 1, dev, st);
      if (nnz) {
        copy_in(T.colind, A->colind, nnz, dev, st);
        copy_in(T.val, A->val, nnz, dev, st);
      }
      if (!block) {
        // a square matrix: sorted, in-range columns, checked on the device
        int flags = 0, longest = 0;
        sg::check_csr(T.rowptr, T.colind, n, nnz, ncols, &flags, &longest, st);
        SG_REQUIRE(!(flags & 1), SG_EINVAL, "rowptr must start at 0 and end at nnz");
        SG_REQUIRE(!(flags & 2), SG_EINVAL, "rowptr not non-decreasing");
        SG_REQUIRE(!(flags & 4), SG_EINVAL, "column index out of range");
        SG_REQUIRE(!(flags & 8), SG_EINVAL, "columns not sorted/unique in a row");
        maxrow = longest;
      }
    } catch (...) {
      free_csr(T);
      throw;
    }
    h->drop_graphs();
    free_equil(h);
    free_csr(h->A);
    free_csr(h->AT);
    h->have_A = h->have_AT = false;
    h->A = T;
    sg::DevCsr& D = h->A;
    D.mean_row = static_cast<double>(nnz) / static_cast<double>(n);
    D.max_row = maxrow;
    sg::build_sell(D, st);
    SG_CUDA(cudaStreamSynchronize(st));
    h->have_A = true;
    h->rows_only = block;
    h->ncols = ncols;
  });
}

sg_status sg_analyze(sg_handle* h, const sg_csr* A) {
  if (!h) return SG_EINVAL;
  return analyze_impl(h, A, A ? A->n : 0, false);
}

sg_status sg_analyze_rows(sg_handle* h, const sg_csr* A, int32_t ncols) {
  if (!h) return SG_EINVAL;
  return analyze_impl(h, A, ncols, true);
}

sg_status sg_gather(const int32_t* idx, int64_t count, const double* src, double* dst,
                    void* stream) {
  if (count < 0 || (count > 0 && (!idx || !src || !dst))) return SG_EINVAL;
  try {
    sg::gather(idx, count, src, dst, static_cast<cudaStream_t>(stream));
  } catch (const sg::Error& e) {
    return e.code;
  }
  return SG_OK;
}

sg_status sg_update_values(sg_handle* h, const double* val, int32_t on_device) {
  if (!h) return SG_EINVAL;
  return guarded(h, [&] {
    SG_REQUIRE(h->have_A, SG_ESTATE, "no matrix: call sg_analyze first");
    SG_REQUIRE(val || h->A.nnz == 0, SG_EINVAL, "val is NULL");
    SG_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = h->own;
    free_equil(h);  // the equilibrated values follow A's
    if (h->A.nnz) copy_in(h->A.val, val, h->A.nnz, on_device != 0, st);
    sg::sell_refill_values(h->A, st);
    if (h->A.val32) make_val32(h->A, st);
    if (h->have_AT) {  // values of the transpose are stale: rebuild lazily
      h->drop_graphs();
      free_csr(h->AT);
      h->have_AT = false;
    }
    SG_CUDA(cudaStreamSynchronize(st));
  });
}

sg_status sg_probe_bounded_waits(int32_t device, double limit_ms,
                                 int32_t* grid_barrier_timed_out,
                                 int32_t* mbarrier_timed_out) {
  if (!grid_barrier_timed_out || !mbarrier_timed_out) return SG_EINVAL;
  try {
    SG_CUDA(cudaSetDevice(device));
    const double ms = std::min(2000.0, std::max(1.0, limit_ms));
    const uint64_t ns = static_cast<uint64_t>(ms * 1e6);
    cudaStream_t st = nullptr;
    SG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    try {
      *grid_barrier_timed_out = sg::probe_grid_barrier_timeout(ns, st) ? 1 : 0;
      *mbarrier_timed_out = sg::probe_mbarrier_timeout(ns, st) ? 1 : 0;
    } catch (...) {
      cudaStreamDestroy(st);
      throw;
    }
    SG_CUDA(cudaStreamDestroy(st));
    return SG_OK;
  } catch (const sg::Error& e) {
    return e.code;
  } catch (...) {
    return SG_ECUDA;
  }
}

sg_status sg_matrix_info(const sg_handle* h, int32_t* sell, int64_t* stored) {
  if (!h) return SG_EINVAL;
  if (!h->have_A) return SG_ESTATE;
  if (sell) *sell = h->A.sptr ? 1 : 0;
  if (stored) *stored = h->A.sptr ? h->A.sell_nnz : h->A.nnz;
  return SG_OK;
}

sg_status sg_solve(sg_handle* h, const double* b, double* x,
                   const sg_opts* opts, sg_result* res) {
  if (!h) return SG_EINVAL;
  return run_solve(h, false, b, x, opts, res);
}

sg_status sg_solve_adjoint(sg_handle* h, const double* g, double* lam,
                           const sg_opts* opts, sg_result* res) {
  if (!h) return SG_EINVAL;
  return run_solve(h, true, g, lam, opts, res);
}

sg_status sg_grad_values(sg_handle* h, const double* lam, const double* x,
                         double* dval, void* stream) {
  if (!h) return SG_EINVAL;
  return guarded(h, [&] {
    SG_REQUIRE(h->have_A, SG_ESTATE, "no matrix");
    SG_REQUIRE(lam && x && dval, SG_EINVAL, "null pointer");
    SG_CUDA(cudaSetDevice(h->device));
    sg::sampled_outer(h->A, lam, x, dval, pick(h, stream));
  });
}

sg_status sg_spmv_newton(sg_handle* h, const double* x, const double* z,
                         double* y, double theta, double c, double gamma,
                         void* stream) {
  if (!h) return SG_EINVAL;
  return guarded(h, [&] {
    SG_REQUIRE(h->have_A, SG_ESTATE, "no matrix");
    SG_REQUIRE(x && y && (c == 0.0 || z), SG_EINVAL, "null pointer");
    SG_REQUIRE(gamma != 0.0, SG_EINVAL, "gamma must be nonzero");
    SG_CUDA(cudaSetDevice(h->device));
    sg::spmv_newton(h->A, x, z, y, theta, c, gamma, pick(h, stream));
  });
}

sg_status sg_residual(sg_handle* h, const double* b, const double* x,
                      double* r, void* stream) {
  if (!h) return SG_EINVAL;
  return guarded(h, [&] {
    SG_REQUIRE(h->have_A, SG_ESTATE, "no matrix");
    SG_REQUIRE(b && x && r, SG_EINVAL, "null pointer");
    SG_CUDA(cudaSetDevice(h->device));
    sg::residual(h->A, b, x, r, pick(h, stream));
  });
}

sg_status sg_mpk(sg_handle* h, const double* q, double* V, int64_t ldv,
                 int32_t s, const double* theta_re, const double* theta_im,
                 const double* gamma, void* stream) {
  if (!h) return SG_EINVAL;
  return guarded(h, [&] {
    SG_REQUIRE(h->have_A, SG_ESTATE, "no matrix");
    SG_REQUIRE(q && V && ldv >= h->A.n && s >= 0, SG_EINVAL, "bad MPK arguments");
    SG_REQUIRE(s == 0 || (theta_re && theta_im && gamma), SG_EINVAL, "null shifts");
    SG_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = pick(h, stream);
    std::vector<sg::BasisStep> steps;
    sg::basis_steps(s, theta_re, theta_im, gamma, steps);
    SG_CUDA(cudaMemcpyAsync(V, q, sizeof(double) * h->A.n, cudaMemcpyDeviceToDevice, st));
    for (int j = 0; j < s; ++j) {
      SG_REQUIRE(steps[j].gamma != 0.0, SG_EINVAL, "gamma must be nonzero");
      const double* z = steps[j].c != 0.0 ? V + static_cast<int64_t>(j - 1) * ldv : nullptr;
      sg::spmv_newton(h->A, V + static_cast<int64_t>(j) * ldv, z,
                      V + static_cast<int64_t>(j + 1) * ldv, steps[j].theta, steps[j].c,
                      steps[j].gamma, st);
    }
  });
}

sg_status sg_arnoldi(sg_handle* h, const double* q, int32_t k, int32_t precision,
                     double* H, int32_t ldh, int32_t* steps, void* stream) {
  if (!h) return SG_EINVAL;
  return guarded(h, [&] {
    SG_REQUIRE(h->have_A, SG_ESTATE, "no matrix");
    SG_REQUIRE(!h->rows_only, SG_ESTATE, "a row block supports the kernel-level calls only");
    SG_REQUIRE(q && H && steps && k >= 1 && ldh >= k + 1, SG_EINVAL, "bad Arnoldi arguments");
    SG_REQUIRE(precision == SG_PREC_FP64 || precision == SG_PREC_FP32_IR, SG_EINVAL,
               "unknown precision");
    SG_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = pick(h, stream);
    const bool fp32 = precision == SG_PREC_FP32_IR;
    if (fp32 && !h->A.val32) make_val32(h->A, st);
    std::vector<double> Hh;
    const int done = sg::ritz_prepass(h, h->A, q, k, fp32, st, Hh);
    for (int c = 0; c < k; ++c)
      for (int r = 0; r <= k; ++r)
        H[r + static_cast<int64_t>(c) * ldh] = Hh[r + static_cast<size_t>(c) * (k + 1)];
    *steps = done;
  });
}

namespace {
void ensure_part(sg_handle* h, int64_t need, cudaStream_t st) {
  if (need <= h->part_cap) return;
  SG_CUDA(cudaStreamSynchronize(st));
  if (h->part) cudaFree(h->part);
  h->part = nullptr;
  h->part_cap = 0;
  SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->part), sizeof(double) * need));
  h->part_cap = need;
}
}  // namespace

sg_status sg_block_dot(sg_handle* h, int64_t n, const double* Q, int64_t ldq,
                       int32_t i, const double* X, int64_t ldx, int32_t s,
                       double* W, int32_t ldw, int32_t sym, void* stream) {
  if (!h) return SG_EINVAL;
  return guarded(h, [&] {
    SG_REQUIRE(n >= 0 && i >= 0 && s >= 0 && ldq >= n && ldx >= n && ldw >= i,
               SG_EINVAL, "bad sizes");
    SG_REQUIRE((Q && X && W) || i == 0 || s == 0, SG_EINVAL, "null pointer");
    SG_REQUIRE(!sym || (Q == X && i == s), SG_EINVAL, "sym needs Q == X");
    SG_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = pick(h, stream);
    const int64_t need = sg::block_dot_part_size(n, i, s);
    if (need > h->part_cap) {
      SG_CUDA(cudaStreamSynchronize(st));
      if (h->part) cudaFree(h->part);
      h->part = nullptr;
      h->part_cap = 0;
      SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->part), sizeof(double) * need));
      h->part_cap = need;
    }
    sg::block_dot(n, Q, ldq, i, X, ldx, s, W, ldw, sym != 0, h->part, h->part_cap, st);
    sg::oz_check_error(st);  // synchronises: reports a tensor-core timeout
  });
}

sg_status sg_block_update(sg_handle* h, int64_t n, const double* Q,
                          int64_t ldq, int32_t i, const double* W,
                          int32_t ldw, double* X, int64_t ldx, int32_t s,
                          double alpha, double beta, int32_t upper,
                          void* stream) {
  if (!h) return SG_EINVAL;
  return guarded(h, [&] {
    SG_REQUIRE(n >= 0 && i >= 0 && s >= 0 && ldq >= n && ldx >= n && ldw >= i,
               SG_EINVAL, "bad sizes");
    SG_REQUIRE(X || s == 0 || n == 0, SG_EINVAL, "null X");
    SG_REQUIRE((Q && W) || i == 0, SG_EINVAL, "null Q/W");
    SG_REQUIRE(!upper || i == s, SG_EINVAL, "upper needs i == s");
    SG_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = pick(h, stream);
    ensure_part(h, sg::block_update_scratch(i), st);
    sg::block_update(n, Q, ldq, i, W, ldw, X, ldx, s, alpha, beta, upper != 0, h->part,
                     h->part_cap, st);
    sg::oz_check_error(st);  // synchronises: reports a tensor-core timeout
  });
}


sg_status sg_block_dot_f32(sg_handle* h, int64_t n, const float* Q,
                           int64_t ldq, int32_t i, const float* X,
                           int64_t ldx, int32_t s, double* W, int32_t ldw,
                           int32_t sym, void* stream) {
  if (!h) return SG_EINVAL;
  return guarded(h, [&] {
    SG_REQUIRE(n >= 0 && i >= 0 && s >= 0 && ldq >= n && ldx >= n && ldw >= i,
               SG_EINVAL, "bad sizes");
    SG_REQUIRE((Q && X && W) || i == 0 || s == 0, SG_EINVAL, "null pointer");
    SG_REQUIRE(!sym || (Q == X && i == s), SG_EINVAL, "sym needs Q == X");
    SG_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = pick(h, stream);
    ensure_part(h, sg::block_dot_part_size(n, i, s), st);
    sg::block_dot32(n, Q, ldq, i, X, ldx, s, W, ldw, sym != 0, h->part, h->part_cap, st);
    sg::tc_check_error(st);  // synchronises: reports a tensor-core timeout
    sg::oz_check_error(st);
  });
}

sg_status sg_block_update_f32(sg_handle* h, int64_t n, const float* Q,
                              int64_t ldq, int32_t i, const double* W,
                              int32_t ldw, float* X, int64_t ldx, int32_t s,
                              double alpha, double beta, int32_t upper,
                              void* stream) {
  if (!h) return SG_EINVAL;
  return guarded(h, [&] {
    SG_REQUIRE(n >= 0 && i >= 0 && s >= 0 && ldq >= n && ldx >= n && ldw >= i,
               SG_EINVAL, "bad sizes");
    SG_REQUIRE(X || s == 0 || n == 0, SG_EINVAL, "null X");
    SG_REQUIRE((Q && W) || i == 0, SG_EINVAL, "null Q/W");
    SG_REQUIRE(!upper || i == s, SG_EINVAL, "upper needs i == s");
    SG_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = pick(h, stream);
    if (i > 0 && s > 0) ensure_part(h, (sg::tc_update_scratch(i, s) + 1) / 2, st);
    sg::block_update32(n, Q, ldq, i, W, ldw, X, ldx, s, alpha, beta, upper != 0,
                       h->part, h->part_cap, st);
    sg::tc_update_check_error(st);  // synchronises: reports a tensor-core timeout
  });
}

sg_status sg_nrm2(sg_handle* h, int64_t n, const double* x, double* out,
                  void* stream) {
  if (!h) return SG_EINVAL;
  return guarded(h, [&] {
    SG_REQUIRE(x && out && n >= 0, SG_EINVAL, "bad arguments");
    SG_CUDA(cudaSetDevice(h->device));
    cudaStream_t st = pick(h, stream);
    if (!h->red) {
      SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&h->red),
                         sizeof(double) * sg::reduction_blocks() * 3));
    }
    double* slot = nullptr;
    SG_CUDA(cudaMalloc(reinterpret_cast<void**>(&slot), sizeof(double)));
    sg::dot_partials(n, x, x, h->red, st);
    sg::finish_sum(h->red, slot, true, st);
    cudaError_t e1 = cudaMemcpyAsync(out, slot, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(slot);
    SG_CUDA(e1);
    SG_CUDA(e2);
  });
}

int32_t sg_host_partial_cholesky(const double* G, int32_t ldg, int32_t s,
                                 double omega, double* R, double* kappa) {
  if (!G || !R || s < 0 || ldg < s) return -1;
  return sg::partial_cholesky(G, ldg, s, omega, R, s, kappa);
}

int32_t sg_host_hessenberg_eigvals(const double* H, int32_t ldh, int32_t k,
                                   double* re, double* im) {
  if (!H || !re || !im || k < 0 || ldh < k) return -1;
  return sg::hessenberg_eigvals(H, ldh, k, re, im);
}

void sg_host_leja_order(int32_t k, const double* re, const double* im,
                        double* out_re, double* out_im) {
  if (k <= 0 || !re || !im || !out_re || !out_im) return;
  sg::leja_order(k, re, im, out_re, out_im);
}

void sg_host_scaling_coefficients(int32_t k, const double* re,
                                  const double* im, double* gamma) {
  if (k <= 0 || !re || !im || !gamma) return;
  sg::scaling_coefficients(k, re, im, gamma);
}

int32_t sg_host_estimate_step(int32_t k, const double* re, const double* im,
                              double eps, double omega_est, int32_t s_min,
                              int32_t s_max, double* norms) {
  if (k < 0 || (k > 0 && (!re || !im))) return -1;
  return sg::estimate_step(k, re, im, eps, omega_est, s_min, s_max, norms);
}

int32_t sg_host_upper_inverse(const double* R, int32_t ldr, int32_t p, double* Ri,
                              int32_t ldri) {
  if (p < 0 || (p > 0 && (!R || !Ri || ldr < p || ldri < p))) return -1;
  if (p > 0) sg::upper_inverse(R, ldr, p, Ri, ldri);
  return 0;
}

int32_t sg_host_basis(int32_t s, const double* re, const double* im,
                      const double* gamma, double* theta, double* c, double* g,
                      double* B, int32_t ldb) {
  if (s < 0 || (s > 0 && (!re || !im || !gamma))) return -1;
  if (B && ldb < s + 1) return -1;
  std::vector<sg::BasisStep> st;
  sg::basis_steps(s, re, im, gamma, st);
  for (int j = 0; j < s; ++j) {
    if (theta) theta[j] = st[j].theta;
    if (c) c[j] = st[j].c;
    if (g) g[j] = st[j].gamma;
  }
  if (B && s > 0) sg::change_of_basis(st, s, B, ldb);
  return 0;
}

int32_t sg_host_combine_r(int32_t i, int32_t q, const double* W, int32_t ldw,
                          const double* Rp, int32_t ldrp, const double* Z1,
                          int32_t ldz1, const double* R2, int32_t ldr2,
                          double* R_top, int32_t ldt, double* R_kk, int32_t ldk) {
  if (i < 1 || q < 1 || !W || !Rp || !Z1 || !R2 || !R_top || !R_kk || ldw < i ||
      ldrp < i || ldz1 < q || ldr2 < q || ldt < i || ldk < q)
    return -1;
  sg::combine_r(i, q, W, ldw, Rp, ldrp, Z1, ldz1, R2, ldr2, R_top, ldt, R_kk, ldk);
  return 0;
}

int32_t sg_host_assemble_hessenberg(double* H, int32_t ldh, int32_t i, int32_t q,
                                    const double* R_top, int32_t ldt,
                                    const double* R_kk, int32_t ldk, const double* B,
                                    int32_t ldb) {
  if (!H || !R_top || !R_kk || !B || i < 1 || q < 1 || ldh < i + q || ldt < i ||
      ldk < q || ldb < q + 1)
    return -1;
  sg::assemble_hessenberg(H, ldh, i, q, R_top, ldt, R_kk, ldk, B, ldb);
  return 0;
}

double sg_host_givens_column(double* Hr, int32_t ldhr, double* cs, double* sn,
                             double* g, const double* H, int32_t ldh, int32_t j) {
  if (!Hr || !cs || !sn || !g || !H || j < 0 || ldhr < j + 2 || ldh < j + 2) return -1.0;
  return sg::givens_column(Hr, ldhr, cs, sn, g, H, ldh, j);
}

int32_t sg_host_givens_solve(const double* Hr, int32_t ldhr, const double* g,
                             int32_t jj, double* y) {
  if (jj < 0 || (jj > 0 && (!Hr || !g || !y || ldhr < jj))) return -1;
  sg::givens_solve(Hr, ldhr, g, jj, y);
  return 0;
}

int64_t sg_host_halo_plan(int32_t rows, const int32_t* rowptr, const int32_t* colind,
                          int32_t lo, int32_t hi, int32_t* local_colind,
                          int32_t* halo_cols) {
  if (rows < 0 || hi - lo != rows || !rowptr || (rowptr[rows] > 0 && !colind)) return -1;
  return sg::halo_plan(rows, rowptr, colind, lo, hi, local_colind, halo_cols);
}

}  // extern "C"
