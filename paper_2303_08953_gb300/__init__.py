"""Python binding of the sm_103a adaptive s-step GMRES library.

Thin ctypes marshalling over the C ABI in include/sgmres.h (same names,
without the ``sg_`` prefix).  Every step of the solver runs in the CUDA
library; this module only passes pointers, sizes and the current torch
stream.  Device memory comes from torch.  There is no CPU fallback: if the
library is missing, importing the library raises.

Dense matrices follow the library's column-major layout: an n x k matrix
with leading dimension ld is held as a torch tensor of shape (k, ld) (its
transpose, row-major), so column j is ``T[j]``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsgmres.so")

SG_OK, SG_EINVAL, SG_ENOMEM, SG_ECUDA, SG_ENOCONV, SG_ENUMERIC, SG_ESTATE = range(7)
STATUS_NAMES = {0: "SG_OK", 1: "SG_EINVAL", 2: "SG_ENOMEM", 3: "SG_ECUDA",
                4: "SG_ENOCONV", 5: "SG_ENUMERIC", 6: "SG_ESTATE"}
BASES = {"scaled_newton": 0, "newton": 1, "monomial": 2}
PRECISIONS = {"fp64": 0, "fp32_ir": 1}
EQUILIBRATIONS = {"none": 0, "scalar": 1, "column": 2}

EXPORTED = (
    "sg_default_opts", "sg_create", "sg_destroy", "sg_last_error",
    "sg_analyze", "sg_solve", "sg_solve_adjoint", "sg_grad_values",
    "sg_spmv_newton", "sg_residual", "sg_mpk", "sg_block_dot",
    "sg_block_update", "sg_nrm2", "sg_host_partial_cholesky",
    "sg_host_hessenberg_eigvals", "sg_host_leja_order",
    "sg_host_scaling_coefficients", "sg_host_estimate_step",
    "sg_kernel_launches", "sg_block_dot_noalloc", "sg_block_dot_f32",
    "sg_block_update_f32", "sg_update_values", "sg_matrix_info",
    "sg_probe_bounded_waits", "sg_arnoldi", "sg_analyze_rows", "sg_gather",
    "sg_host_upper_inverse", "sg_host_basis", "sg_host_combine_r",
    "sg_host_assemble_hessenberg", "sg_host_givens_column",
    "sg_host_givens_solve", "sg_host_halo_plan", "sg_set_tc_policy",
)


def probe_bounded_waits(device=0, limit_ms=50.0):
    """(grid barrier timed out, mbarrier timed out): runs the library's
    failure-detection probe (waits that cannot complete, bounded by
    limit_ms) and reports whether each was caught and reported."""
    a, b = C.c_int32(0), C.c_int32(0)
    rc = lib.sg_probe_bounded_waits(device, limit_ms, C.byref(a), C.byref(b))
    if rc != 0:
        raise SgError(rc, "sg_probe_bounded_waits failed")
    return bool(a.value), bool(b.value)


class SgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class sg_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("colind", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int32)]


_DP = C.POINTER(C.c_double)


class sg_opts(C.Structure):
    _fields_ = [("m", C.c_int32), ("s", C.c_int32), ("s_min", C.c_int32),
                ("s_max", C.c_int32), ("tol", C.c_double),
                ("max_iters", C.c_int32), ("omega", C.c_double),
                ("omega_est", C.c_double), ("basis", C.c_int32),
                ("precision", C.c_int32), ("inner_tol", C.c_double),
                ("max_refine", C.c_int32), ("vectors_on_device", C.c_int32),
                ("stream", C.c_void_p), ("equilibrate", C.c_int32),
                ("n_ritz", C.c_int32), ("ritz_re", _DP), ("ritz_im", _DP)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int32)


class sg_result(C.Structure):
    _fields_ = [("converged", C.c_int32), ("s0", C.c_int32),
                ("iters", C.c_int32), ("restarts", C.c_int32),
                ("refinements", C.c_int32), ("final_relres", C.c_double),
                ("hist_cap", C.c_int32), ("relres_hist", _D),
                ("n_hist", C.c_int32),
                ("blocks_cap", C.c_int32), ("s_eff_hist", _I),
                ("p1_hist", _I), ("s_hist", _I), ("n_blocks", C.c_int32),
                ("cycles_cap", C.c_int32), ("cycle_relres", _D),
                ("cycle_iters", _I), ("n_cycles", C.c_int32),
                ("ritz_cap", C.c_int32), ("ritz_re", _D), ("ritz_im", _D),
                ("gamma", _D), ("n_ritz", C.c_int32),
                ("t_prepass_ms", C.c_double), ("t_mpk_ms", C.c_double),
                ("t_ortho_ms", C.c_double), ("t_host_ms", C.c_double),
                ("t_total_ms", C.c_double), ("fp64_iters", C.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is not built; run `python -c \"import "
            "__graft_entry__ as g; g.build()\"` (needs nvcc)")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "sg_default_opts": (None, [C.POINTER(sg_opts)]),
        "sg_create": (i32, [C.c_int, C.POINTER(vp)]),
        "sg_destroy": (None, [vp]),
        "sg_last_error": (C.c_char_p, [vp]),
        "sg_analyze": (i32, [vp, C.POINTER(sg_csr)]),
        "sg_update_values": (i32, [vp, vp, i32]),
        "sg_matrix_info": (i32, [vp, C.POINTER(i32), C.POINTER(i64)]),
        "sg_probe_bounded_waits": (i32, [i32, f64, C.POINTER(i32), C.POINTER(i32)]),
        "sg_solve": (i32, [vp, vp, vp, C.POINTER(sg_opts), C.POINTER(sg_result)]),
        "sg_solve_adjoint": (i32, [vp, vp, vp, C.POINTER(sg_opts), C.POINTER(sg_result)]),
        "sg_grad_values": (i32, [vp, vp, vp, vp, vp]),
        "sg_spmv_newton": (i32, [vp, vp, vp, vp, f64, f64, f64, vp]),
        "sg_residual": (i32, [vp, vp, vp, vp, vp]),
        "sg_mpk": (i32, [vp, vp, vp, i64, i32, _D, _D, _D, vp]),
        "sg_arnoldi": (i32, [vp, vp, i32, i32, _D, i32, C.POINTER(i32), vp]),
        "sg_block_dot": (i32, [vp, i64, vp, i64, i32, vp, i64, i32, vp, i32, i32, vp]),
        "sg_block_update": (i32, [vp, i64, vp, i64, i32, vp, i32, vp, i64, i32,
                                  f64, f64, i32, vp]),
        "sg_nrm2": (i32, [vp, i64, vp, _D, vp]),
        "sg_block_dot_f32": (i32, [vp, i64, vp, i64, i32, vp, i64, i32, vp, i32, i32, vp]),
        "sg_block_update_f32": (i32, [vp, i64, vp, i64, i32, vp, i32, vp, i64, i32,
                                      f64, f64, i32, vp]),
        "sg_host_partial_cholesky": (i32, [_D, i32, i32, f64, _D, _D]),
        "sg_host_hessenberg_eigvals": (i32, [_D, i32, i32, _D, _D]),
        "sg_host_leja_order": (None, [i32, _D, _D, _D, _D]),
        "sg_host_scaling_coefficients": (None, [i32, _D, _D, _D]),
        "sg_host_estimate_step": (i32, [i32, _D, _D, f64, f64, i32, i32, _D]),
        "sg_kernel_launches": (i64, []),
        "sg_set_tc_policy": (i32, [i32]),
        "sg_analyze_rows": (i32, [vp, C.POINTER(sg_csr), i32]),
        "sg_gather": (i32, [vp, i64, vp, vp, vp]),
        "sg_host_upper_inverse": (i32, [_D, i32, i32, _D, i32]),
        "sg_host_basis": (i32, [i32, _D, _D, _D, _D, _D, _D, _D, i32]),
        "sg_host_combine_r": (i32, [i32, i32, _D, i32, _D, i32, _D, i32, _D, i32,
                                    _D, i32, _D, i32]),
        "sg_host_assemble_hessenberg": (i32, [_D, i32, i32, i32, _D, i32, _D, i32,
                                              _D, i32]),
        "sg_host_givens_column": (f64, [_D, i32, _D, _D, _D, _D, i32, i32]),
        "sg_host_givens_solve": (i32, [_D, i32, _D, i32, _D]),
        "sg_host_halo_plan": (i64, [i32, _I, _I, i32, i32, _I, _I]),
        "sg_block_dot_noalloc": (i32, [i64, vp, i64, i32, vp, i64, i32, vp, i32,
                                       vp, C.c_char_p, i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(_I)


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib.sg_kernel_launches())


TC_POLICIES = {"auto": 0, "never": 1, "always": 2}


def set_tc_policy(policy: str) -> str:
    """Tensor-core policy of the FP64 block products, process-wide: "auto"
    (cost model), "never" (FP64 pipe) or "always" (tensor cores wherever the
    layout allows).  Returns the previous policy."""
    old = int(lib.sg_set_tc_policy(TC_POLICIES[policy]))
    if old < 0:
        raise ValueError(policy)
    return {v: k for k, v in TC_POLICIES.items()}[old]


# ------------------------------------------------------- host algebra
def partial_cholesky(G, omega=1e7):
    """Alg. 3 with the ICE stop: returns (p, R_p, kappas)."""
    G = np.asfortranarray(G, dtype=np.float64)
    s = G.shape[0]
    R = np.zeros((s, s), order="F")
    kap = np.zeros(max(s, 1))
    p = lib.sg_host_partial_cholesky(_dp(G), s, s, omega, _dp(R), _dp(kap))
    if p < 0:
        raise SgError(SG_EINVAL, "partial_cholesky: bad arguments")
    kk = min(s, p + 1)
    return p, np.array(R[:p, :p]), kap[:kk].copy()


def hessenberg_eigvals(H):
    H = np.asfortranarray(H, dtype=np.float64)
    k = H.shape[1]
    re = np.zeros(k)
    im = np.zeros(k)
    rc = lib.sg_host_hessenberg_eigvals(_dp(H), H.shape[0], k, _dp(re), _dp(im))
    if rc != 0:
        raise SgError(SG_ENUMERIC, "Hessenberg QR did not converge")
    return re + 1j * im


def leja_order(theta):
    th = np.asarray(theta, dtype=np.complex128)
    re, im = np.ascontiguousarray(th.real), np.ascontiguousarray(th.imag)
    ore, oim = np.zeros_like(re), np.zeros_like(im)
    lib.sg_host_leja_order(th.size, _dp(re), _dp(im), _dp(ore), _dp(oim))
    return ore + 1j * oim


def scaling_coefficients(theta):
    th = np.asarray(theta, dtype=np.complex128)
    re, im = np.ascontiguousarray(th.real), np.ascontiguousarray(th.imag)
    g = np.zeros_like(re)
    lib.sg_host_scaling_coefficients(th.size, _dp(re), _dp(im), _dp(g))
    return g


def estimate_step(theta, eps=2.0 ** -53, omega_est=1e7, s_min=1, s_max=0):
    th = np.asarray(theta, dtype=np.complex128)
    re, im = np.ascontiguousarray(th.real), np.ascontiguousarray(th.imag)
    norms = np.zeros(max(th.size, 1))
    s0 = lib.sg_host_estimate_step(th.size, _dp(re), _dp(im), eps, omega_est,
                                   s_min, s_max, _dp(norms))
    return int(s0), norms[:th.size].copy()


def _f(a):
    """Column-major float64 copy (or view) for the host calls."""
    return np.asfortranarray(a, dtype=np.float64)


def _ok(rc, what):
    if rc != 0:
        raise SgError(SG_EINVAL, f"{what}: bad arguments")


def upper_inverse(R, p=None):
    """Inverse of the leading p x p block of upper-triangular R."""
    R = _f(R)
    p = R.shape[0] if p is None else p
    Ri = np.zeros((p, p), order="F")
    _ok(lib.sg_host_upper_inverse(_dp(R), R.shape[0], p, _dp(Ri), max(p, 1)), "upper_inverse")
    return Ri


def basis(theta, gamma, s):
    """(theta, c, g, B) of s matrix-powers steps: per-step shift, pair
    coefficient and scale, and the (s+1) x s change-of-basis matrix."""
    th = np.asarray(theta, dtype=np.complex128)[:s]
    re, im = np.ascontiguousarray(th.real), np.ascontiguousarray(th.imag)
    gm = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64)[:s])
    t, c, g = np.zeros(s), np.zeros(s), np.zeros(s)
    B = np.zeros((s + 1, s), order="F")
    _ok(lib.sg_host_basis(s, _dp(re), _dp(im), _dp(gm), _dp(t), _dp(c), _dp(g),
                          _dp(B), s + 1), "basis")
    return t, c, g, B


def combine_r(W, Rp, Z1, R2, q):
    """(R_top, R_kk) of Alg. 4 'Combine both steps' (first q columns)."""
    W, Rp, Z1, R2 = _f(W), _f(Rp), _f(Z1), _f(R2)
    i = W.shape[0]
    Rt = np.zeros((i, q), order="F")
    Rk = np.zeros((q, q), order="F")
    _ok(lib.sg_host_combine_r(i, q, _dp(W), i, _dp(Rp), Rp.shape[0], _dp(Z1), Z1.shape[0],
                              _dp(R2), R2.shape[0], _dp(Rt), i, _dp(Rk), q), "combine_r")
    return Rt, Rk


def assemble_hessenberg(H, i, R_top, R_kk, B):
    """New columns i..i+q-1 (1-based i) of H (Fortran-ordered, updated in
    place)."""
    assert H.flags.f_contiguous and H.dtype == np.float64
    R_top, R_kk, B = _f(R_top), _f(R_kk), _f(B)
    q = R_kk.shape[0]
    _ok(lib.sg_host_assemble_hessenberg(_dp(H), H.shape[0], i, q, _dp(R_top), R_top.shape[0],
                                        _dp(R_kk), q, _dp(B), B.shape[0]), "assemble_hessenberg")


def givens_column(Hr, cs, sn, g, H, j):
    """Rotate column j of H into Hr (Fortran-ordered arrays updated in
    place); returns |g[j+1]|."""
    assert Hr.flags.f_contiguous and H.flags.f_contiguous
    r = lib.sg_host_givens_column(_dp(Hr), Hr.shape[0], _dp(cs), _dp(sn), _dp(g), _dp(H),
                                  H.shape[0], j)
    if r < 0:
        raise SgError(SG_EINVAL, "givens_column: bad arguments")
    return r


def givens_solve(Hr, g, jj):
    y = np.zeros(max(jj, 1))
    _ok(lib.sg_host_givens_solve(_dp(Hr), Hr.shape[0], _dp(g), jj, _dp(y)), "givens_solve")
    return y[:jj]


def halo_plan(rowptr, colind, lo, hi):
    """(local_colind, halo_cols) of the row block [lo, hi) (global columns)."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    loc = np.zeros(max(ci.size, 1), dtype=np.int32)
    halo = np.zeros(max(ci.size, 1), dtype=np.int32)
    nh = lib.sg_host_halo_plan(hi - lo, _ip(rp), _ip(ci), lo, hi, _ip(loc), _ip(halo))
    if nh < 0:
        raise SgError(SG_EINVAL, "halo_plan: bad arguments")
    return loc[:ci.size].copy(), halo[:nh].copy()


def gather(idx, src, out, stream=None):
    """out[k] = src[idx[k]] on the device (idx an int32 CUDA tensor)."""
    rc = lib.sg_gather(C.c_void_p(idx.data_ptr()), idx.numel(), C.c_void_p(src.data_ptr()),
                       C.c_void_p(out.data_ptr()), _stream_ptr(stream))
    if rc != 0:
        raise SgError(rc, "sg_gather failed")
    return out


# ------------------------------------------------------------ solver
@dataclass
class SolveInfo:
    status: int
    converged: bool
    s0: int
    iters: int
    restarts: int
    refinements: int
    final_relres: float
    relres_hist: np.ndarray
    s_eff_hist: np.ndarray
    p1_hist: np.ndarray
    s_hist: np.ndarray
    cycle_relres: np.ndarray
    cycle_iters: np.ndarray
    ritz: np.ndarray
    gamma: np.ndarray
    times_ms: dict = field(default_factory=dict)
    fp64_iters: int = 0


def _torch():
    import torch
    return torch


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream


def _stream_ptr(stream=None):
    """cudaStream_t of a torch stream.  torch's default stream has handle
    0, which the C ABI reads as "the handle's own stream"; it is passed as
    cudaStreamLegacy instead so the work stays ordered with torch's."""
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream or CUDA_STREAM_LEGACY)


class Solver:
    """One handle of the C library bound to a CUDA device."""

    def __init__(self, device: int = 0):
        self._h = C.c_void_p()
        rc = lib.sg_create(device, C.byref(self._h))
        if rc != SG_OK:
            raise SgError(rc, f"sg_create(device={device}) failed")
        self.device = device
        self.n = None
        self.nnz = None

    def close(self):
        if self._h:
            lib.sg_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != SG_OK and rc not in allow:
            raise SgError(rc, lib.sg_last_error(self._h).decode())
        return rc

    # -------------------------------------------------- ingest
    def analyze(self, rowptr, colind, val, n=None):
        """Ingest a CSR matrix.  Arrays may be numpy (host) or torch
        tensors on this device (int32, int32, float64)."""
        torch = _torch()
        on_dev = isinstance(val, torch.Tensor) and val.is_cuda
        keep = []
        if on_dev:
            rp, ci, v = (t.contiguous() for t in (rowptr, colind, val))
            assert rp.dtype == torch.int32 and ci.dtype == torch.int32
            assert v.dtype == torch.float64
            keep = [rp, ci, v]
            ptrs = [t.data_ptr() for t in keep]
            nn = rp.numel() - 1
            nnz = ci.numel()
        else:
            rp = np.ascontiguousarray(rowptr, dtype=np.int32)
            ci = np.ascontiguousarray(colind, dtype=np.int32)
            v = np.ascontiguousarray(val, dtype=np.float64)
            keep = [rp, ci, v]
            ptrs = [a.ctypes.data for a in keep]
            nn = rp.size - 1
            nnz = ci.size
        if n is not None:
            assert n == nn
        A = sg_csr(nn, nnz, ptrs[0], ptrs[1], ptrs[2], 1 if on_dev else 0)
        self._check(lib.sg_analyze(self._h, C.byref(A)))
        self.n, self.nnz = nn, nnz
        return self

    def matrix_info(self):
        """(sell, stored): whether the SpMV uses the SELL-32 copy, and the
        entries it reads per product."""
        sell, stored = C.c_int32(0), C.c_int64(0)
        self._check(lib.sg_matrix_info(self._h, C.byref(sell), C.byref(stored)))
        return bool(sell.value), int(stored.value)

    def update_values(self, val):
        """New values for the analysed pattern (numpy or a CUDA tensor)."""
        torch = _torch()
        if isinstance(val, torch.Tensor) and val.is_cuda:
            v = val.to(torch.float64).contiguous()
            torch.cuda.current_stream().synchronize()
            self._check(lib.sg_update_values(self._h, C.c_void_p(v.data_ptr()), 1))
        else:
            v = np.ascontiguousarray(val, dtype=np.float64)
            self._check(lib.sg_update_values(self._h, C.c_void_p(v.ctypes.data), 0))
        return self

    def analyze_rows(self, rowptr, colind, val, ncols):
        """Ingest a row block with local columns in [0, ncols) (host numpy
        arrays; see sg_analyze_rows)."""
        rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(colind, dtype=np.int32)
        v = np.ascontiguousarray(val, dtype=np.float64)
        A = sg_csr(rp.size - 1, ci.size, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, 0)
        self._check(lib.sg_analyze_rows(self._h, C.byref(A), ncols))
        self.n, self.nnz = rp.size - 1, ci.size
        return self

    def analyze_csr(self, A):
        """Ingest a workloads.CSR (host numpy arrays)."""
        return self.analyze(A.rowptr, A.colind, A.val)

    # -------------------------------------------------- solve
    @staticmethod
    def make_opts(m=60, s=10, s_min=1, s_max=0, tol=1e-10, max_iters=0,
                  omega=1e7, omega_est=1e7, basis="scaled_newton",
                  precision="fp64", inner_tol=1e-4, max_refine=20,
                  equilibrate="none", ritz=None):
        """sg_opts from keywords.  ritz: Ritz values to use instead of the
        pre-pass (the arrays are kept on the returned object)."""
        o = sg_opts()
        lib.sg_default_opts(C.byref(o))
        o.m, o.s, o.s_min, o.s_max = m, s, s_min, s_max
        o.tol, o.max_iters = tol, max_iters
        o.omega, o.omega_est = omega, omega_est
        o.basis = BASES[basis] if isinstance(basis, str) else basis
        o.precision = (PRECISIONS[precision] if isinstance(precision, str)
                       else precision)
        o.inner_tol, o.max_refine = inner_tol, max_refine
        o.equilibrate = (EQUILIBRATIONS[equilibrate] if isinstance(equilibrate, str)
                         else equilibrate)
        if ritz is not None:
            th = np.asarray(ritz, dtype=np.complex128).ravel()
            o._ritz = (np.ascontiguousarray(th.real), np.ascontiguousarray(th.imag))
            o.n_ritz = th.size
            o.ritz_re, o.ritz_im = _dp(o._ritz[0]), _dp(o._ritz[1])
        return o

    def _solve(self, fn, b, x0, opts, stream, hist_cap):
        torch = _torch()
        on_dev = isinstance(b, torch.Tensor) and b.is_cuda
        if on_dev:
            assert b.dtype == torch.float64 and b.numel() == self.n
            bb = b.contiguous()
            x = (torch.zeros_like(bb) if x0 is None
                 else x0.to(torch.float64).contiguous().clone())
            opts.vectors_on_device = 1
            opts.stream = _stream_ptr(stream)
            bp, xp = bb.data_ptr(), x.data_ptr()
        else:
            bb = np.ascontiguousarray(b, dtype=np.float64)
            x = (np.zeros(self.n) if x0 is None
                 else np.array(x0, dtype=np.float64, copy=True))
            opts.vectors_on_device = 0
            opts.stream = (_stream_ptr(stream) if stream is not None else None)
            bp, xp = bb.ctypes.data, x.ctypes.data
        res = sg_result()
        hist = np.zeros(hist_cap)
        nb = hist_cap
        s_eff = np.zeros(nb, np.int32)
        p1 = np.zeros(nb, np.int32)
        sh = np.zeros(nb, np.int32)
        cyc = np.zeros(nb)
        cyi = np.zeros(nb, np.int32)
        rcap = max(opts.s_max, opts.s, opts.m) + 1
        rre, rim, gam = np.zeros(rcap), np.zeros(rcap), np.zeros(rcap)
        res.hist_cap, res.relres_hist = hist_cap, _dp(hist)
        res.blocks_cap, res.s_eff_hist, res.p1_hist, res.s_hist = nb, _ip(s_eff), _ip(p1), _ip(sh)
        res.cycles_cap, res.cycle_relres, res.cycle_iters = nb, _dp(cyc), _ip(cyi)
        res.ritz_cap, res.ritz_re, res.ritz_im, res.gamma = rcap, _dp(rre), _dp(rim), _dp(gam)
        rc = fn(self._h, C.c_void_p(bp), C.c_void_p(xp), C.byref(opts),
                C.byref(res))
        self._check(rc, allow=(SG_ENOCONV,))
        nh = min(res.n_hist, hist_cap)
        nbk = min(res.n_blocks, nb)
        nc = min(res.n_cycles, nb)
        nr = min(res.n_ritz, rcap)
        info = SolveInfo(
            status=rc, converged=bool(res.converged), s0=res.s0,
            iters=res.iters, restarts=res.restarts,
            refinements=res.refinements, final_relres=res.final_relres,
            relres_hist=hist[:nh].copy(), s_eff_hist=s_eff[:nbk].copy(),
            p1_hist=p1[:nbk].copy(), s_hist=sh[:nbk].copy(),
            cycle_relres=cyc[:nc].copy(), cycle_iters=cyi[:nc].copy(),
            ritz=rre[:nr] + 1j * rim[:nr], gamma=gam[:nr].copy(),
            times_ms=dict(prepass=res.t_prepass_ms, mpk=res.t_mpk_ms,
                          ortho=res.t_ortho_ms, host=res.t_host_ms,
                          total=res.t_total_ms),
            fp64_iters=res.fp64_iters)
        return x, info

    def solve(self, b, x0=None, stream=None, hist_cap=1 << 16, **kw):
        """Solve A x = b (Alg. 4 with restarts).  b: numpy (host) or a
        float64 CUDA tensor.  Returns (x, SolveInfo)."""
        return self._solve(lib.sg_solve, b, x0, self.make_opts(**kw), stream,
                           hist_cap)

    def solve_adjoint(self, g, lam0=None, stream=None, hist_cap=1 << 16, **kw):
        """Solve A^T lam = g with the same method (transposed CSR)."""
        return self._solve(lib.sg_solve_adjoint, g, lam0, self.make_opts(**kw),
                           stream, hist_cap)

    def grad_values(self, lam, x, out=None, stream=None):
        """dval[k] = -lam[row(k)] x[col(k)] on A's pattern (device)."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.nnz, dtype=torch.float64, device=lam.device)
        self._check(lib.sg_grad_values(self._h, C.c_void_p(lam.data_ptr()),
                                       C.c_void_p(x.data_ptr()),
                                       C.c_void_p(out.data_ptr()),
                                       _stream_ptr(stream)))
        return out

    # ------------------------------------------------ kernel-level calls
    def spmv_newton(self, x, theta=0.0, gamma=1.0, z=None, c=0.0, out=None,
                    stream=None):
        torch = _torch()
        y = torch.empty_like(x) if out is None else out
        self._check(lib.sg_spmv_newton(
            self._h, C.c_void_p(x.data_ptr()),
            C.c_void_p(z.data_ptr() if z is not None else 0),
            C.c_void_p(y.data_ptr()), theta, c, gamma, _stream_ptr(stream)))
        return y

    def residual(self, b, x, out=None, stream=None):
        torch = _torch()
        r = torch.empty_like(b) if out is None else out
        self._check(lib.sg_residual(self._h, C.c_void_p(b.data_ptr()),
                                    C.c_void_p(x.data_ptr()),
                                    C.c_void_p(r.data_ptr()),
                                    _stream_ptr(stream)))
        return r

    def mpk(self, q, s, theta, gamma, stream=None):
        """V (as a (s+1, n) tensor, row j = column j) of Sec. 2's MPK."""
        torch = _torch()
        th = np.asarray(theta, dtype=np.complex128)
        re = np.ascontiguousarray(th.real[:s])
        im = np.ascontiguousarray(th.imag[:s])
        gm = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64)[:s])
        V = torch.empty((s + 1, self.n), dtype=torch.float64, device=q.device)
        self._check(lib.sg_mpk(self._h, C.c_void_p(q.data_ptr()),
                               C.c_void_p(V.data_ptr()), self.n, s, _dp(re),
                               _dp(im), _dp(gm), _stream_ptr(stream)))
        return V

    def arnoldi(self, q, k, precision="fp64", stream=None):
        """(H, steps): k steps of the Ritz pre-pass (Sec. 3.4) from the unit
        device vector q; H is the (k+1) x k Hessenberg matrix."""
        H = np.zeros((k, k + 1))   # column-major (k+1) x k
        steps = C.c_int32(0)
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        self._check(lib.sg_arnoldi(self._h, C.c_void_p(q.data_ptr()), k, prec,
                                   _dp(H), k + 1, C.byref(steps), _stream_ptr(stream)))
        return H.T.copy(), int(steps.value)

    def block_dot(self, Qt, Xt, sym=False, stream=None):
        """W = Q^T X for column-major Q (tensor (i, ld)) and X ((s, ld));
        returns W as an (s, i) tensor (column-major i x s)."""
        torch = _torch()
        i, ldq = Qt.shape
        s, ldx = Xt.shape
        n = min(ldq, ldx) if self.n is None else self.n
        W = torch.empty((s, i), dtype=torch.float64, device=Qt.device)
        self._check(lib.sg_block_dot(
            self._h, n, C.c_void_p(Qt.data_ptr()), ldq, i,
            C.c_void_p(Xt.data_ptr()), ldx, s, C.c_void_p(W.data_ptr()), i,
            1 if sym else 0, _stream_ptr(stream)))
        return W

    def block_update(self, Qt, Wt, Xt, alpha=-1.0, beta=1.0, upper=False,
                     n=None, stream=None):
        """X = beta X + alpha Q W in place (X as an (s, ld) tensor, W as
        (s, i) = column-major i x s)."""
        i, ldq = Qt.shape
        s, ldx = Xt.shape
        n = n if n is not None else (self.n if self.n is not None else ldq)
        self._check(lib.sg_block_update(
            self._h, n, C.c_void_p(Qt.data_ptr()), ldq, i,
            C.c_void_p(Wt.data_ptr()), i, C.c_void_p(Xt.data_ptr()), ldx, s,
            alpha, beta, 1 if upper else 0, _stream_ptr(stream)))
        return Xt

    def block_dot32(self, Qt, Xt, sym=False, stream=None):
        """FP32 form of block_dot (Q, X float32; W returned float64)."""
        torch = _torch()
        i, ldq = Qt.shape
        s, ldx = Xt.shape
        n = min(ldq, ldx) if self.n is None else self.n
        W = torch.empty((s, i), dtype=torch.float64, device=Qt.device)
        self._check(lib.sg_block_dot_f32(
            self._h, n, C.c_void_p(Qt.data_ptr()), ldq, i,
            C.c_void_p(Xt.data_ptr()), ldx, s, C.c_void_p(W.data_ptr()), i,
            1 if sym else 0, _stream_ptr(stream)))
        return W

    def block_update32(self, Qt, Wt, Xt, alpha=-1.0, beta=1.0, upper=False,
                       n=None, stream=None):
        """FP32 form of block_update (Q, X float32; W float64)."""
        i, ldq = Qt.shape
        s, ldx = Xt.shape
        n = n if n is not None else (self.n if self.n is not None else ldq)
        self._check(lib.sg_block_update_f32(
            self._h, n, C.c_void_p(Qt.data_ptr()), ldq, i,
            C.c_void_p(Wt.data_ptr()), i, C.c_void_p(Xt.data_ptr()), ldx, s,
            alpha, beta, 1 if upper else 0, _stream_ptr(stream)))
        return Xt

    def nrm2(self, x, stream=None):
        out = C.c_double()
        self._check(lib.sg_nrm2(self._h, x.numel(), C.c_void_p(x.data_ptr()),
                                C.byref(out), _stream_ptr(stream)))
        return out.value
