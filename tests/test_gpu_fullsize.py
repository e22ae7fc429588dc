"""Full-size workloads (the 192^3 mixed-precision, 1024^2 differentiation
and 4M-row random-sparse cases) through the C ABI: parity on sampled
outputs the oracle computes one by one, and properties that hold at any
size (true residuals checked on the host, residual monotonicity of
restarted runs, the sampled outer product of the gradient).  Where
unpreconditioned restarted GMRES does not reach 1e-10 at full size (the
192^3 and 1024^2 recipes), the convergence checks (FP32 basis +
refinement against plain FP64, adjoint gradients against a sparse-LU
oracle and its central differences) run on the same recipes at the
largest sizes that converge.  The 128^3 case is in test_gpu_parity.py.
"""
import numpy as np
import pytest

import workloads as W
from oracle import sgmres_oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2303_08953_gb300 as sg  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def host(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def solver():
    s = sg.Solver(0)
    yield s
    s.close()


def _sampled_spmv(solver, A, seed, rows=2000):
    """Newton-step SpMV rows against the CSR sum written out per row."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, A.n)
    y = host(solver.spmv_newton(dev(x), 1.3, 2.1))
    for r in rng.choice(A.n, rows, replace=False):
        a, e = A.rowptr[r], A.rowptr[r + 1]
        ref = (np.dot(A.val[a:e], x[A.colind[a:e]]) - 1.3 * x[r]) / 2.1
        bound = np.abs(A.val[a:e]) @ np.abs(x[A.colind[a:e]]) + 1.3 * abs(x[r])
        assert abs(y[r] - ref) <= 1e-14 * bound


def _relres(op, x, b):
    return np.linalg.norm(b - op @ x) / np.linalg.norm(b)


def _monotone_cycles(info):
    h, k = info.relres_hist, 0
    for n_c in info.cycle_iters:
        seg = h[k:k + n_c]
        assert np.all(np.diff(seg) <= 1e-12 * seg[:-1])
        k += n_c


def _cycles_consistent(info, op, x, b, across=True):
    """Properties of any restarted run, converged or not: implicit
    residuals non-increasing within each cycle, true residuals
    non-increasing from cycle to cycle (each FP64 cycle minimises over a
    space that contains the current x; `across` = False for the FP32
    basis, whose inner minimisation is inexact), and the reported final
    residual equal to the host's ||b - A x|| / ||b||."""
    _monotone_cycles(info)
    cr = info.cycle_relres
    if across:
        assert np.all(cr[1:] <= cr[:-1] * (1 + 1e-6))
    assert abs(_relres(op, x, b) - info.final_relres) <= 1e-6 * info.final_relres


def test_full_size_c3_capped_fp64_and_fp32_ir(solver):
    """192^3 variable-coefficient diffusion at full size.  Unpreconditioned
    GMRES(200) needs about 9,000 columns for 1e-10 here, so both forms run
    under a cap of 1,200 columns and are checked for the properties any
    restarted run has; the FP32-basis form must also make progress."""
    c = W.config_c3()
    A = c["A"]
    op = O.as_operator(A)
    solver.analyze_csr(A)
    assert solver.matrix_info()[0]
    _sampled_spmv(solver, A, 41)
    kw = dict(m=c["m"], s=0, s_min=c["s_min"], s_max=c["s_max"], tol=c["tol"],
              max_iters=1200)
    b = dev(c["b"])
    for prec in ["fp64", "fp32_ir"]:
        x, info = solver.solve(b, precision=prec, **kw)
        xh = host(x)
        print(f"c3 {prec}: iters {info.iters} s0 {info.s0} relres {info.final_relres:.2e} "
              f"fp64_iters {info.fp64_iters}")
        assert 1 <= info.s0 <= c["s_max"]
        _cycles_consistent(info, op, xh, c["b"], across=prec == "fp64")
        assert info.final_relres <= 1e-3


def test_c3_recipe_fp32_ir_reaches_fp64_accuracy():
    """The 192^3 recipe at 48^3 and 32^3, where GMRES(200) converges: FP32
    basis + refinement reaches true relres 1e-10 like the plain FP64 solve.
    At 32^3 the FP32 inner solve stops contracting (kappa eps_32 ~ 1) and
    the remaining columns run with the FP64 basis."""
    s = sg.Solver(0)
    try:
        for n in (48, 32):
            A, rng = W.vardiff3d(n)
            xs = W.uniform_vector(A.n, rng)
            b = W.rhs_from_solution(A, xs)
            op = O.as_operator(A)
            s.analyze_csr(A)
            kw = dict(m=200, s=0, s_min=1, s_max=60, tol=1e-10, max_iters=20000)
            x64, i64 = s.solve(dev(b), precision="fp64", **kw)
            x32, i32 = s.solve(dev(b), precision="fp32_ir", **kw)
            x64, x32 = host(x64), host(x32)
            print(f"vardiff3d {n}: fp64 {i64.iters} fp32_ir {i32.iters} "
                  f"(fp64 basis {i32.fp64_iters})")
            assert i64.converged and i32.converged
            assert _relres(op, x64, b) <= 1e-10 and _relres(op, x32, b) <= 1e-10
            if n == 32:
                assert i32.fp64_iters > 0
            e64 = np.linalg.norm(x64 - xs) / np.linalg.norm(xs)
            d = np.linalg.norm(x32 - x64) / np.linalg.norm(x64)
            assert d <= 10 * max(e64, 1e-12)
    finally:
        s.close()


def _gradient_check(solver, A, b, xt, opts, fd_dirs=16):
    from paper_2303_08953_gb300.autograd import sparse_solve
    solver.analyze_csr(A)
    vals = dev(A.val).requires_grad_(True)
    bt = dev(b).requires_grad_(True)
    x = sparse_solve(vals, bt, solver, **opts)
    L = 0.5 * ((x - dev(xt)) ** 2).sum()
    L.backward()
    gv, gb = host(vals.grad), host(bt.grad)
    S = O.SparseLoss(A, b, xt)
    L0, dv, db, _ = S.gradients()
    ev = np.linalg.norm(gv - dv) / np.linalg.norm(dv)
    eb = np.linalg.norm(gb - db) / np.linalg.norm(db)
    assert abs(L.item() - L0) <= 1e-9 * abs(L0)
    assert ev <= 1e-6 and eb <= 1e-6, (ev, eb)
    h = 1e-6
    for k in range(fd_dirs):
        d = np.random.default_rng(100 + k).standard_normal(A.nnz)
        e = np.random.default_rng(200 + k).standard_normal(A.n)
        fd = (S.loss(h * d, h * e) - S.loss(-h * d, -h * e)) / (2 * h)
        an = gv @ d + gb @ e
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (k, fd, an)


def test_c4_recipe_gradients_against_sparse_oracle(solver):
    """The 1024^2 differentiation recipe at 128^2: FP64 forward and adjoint
    solves to relres 1e-13, dL/dvalues and dL/db against the sparse-LU
    oracle (1e-6 relative) and against the oracle's central differences
    along 16 seeded directions, step 1e-6.  The gradient error is about
    kappa(A) times the solve tolerance; kappa grows 4x per doubling of the
    grid (about 1e7 at 256^2, where relres 1e-12 measured 1e-5), so 128^2
    at 1e-13 is the size that supports the 1e-6 bound."""
    A, rng = W.aniso2d(128)
    xs = W.uniform_vector(A.n, rng)
    xt = W.uniform_vector(A.n, rng)
    b = W.rhs_from_solution(A, xs)
    _gradient_check(solver, A, b, xt, dict(m=120, s=0, s_min=1, s_max=120,
                                           tol=1e-13, max_iters=60000))


def test_full_size_c4_forward_and_adjoint_capped(solver):
    """1024^2 anisotropic diffusion at full size.  Unpreconditioned
    GMRES(120) stagnates near 2.5e-9 here (40,000 columns measured), so the
    forward and adjoint solves run under a cap of 3,000 columns: both keep
    the restarted-run properties, the adjoint runs on the transposed
    matrix, and the value gradient equals -lam_i x_j on sampled entries."""
    c = W.config_c4()
    A = c["A"]
    op = O.as_operator(A)
    solver.analyze_csr(A)
    _sampled_spmv(solver, A, 43)
    kw = dict(m=c["m"], s=0, s_min=c["s_min"], s_max=c["s_max"], tol=c["tol"],
              max_iters=3000)
    x, info = solver.solve(dev(c["b"]), **kw)
    xh = host(x)
    _cycles_consistent(info, op, xh, c["b"])
    g = x - dev(c["xtarget"])
    lam, ainfo = solver.solve_adjoint(g, **kw)
    lh, gh = host(lam), host(g)
    opT = op.T.tocsr()
    _cycles_consistent(ainfo, opT, lh, gh)
    print(f"c4: fwd {info.iters} its relres {info.final_relres:.2e}; "
          f"adj {ainfo.iters} its relres {ainfo.final_relres:.2e}")
    assert info.final_relres <= 1e-2 and ainfo.final_relres <= 1e-2
    dval = host(solver.grad_values(lam, x))
    rng = np.random.default_rng(59)
    for k in rng.choice(A.nnz, 5000, replace=False):
        r = np.searchsorted(A.rowptr, k, side="right") - 1
        assert dval[k] == -lh[r] * xh[A.colind[k]]


def test_full_size_c5_fp32_ir_forward_and_adjoint(solver):
    """4M-row random sparse matrix (105M nonzeros): FP32 basis + FP64
    refinement forward and adjoint solves reach true relres 1e-10 (checked
    with A and A^T on the host), and the value gradient equals
    -lam_i x_j on sampled entries of the pattern."""
    c = W.config_c5()
    A = c["A"]
    op = O.as_operator(A)
    solver.analyze_csr(A)
    sell, stored = solver.matrix_info()
    assert sell and stored == A.nnz   # 25 entries in every row: no padding
    _sampled_spmv(solver, A, 47)
    kw = dict(m=c["m"], s=0, s_min=c["s_min"], s_max=c["s_max"], tol=c["tol"],
              precision="fp32_ir")
    x, info = solver.solve(dev(c["b"]), **kw)
    assert info.converged
    g = x - dev(c["xtarget"])
    lam, ainfo = solver.solve_adjoint(g, **kw)
    assert ainfo.converged
    xh, lh, gh = host(x), host(lam), host(g)
    rf, ra = _relres(op, xh, c["b"]), np.linalg.norm(gh - op.T @ lh) / np.linalg.norm(gh)
    print(f"c5: iters {info.iters}/{ainfo.iters} s0 {info.s0}/{ainfo.s0} "
          f"relres {rf:.2e}/{ra:.2e}")
    assert rf <= 1e-10 and ra <= 1e-10
    dval = host(solver.grad_values(lam, x))
    rng = np.random.default_rng(53)
    for k in rng.choice(A.nnz, 5000, replace=False):
        r = np.searchsorted(A.rowptr, k, side="right") - 1
        assert dval[k] == -lh[r] * xh[A.colind[k]]


# ------------------------------------------- full-size decision parity
def _golden(name):
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", f"fullsize_{name}.json")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["c5", "c2"])
def test_full_size_decisions_match_oracle(solver, name):
    """The FP64 solve of the full-size workload against the oracle's run
    (tests/golden/fullsize_<name>.json, written by make_fullsize_golden.py
    from oracle/ alone), both from the oracle's Ritz values: a 120-step
    Arnoldi pre-pass amplifies rounding-order differences through its
    Krylov basis (kappa grows several-fold per step), so its unconverged
    Ritz values are not reproducible and neither is anything decided from
    them; the pre-pass itself is checked on its converged Ritz values
    below.  Given the same Ritz values: step size s0 from the estimator
    (Sec. 3.5), every block's p and p' (Alg. 3 inside Alg. 4), columns per
    cycle and restarts identical; per-cycle true residuals within 1e-8
    relative or the FP64 evaluation floor; implicit residuals within 1e-6;
    the solution within 1e-9 relative, checked through what that bound
    implies on 1024 sampled entries (their RMS error, scaled to the whole
    vector), on ||x|| and on eight seeded Gaussian functionals u.x
    (|u.(x - x_o)| <= ||u|| 1e-9 ||x_o||)."""
    g = _golden(name)
    c = W.CONFIGS[name]()
    A, b = c["A"], c["b"]
    assert A.n == g["n"] and A.nnz == g["nnz"]
    solver.analyze_csr(A)
    ritz = np.asarray(g["ritz_re"]) + 1j * np.asarray(g["ritz_im"])
    xd, info = solver.solve(dev(b), ritz=ritz, **g["opts"])
    assert np.array_equal(info.ritz, ritz)        # Leja order kept
    assert info.converged == g["converged"]
    assert info.s0 == g["s0"]
    assert list(info.s_hist) == g["s_hist"]
    assert list(info.p1_hist) == g["p1_hist"]
    assert list(info.s_eff_hist) == g["s_eff_hist"]
    assert info.iters == g["iters"] and info.restarts == g["restarts"]
    assert list(info.cycle_iters) == g["cycle_iters"]
    # FP64 evaluation floor of ||b - A x|| / ||b|| (see residual_floor in
    # test_gpu_parity.py), with the exact solution x* standing in for x
    op = O.as_operator(A)
    k = int(np.max(np.diff(op.indptr)))
    floor = 2 * (k + 11) * 2.0 ** -53 * np.linalg.norm(
        np.abs(b) + abs(op) @ np.abs(c["xstar"])) / np.linalg.norm(b)
    co = np.array(g["cycle_relres"])
    assert np.all(np.abs(info.cycle_relres - co) <= np.maximum(1e-8 * co, floor))
    ho = np.array(g["relres_hist"])
    assert info.relres_hist.size == ho.size
    assert np.all(np.abs(info.relres_hist - ho) <= np.maximum(1e-6 * ho, floor))
    x = host(xd)
    xo_norm = g["x_norm"]
    idx = np.asarray(g["x_idx"])
    d = x[idx] - np.asarray(g["x_sample"])
    assert np.sqrt(A.n * np.mean(d * d)) <= 1e-9 * xo_norm
    assert abs(np.linalg.norm(x) - xo_norm) <= 1e-9 * xo_norm
    for k_, fo in enumerate(g["x_functionals"]):
        u = np.random.default_rng([g["sample_seed"], k_]).standard_normal(A.n)
        assert abs(u @ x - fo) <= np.linalg.norm(u) * 1e-9 * xo_norm


@pytest.mark.parametrize("name", ["c5", "c2"])
def test_full_size_prepass_converged_ritz_values(solver, name):
    """The library's own 120-step pre-pass (Sec. 3.4) on the full-size
    workload: every Ritz value the oracle's pre-pass has converged (Ritz-pair
    residual below 1e-9 of the largest modulus; values within 1e-6 of zero
    are left out: this diagonally dominant matrix has no eigenvalue there,
    they are ghosts of the basis's lost orthogonality) is matched by one of
    the library's within ten times that residual (plus 1e-10 of the largest
    modulus).  The 128^3 stencil has no converged Ritz value after 120 steps
    (smallest residual 0.25), so there only the largest modulus is compared,
    to its residual.  And the library's solve from its own Ritz values
    reaches the tolerance with a solution near the seeded exact solution x*
    (forward error <= kappa(A) x relres; 1000 tol bounds it here)."""
    g = _golden(name)
    c = W.CONFIGS[name]()
    A, b = c["A"], c["b"]
    solver.analyze_csr(A)
    xd, info = solver.solve(dev(b), **g["opts"])
    assert info.converged and info.final_relres <= g["opts"]["tol"]
    th = np.asarray(g["prepass_ritz_re"]) + 1j * np.asarray(g["prepass_ritz_im"])
    res = np.asarray(g["prepass_ritz_residual"])
    scale = np.max(np.abs(th))
    conv = (res <= 1e-9 * scale) & (np.abs(th) >= 1e-6 * scale)
    got = info.ritz
    for z, r in zip(th[conv], res[conv]):
        assert np.min(np.abs(got - z)) <= 10 * r + 1e-10 * scale, (z, r)
    top = np.argmax(np.abs(th))
    assert abs(np.max(np.abs(got)) - scale) <= 10 * res[top] + 1e-10 * scale
    x = host(xd)
    xs = c["xstar"]
    assert np.linalg.norm(x - xs) <= 1000 * g["opts"]["tol"] * np.linalg.norm(xs)
