"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle
on the same seeded inputs.

Per-step kernels are compared element by element; whole solves must give
identical step-size decisions and iteration counts, per-cycle true
residual norms within 1e-8 relative and the final x within 1e-9 relative
(the FP64 parity bar).  Sizes span several tiles and a ragged tail.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import sgmres_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2303_08953_gb300 as sg  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def host(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def solver():
    s = sg.Solver(0)
    yield s
    s.close()


def _analyze(solver, A):
    solver.analyze_csr(A)
    return O.as_operator(A)


SMALL_MATRICES = {
    "stencil2d_37x29": lambda: W.stencil2d(37, 29),
    "convdiff3d_11": lambda: W.stencil3d_convdiff(11),
    "randband_5003": lambda: W.random_band(5003, k=24, band=300)[0],
    "vardiff3d_9": lambda: W.vardiff3d(9)[0],
    "aniso2d_41": lambda: W.aniso2d(41)[0],
}


# ------------------------------------------------------------- SpMV / MPK
@pytest.mark.parametrize("name", list(SMALL_MATRICES))
def test_spmv_newton_matches_oracle(solver, name):
    A = SMALL_MATRICES[name]()
    op = _analyze(solver, A)
    rng = np.random.default_rng(21)
    x = rng.uniform(-1, 1, A.n)
    z = rng.uniform(-1, 1, A.n)
    for theta, c, gamma in [(0.0, 0.0, 1.0), (1.7, 0.0, 2.5), (-0.3, 0.8, 0.9)]:
        y = host(solver.spmv_newton(dev(x), theta, gamma, dev(z) if c else None, c))
        ref = (O.spmv(op, x) - theta * x + c * z) / gamma
        scale = (np.abs(op) @ np.abs(x) + abs(theta) * np.abs(x) + abs(c) * np.abs(z)) / abs(gamma)
        assert np.all(np.abs(y - ref) <= 1e-14 * scale + 1e-300)


def test_residual_matches_oracle(solver):
    A = W.stencil3d_convdiff(13)
    op = _analyze(solver, A)
    rng = np.random.default_rng(22)
    x, b = rng.uniform(-1, 1, A.n), rng.uniform(-1, 1, A.n)
    r = host(solver.residual(dev(b), dev(x)))
    assert np.allclose(r, b - op @ x, rtol=0, atol=1e-14 * (np.abs(b).max() + 10))


def test_mpk_matches_oracle_with_pair(solver):
    A = W.stencil2d(33, 21)
    op = _analyze(solver, A)
    q = np.random.default_rng(23).uniform(-1, 1, A.n)
    q /= np.linalg.norm(q)
    theta = np.array([7.1, 0.4, 3.0 + 1.2j, 3.0 - 1.2j, 5.5, 1.9 + 0.4j, 1.9 - 0.4j])
    gamma = np.array([3.0, 3.6, 1.3, 1.3, 1.9, 2.2, 2.2])
    V_o, _ = O.mpk(op, q, 7, theta, gamma)
    V_g = host(solver.mpk(dev(q), 7, theta, gamma)).T
    assert np.allclose(V_g, V_o, rtol=1e-12, atol=1e-13 * np.abs(V_o).max())


def _skewed_csr(n=3001, seed=7):
    """Sparse rows plus one row of 900 entries: padding every slice of 32
    rows to its longest row would more than double the stored entries."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=3.0 / n, random_state=seed, format="lil")
    M.setdiag(4.0)
    M[5, np.sort(rng.choice(n, 900, replace=False))] = rng.standard_normal(900)
    M = M.tocsr()
    M.sort_indices()
    return W.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32),
                 M.data.astype(np.float64))


@pytest.mark.parametrize("kind", ["stencil", "skewed"])
def test_spmv_storage_choice_and_value_update(solver, kind):
    """SELL-32 for a stencil, CSR for a skewed pattern; both match the
    oracle, before and after a value update on the same pattern."""
    A = W.stencil3d_convdiff(11) if kind == "stencil" else _skewed_csr()
    op = _analyze(solver, A)
    sell, stored = solver.matrix_info()
    assert sell == (kind == "stencil")
    if sell:
        assert A.nnz <= stored <= 1.2 * A.nnz + 32 * ((A.n + 31) // 32)
    else:
        assert stored == A.nnz
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, A.n)
    for _ in range(2):
        y = host(solver.spmv_newton(dev(x), 0.7, 1.9))
        ref = (O.spmv(op, x) - 0.7 * x) / 1.9
        scale = (np.abs(op) @ np.abs(x) + 0.7 * np.abs(x)) / 1.9
        assert np.all(np.abs(y - ref) <= 1e-14 * scale + 1e-300)
        r = host(solver.residual(dev(x), dev(x)))
        assert np.all(np.abs(r - (x - O.spmv(op, x))) <= 1e-14 * (np.abs(op) @ np.abs(x) + 1))
        new = rng.standard_normal(A.nnz)
        solver.update_values(new)
        A = W.CSR(A.n, A.rowptr, A.colind, new)
        op = O.as_operator(A)


def test_spmv_empty_rows(solver):
    # rows with no entries produce zero (times 1/gamma) plus the shift part
    rowptr = np.array([0, 1, 1, 3, 3], np.int32)
    colind = np.array([0, 0, 3], np.int32)
    val = np.array([2.0, -1.0, 4.0])
    solver.analyze(rowptr, colind, val)
    x = np.array([1.0, 2.0, 3.0, 4.0])
    y = host(solver.spmv_newton(dev(x), 0.5, 2.0))
    Ax = np.array([2.0, 0.0, -1.0 + 16.0, 0.0])
    assert np.allclose(y, (Ax - 0.5 * x) / 2.0, rtol=0, atol=1e-15)


# ------------------------------------------------------ dense block kernels
@pytest.fixture(params=["never", "always"])
def tc_path(request):
    """Runs a test with the FP64 block products on the FP64 pipe and on the
    tensor cores (wherever their layout allows), whatever the cost model
    would pick for the shape."""
    old = sg.set_tc_policy(request.param)
    yield request.param
    sg.set_tc_policy(old)


@pytest.fixture
def tc_always():
    old = sg.set_tc_policy("always")
    yield
    sg.set_tc_policy(old)


@pytest.mark.parametrize("n", [1, 97, 4133, 70001])
@pytest.mark.parametrize("i,s", [(1, 1), (1, 120), (5, 7), (13, 12), (8, 33), (9, 32),
                                 (33, 65), (121, 120), (241, 17)])
def test_block_dot_matches_definition(solver, tc_path, n, i, s):
    rng = np.random.default_rng(100 * i + s)
    ld = n + (7 if n > 1 else 0)
    Q = rng.standard_normal((i, ld))
    X = rng.standard_normal((s, ld))
    Wt = host(_block_dot(solver, Q, X, n))
    ref = Q[:, :n] @ X[:, :n].T        # (i, s): Q^T X in column-major terms
    scale = np.abs(Q[:, :n]) @ np.abs(X[:, :n]).T
    assert np.all(np.abs(Wt.T - ref) <= 1e-14 * scale + 1e-300)


def _even_ld(A, fill=0.0):
    """A (k, n) copied into rows of an even length (16-byte strides, which
    the tensor-core forms need), the padding set to `fill`."""
    k, n = A.shape
    out = np.full((k, n + (n & 1)), fill)
    out[:, :n] = A
    return out


def _block_dot(solver, Q, X, n, sym=False):
    i, ld = Q.shape
    s = i if sym else X.shape[0]
    Qd = dev(Q)
    Xd = Qd if sym else dev(X)
    W = torch.empty((s, i), dtype=torch.float64, device=DEV)
    import ctypes as C
    rc = sg.lib.sg_block_dot(solver._h, n, C.c_void_p(Qd.data_ptr()), ld, i,
                             C.c_void_p(Xd.data_ptr()), ld, s,
                             C.c_void_p(W.data_ptr()), i, 1 if sym else 0,
                             sg._stream_ptr())
    assert rc == 0, sg.lib.sg_last_error(solver._h)
    return W


@pytest.mark.parametrize("n,i,s", [(70001, 107, 106), (4133, 241, 17), (9000, 3, 130)])
def test_block_dot_fp64_tensor_cores_exact_on_integers(solver, tc_always, n, i, s):
    """The FP64 block dot on the tensor cores (8-bit digit slices, exact
    level sums) returns exact dot products: integer inputs of magnitude up
    to 2^15 have exact FP64 dot products (< 2^53), and every entry must
    equal numpy's exactly.  Columns of very different magnitudes (2^-40 ..
    2^40 scaling) check the per-column exponents."""
    rng = np.random.default_rng(n + i + s)
    Q = rng.integers(-2 ** 15, 2 ** 15, size=(i, n)).astype(np.float64)
    X = rng.integers(-2 ** 15, 2 ** 15, size=(s, n)).astype(np.float64)
    Q *= np.exp2(rng.integers(-40, 41, size=(i, 1)))
    X *= np.exp2(rng.integers(-40, 41, size=(s, 1)))
    Wt = host(_block_dot(solver, _even_ld(Q), _even_ld(X), n))
    assert np.array_equal(Wt.T, Q @ X.T)
    G = host(_block_dot(solver, _even_ld(X), None, n, sym=True))
    assert np.array_equal(G, X @ X.T)


@pytest.mark.parametrize("n,s", [(4133, 1), (70001, 12), (4133, 21), (4133, 31), (70001, 64),
                                 (3001, 120)])
def test_block_dot_symmetric_gram(solver, tc_path, n, s):
    rng = np.random.default_rng(s)
    X = rng.standard_normal((s, n))
    G = host(_block_dot(solver, _even_ld(X), None, n, sym=True))
    ref = X @ X.T
    assert np.array_equal(G, G.T)
    assert np.allclose(G, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("n", [1, 63, 64, 65, 5000, 70001])
@pytest.mark.parametrize("i,s,upper", [(1, 1, False), (3, 120, False),
                                       (121, 40, False), (33, 33, True),
                                       (120, 120, True), (7, 7, True)])
def test_block_update_matches_definition(solver, tc_path, n, i, s, upper):
    rng = np.random.default_rng(n + i + s)
    Q = rng.standard_normal((i, n))
    Wm = rng.standard_normal((i, s))          # i x s
    if upper:
        Wm = np.triu(Wm) + np.tril(np.full((i, s), np.nan), -1)
    X = rng.standard_normal((s, n))
    Wt = dev(np.ascontiguousarray(Wm.T))      # (s, i) = column-major i x s
    Xd = dev(_even_ld(X, np.inf))
    solver.block_update(dev(_even_ld(Q)), Wt, Xd, alpha=-0.7,
                        beta=1.3 if not upper else 0.0, upper=upper, n=n)
    Wz = np.nan_to_num(Wm, nan=0.0)
    ref = (1.3 if not upper else 0.0) * X + (-0.7) * (Q.T @ Wz).T
    scale = np.abs(X) + 0.7 * (np.abs(Q).T @ np.abs(Wz)).T
    got = host(Xd)
    assert np.all(np.abs(got[:, :n] - ref) <= 1e-14 * scale + 1e-300)
    assert np.all(got[:, n:] == np.inf)       # rows past n untouched


@pytest.mark.parametrize("n,i,s,upper", [(70001, 107, 106, False), (9000, 241, 40, False),
                                         (20000, 120, 120, True), (4133, 64, 33, False),
                                         (513, 1, 1, False), (600, 17, 5, False),
                                         (1000, 33, 33, True), (2049, 16, 70, False)])
def test_block_update_fp64_tensor_cores_exact_on_integers(solver, tc_always, n, i, s, upper):
    """The FP64 block update on the tensor cores (Q's digits relative to its
    column exponents, W' = W 2^(e_k) cut relative to its own column
    exponents) is exact: integer Q and W with per-column scales 2^-30 ..
    2^30 (Q) and 2^-20 .. 2^20 (W rows, so that every product of an output
    has one scale) give X = X - Q W equal to numpy's exact result, bit for
    bit; the upper form skips W's lower triangle (NaN there)."""
    rng = np.random.default_rng(3 * n + i + s)
    Q = rng.integers(-2 ** 12, 2 ** 12, size=(i, n)).astype(np.float64)
    Wm = rng.integers(-2 ** 12, 2 ** 12, size=(i, s)).astype(np.float64)
    X = rng.integers(-2 ** 20, 2 ** 20, size=(s, n)).astype(np.float64)
    sc = rng.integers(-30, 31, size=i)
    Q *= np.exp2(sc)[:, None]
    Wm *= np.exp2(-sc)[:, None]            # Q[r,k] W[k,c]: one scale per output
    Wm *= np.exp2(rng.integers(-20, 21, size=s))[None, :]
    if upper:
        Wm = np.triu(Wm) + np.tril(np.full((i, s), np.nan), -1)
    Wz = np.nan_to_num(Wm, nan=0.0)
    Xd = dev(_even_ld(X, np.inf))
    solver.block_update(dev(_even_ld(Q)), dev(np.ascontiguousarray(Wm.T)), Xd, alpha=-1.0,
                        beta=1.0, upper=upper, n=n)
    ref = X - (Q.T @ Wz).T
    got = host(Xd)
    assert np.array_equal(got[:, :n], ref)
    assert np.all(got[:, n:] == np.inf)


@pytest.mark.parametrize("n", [97, 4133, 70001])
@pytest.mark.parametrize("i,s", [(1, 120), (5, 7), (9, 6), (33, 65), (121, 40)])
def test_block_dot_f32_matches_definition(solver, n, i, s):
    """FP32 projections accumulate in FP32 per 32-row stage with a
    compensated fold: error within a few FP32 roundings of sum |q||x|."""
    rng = np.random.default_rng(300 + i + s)
    Q = rng.standard_normal((i, n)).astype(np.float32)
    X = rng.standard_normal((s, n)).astype(np.float32)
    solver.n = n
    Wt = host(solver.block_dot32(dev(Q, torch.float32), dev(X, torch.float32)))
    ref = Q.astype(np.float64) @ X.astype(np.float64).T
    scale = np.abs(Q.astype(np.float64)) @ np.abs(X.astype(np.float64)).T
    assert np.all(np.abs(Wt.T - ref) <= 64 * 2.0 ** -24 * scale)


@pytest.mark.parametrize("n", [256, 4133, 70001, 1 << 20])
@pytest.mark.parametrize("i,s", [(1, 1), (7, 16), (33, 120), (107, 106),
                                 (128, 128), (241, 17), (240, 106)])
def test_block_dot_f32_tensor_cores(solver, n, i, s):
    """Aligned leading dimensions take the TMA + tcgen05 path (TF32 hi/lo
    split, three products) from n = 512 rows on (n = 256 stays on the FFMA
    path); an unaligned copy of the same data takes the FFMA path.  Both must sit within a few FP32 roundings of the FP64
    product (the dropped lo*lo term is ~2^-22 of |q||x|)."""
    rng = np.random.default_rng(500 + i + s)
    ld_tc = (n + 3) // 4 * 4
    Q = np.zeros((i, ld_tc), np.float32)
    X = np.zeros((s, ld_tc), np.float32)
    Q[:, :n] = rng.standard_normal((i, n))
    X[:, :n] = rng.standard_normal((s, n))
    solver.n = n
    W_tc = host(solver.block_dot32(dev(Q, torch.float32), dev(X, torch.float32)))
    Qu = np.zeros((i, n + 1), np.float32)
    Xu = np.zeros((s, n + 1), np.float32)
    Qu[:, :n], Xu[:, :n] = Q[:, :n], X[:, :n]
    W_si = host(solver.block_dot32(dev(Qu, torch.float32), dev(Xu, torch.float32)))
    Q64, X64 = Q[:, :n].astype(np.float64), X[:, :n].astype(np.float64)
    ref = Q64 @ X64.T
    scale = np.abs(Q64) @ np.abs(X64).T
    for Wt in (W_tc, W_si):
        err = np.abs(Wt.T - ref)
        assert np.all(err <= 2.0 ** -18 * scale), (err / scale).max()


@pytest.mark.parametrize("n,s", [(1, 5), (70001, 1), (4133, 6), (70001, 33), (70001, 120),
                                 (4133, 130)])
def test_gram_f32_is_nearly_exact(solver, tc_path, n, s):
    """The FP32 Gram uses exact products: on the FP32 pipe with two-sum
    accumulation, on the tensor cores from exact digit slices.  Either way
    its error is at the eps_32^2 level relative to sum |x_k y_k| for data
    without extreme dynamic range.  Up to 128 columns the triangle kernel
    (or the tensor-core Gram, from 256 rows) computes it (one row, one
    column and a partial last 4 x 4 block included); 130 columns take the
    square-tile kernel."""
    rng = np.random.default_rng(400 + s)
    X = rng.standard_normal((s, n)).astype(np.float32)
    Xd = dev(X, torch.float32)
    solver.n = n
    G = host(solver.block_dot32(Xd, Xd, sym=True))
    X64 = X.astype(np.float64)
    ref = X64 @ X64.T
    scale = np.abs(X64) @ np.abs(X64).T
    assert np.all(np.abs(G - ref) <= 1e-12 * scale)


def _gram32(solver, X, n):
    """G = X^T X of the FP32 columns X (s, ld) through the C ABI."""
    Xd = dev(X, torch.float32)
    solver.n = n
    return host(solver.block_dot32(Xd, Xd, sym=True)).T


GRAM32_SHAPES = [(256, 1), (257, 7), (4133, 32), (4133, 33), (70001, 64), (70001, 100),
                 (70001, 106), (70001, 128), ((1 << 20) + 3, 106)]


@pytest.mark.parametrize("n,s", GRAM32_SHAPES)
def test_gram_f32_tensor_cores_exact_on_integers(solver, tc_always, n, s):
    """Integers of at most 11 bits are exact in six digit slices (every
    value within 2^23 of its column's largest), their products and level
    sums are exact, and the Gram entries (< 2^53) round exactly: the
    tensor-core Gram must equal X^T X bit for bit.  The shapes cover one
    to four quarters of 32 output columns, a ragged last stage and splits
    of many 128-row groups."""
    rng = np.random.default_rng(n + 31 * s)
    ld = (n + 3) // 4 * 4                      # 16-byte column stride for TMA
    X = np.zeros((s, ld), dtype=np.float32)
    X[:, :n] = rng.integers(-1000, 1001, size=(s, n))
    X[:, n:] = 7.0                             # padding rows must not count
    G = _gram32(solver, X, n)
    X64 = X[:, :n].astype(np.float64)
    assert np.array_equal(G, X64 @ X64.T)


@pytest.mark.parametrize("n,s", [(4133, 33), (70001, 106), (70001, 128)])
def test_gram_f32_tensor_cores_error_bound(solver, tc_always, n, s):
    """Columns scaled over 2^-40 .. 2^40, some with single large outliers,
    one all zero: each value is kept to 2^-47 of its column's largest
    (six base-256 digits) and the digit pairs of levels above 7 are left
    out, so entry (a, b) is within
    2^-46 (max|x_a| sum|x_b| + max|x_b| sum|x_a|) + n 2^-58 max|x_a| max|x_b|
    of X^T X, plus the final rounding."""
    rng = np.random.default_rng(7 * n + s)
    ld = (n + 3) // 4 * 4
    X = np.zeros((s, ld), dtype=np.float32)
    scales = 2.0 ** rng.uniform(-40, 40, size=s)
    X[:, :n] = rng.standard_normal((s, n)) * scales[:, None]
    for c in range(0, s, 5):                   # outliers 2^10 .. 2^20 above the rest
        X[c, rng.integers(0, n)] *= 2.0 ** rng.uniform(10, 20)
    X[s // 2, :] = 0.0
    G = _gram32(solver, X, n)
    X64 = X[:, :n].astype(np.float64)
    ref = X64 @ X64.T
    A = np.abs(X64)
    mx = A.max(axis=1)
    sm = A.sum(axis=1)
    bound = (2.0 ** -46 * (np.outer(mx, sm) + np.outer(sm, mx)) + n * 2.0 ** -58 * np.outer(mx, mx)
             + 2.0 ** -52 * np.abs(ref))
    # the FP64 reference itself carries n u sum|x_a x_b|
    bound += 2 * n * 2.0 ** -53 * (A @ A.T)
    assert np.all(np.abs(G - ref) <= bound)
    assert np.all(G[s // 2, :] == 0.0) and np.all(G[:, s // 2] == 0.0)
    assert np.array_equal(G, G.T)


def test_gram_f32_tensor_cores_non_finite_column(solver, tc_always):
    """An Inf or NaN in a column makes that column's row and column of the
    Gram NaN (so the Cholesky of CholQR stops), and leaves the rest exact."""
    n, s = 4133, 40
    rng = np.random.default_rng(11)
    X = rng.integers(-100, 101, size=(s, 4136)).astype(np.float32)
    X[3, 1000] = np.inf
    X[17, 5] = np.nan
    G = _gram32(solver, X, n)
    bad = np.zeros(s, dtype=bool)
    bad[[3, 17]] = True
    assert np.all(np.isnan(G[bad, :])) and np.all(np.isnan(G[:, bad]))
    X64 = X[~bad, :n].astype(np.float64)
    assert np.array_equal(G[np.ix_(~bad, ~bad)], X64 @ X64.T)


@pytest.mark.parametrize("n", [65, 70001])
@pytest.mark.parametrize("i,s,upper", [(3, 6, False), (121, 40, False), (33, 33, True)])
def test_block_update_f32_matches_definition(solver, n, i, s, upper):
    rng = np.random.default_rng(n + 7 * i + s)
    Q = rng.standard_normal((i, n)).astype(np.float32)
    Wm = rng.standard_normal((i, s))
    if upper:
        Wm = np.triu(Wm)
    X = rng.standard_normal((s, n)).astype(np.float32)
    Xd = dev(X, torch.float32)
    solver.block_update32(dev(Q, torch.float32), dev(np.ascontiguousarray(Wm.T)), Xd,
                          alpha=-0.7, beta=0.0 if upper else 1.3, upper=upper, n=n)
    ref = (0.0 if upper else 1.3) * X.astype(np.float64) - 0.7 * (Q.astype(np.float64).T @ Wm).T
    scale = np.abs(X) + 0.7 * (np.abs(Q.astype(np.float64)).T @ np.abs(Wm)).T
    assert np.all(np.abs(host(Xd) - ref) <= 64 * 2.0 ** -24 * scale)


@pytest.mark.parametrize("n", [128, 4133, 70001, 1 << 20])
@pytest.mark.parametrize("i,s,upper", [(1, 1, False), (7, 16, False), (33, 120, False),
                                       (107, 106, False), (128, 128, False),
                                       (200, 44, False), (241, 17, False), (241, 106, False),
                                       (33, 33, True), (120, 120, True)])
def test_block_update_f32_tensor_cores(solver, n, i, s, upper):
    """Aligned leading dimensions take the TMA + tcgen05 update (Q tile as an
    MN-major operand, TF32 hi/lo split); an unaligned copy of the same data
    takes the FFMA path.  Both within a few FP32 roundings of the FP64
    result.  W's chunks stay resident in shared memory up to (128, 128) and
    (200, 44); (241, 106) re-fetches them every stage."""
    rng = np.random.default_rng(900 + i + s + n % 97)
    ld = (n + 3) // 4 * 4
    Q = np.zeros((i, ld), np.float32)
    Q[:, :n] = rng.standard_normal((i, n))
    Wm = rng.standard_normal((i, s))
    if upper:
        Wm = np.triu(Wm) + np.tril(np.full((i, s), np.nan), -1)
    X = np.zeros((s, ld), np.float32)
    X[:, :n] = rng.standard_normal((s, n))
    beta = 0.0 if upper else 1.3
    Wz = np.nan_to_num(Wm, nan=0.0)
    Q64, X64 = Q[:, :n].astype(np.float64), X[:, :n].astype(np.float64)
    ref = beta * X64 - 0.7 * (Q64.T @ Wz).T
    scale = np.abs(X64) * abs(beta) + 0.7 * (np.abs(Q64).T @ np.abs(Wz)).T
    Wt = dev(np.ascontiguousarray(Wm.T))
    Xd = dev(X, torch.float32)
    solver.block_update32(dev(Q, torch.float32), Wt, Xd, alpha=-0.7, beta=beta,
                          upper=upper, n=n)
    Xu = np.zeros((s, n + 1), np.float32)
    Xu[:, :n] = X[:, :n]
    Qu = np.zeros((i, n + 1), np.float32)
    Qu[:, :n] = Q[:, :n]
    Xud = dev(Xu, torch.float32)
    solver.block_update32(dev(Qu, torch.float32), Wt, Xud, alpha=-0.7, beta=beta,
                          upper=upper, n=n)
    for got in (host(Xd)[:, :n], host(Xud)[:, :n]):
        err = np.abs(got - ref)
        assert np.all(err <= 2.0 ** -18 * scale + 1e-30), (err / (scale + 1e-30)).max()


def test_nrm2(solver):
    x = np.random.default_rng(5).standard_normal(123457)
    assert solver.nrm2(dev(x)) == pytest.approx(np.linalg.norm(x), rel=1e-14)


# ------------------------------------------------------------ whole solves
def residual_floor(A, b, x, x0=None):
    """Rounding floor of a true relative residual ||b - A x|| / ||b - A x0||
    in FP64: evaluating b - A x costs up to k+1 roundings per row (k = the
    longest row), and each component of x itself carries up to ~10
    roundings from its update x += Q y, so two correct runs can differ by
    2 (k + 11) u || |b| + |A||x| || / beta0."""
    op = O.as_operator(A)
    k = int(np.max(np.diff(op.indptr)))
    u = 2.0 ** -53
    x0 = np.zeros_like(b) if x0 is None else x0
    beta0 = np.linalg.norm(b - op @ x0)
    return 2 * (k + 11) * u * np.linalg.norm(np.abs(b) + abs(op) @ np.abs(x)) / beta0


def _compare(res_o, x_g, info, A, b, x0=None, xrel=1e-9, crel=1e-8, hrel=1e-6):
    """Decisions identical; per-cycle true residuals within 1e-8 relative
    (or the FP64 evaluation floor); x within 1e-9 relative."""
    assert info.s0 == res_o.s0
    assert list(info.s_hist) == list(res_o.s_hist)
    assert list(info.p1_hist) == list(res_o.p1_hist)
    assert list(info.s_eff_hist) == list(res_o.s_eff_hist)
    assert info.iters == res_o.iters and info.restarts == res_o.restarts
    assert list(info.cycle_iters) == list(res_o.cycle_iters)
    assert info.converged == res_o.converged
    floor = residual_floor(A, b, res_o.x, x0)
    co = np.array(res_o.cycle_relres)
    dc = np.abs(info.cycle_relres - co)
    assert np.all(dc <= np.maximum(crel * co, floor)), (dc, co, floor)
    ho = np.array(res_o.relres_hist)
    assert info.relres_hist.size == ho.size
    dh = np.abs(info.relres_hist - ho)
    assert np.all(dh <= np.maximum(hrel * ho, floor)), (dh.max(), floor)
    err = np.linalg.norm(x_g - res_o.x) / np.linalg.norm(res_o.x)
    assert err <= xrel, err


def test_solve_c1_matches_oracle(solver):
    c = W.config_c1()
    _analyze(solver, c["A"])
    ro = O.adaptive_sgmres(c["A"], c["b"], m=c["m"], s=c["s"], tol=c["tol"])
    x, info = solver.solve(c["b"], m=c["m"], s=c["s"], tol=c["tol"])
    assert info.converged and info.final_relres <= 1e-10
    _compare(ro, x, info, c["A"], c["b"])
    # Ritz values and scaling coefficients agree too
    assert np.allclose(info.ritz, ro.ritz, rtol=1e-9)
    assert np.allclose(info.gamma, ro.gamma, rtol=1e-9)


def test_solve_device_vectors_and_x0(solver):
    c = W.config_c1(40)
    _analyze(solver, c["A"])
    x0 = np.random.default_rng(3).uniform(-1, 1, c["A"].n)
    ro = O.adaptive_sgmres(c["A"], c["b"], x0=x0, m=50, s=8, tol=1e-10)
    xd, info = solver.solve(dev(c["b"]), x0=dev(x0), m=50, s=8, tol=1e-10)
    _compare(ro, host(xd), info, c["A"], c["b"], x0)


def test_solve_estimator_c2_small(solver):
    c = W.config_c2(16)
    _analyze(solver, c["A"])
    ro = O.adaptive_sgmres(c["A"], c["b"], m=80, s=0, s_min=4, s_max=40, tol=1e-10)
    x, info = solver.solve(c["b"], m=80, s=0, s_min=4, s_max=40, tol=1e-10)
    _compare(ro, x, info, c["A"], c["b"])


@pytest.mark.parametrize("s", [0, 6])
def test_solve_with_supplied_ritz_values(solver, s):
    """Ritz values supplied through sg_opts replace the pre-pass (Sec. 3.4):
    given the oracle's Ritz values (in any order: they are Leja-ordered),
    the solve takes the oracle's decisions, estimated (s = 0) or fixed."""
    c = W.config_c2(14)
    _analyze(solver, c["A"])
    kw = dict(m=60, s=s, s_min=3, s_max=24, tol=1e-10)
    ro = O.adaptive_sgmres(c["A"], c["b"], **kw)
    shuffled = ro.ritz[np.random.default_rng(2).permutation(ro.ritz.size)]
    ro2 = O.adaptive_sgmres(c["A"], c["b"], ritz=shuffled, **kw)
    x, info = solver.solve(c["b"], ritz=shuffled, **kw)
    assert np.array_equal(info.ritz, ro2.ritz)
    _compare(ro2, x, info, c["A"], c["b"])
    assert info.times_ms["prepass"] < 1.0


def test_supplied_ritz_values_are_validated(solver):
    c = W.config_c1(8)
    _analyze(solver, c["A"])
    for bad in ([1.0 + 2.0j, 3.0], [np.nan, 1.0]):
        with pytest.raises(sg.SgError):
            solver.solve(c["b"], m=20, s=4, ritz=np.array(bad))


@pytest.mark.parametrize("basis", ["newton", "monomial"])
def test_solve_other_bases(solver, basis):
    c = W.config_c1(24)
    _analyze(solver, c["A"])
    ro = O.adaptive_sgmres(c["A"], c["b"], m=40, s=6, tol=1e-10, basis=basis)
    x, info = solver.solve(c["b"], m=40, s=6, tol=1e-10, basis=basis)
    _compare(ro, x, info, c["A"], c["b"])


def _xrel_from_residuals(A, b, x, relres):
    """Two solutions whose residuals are both <= relres ||b|| differ by at
    most 2 relres ||A^-1|| ||b||: the x tolerance when the two sides use
    differently rounded (equilibrated) matrices."""
    Ad = O.as_operator(A).toarray()
    inv = 1.0 / np.linalg.svd(Ad, compute_uv=False)[-1]
    return 2.0 * relres * inv * np.linalg.norm(b) / np.linalg.norm(x)


@pytest.mark.parametrize("mode,basis,s,grid", [
    ("scalar", "monomial", 6, "c1"), ("scalar", "newton", 6, "c1"),
    ("scalar", "scaled_newton", 10, "c1"),
    ("column", "scaled_newton", 20, "aniso"), ("column", "monomial", 6, "aniso")])
def test_equilibrated_solve_matches_oracle(solver, mode, basis, s, grid):
    """Eq. (equil): scalar scaling (gamma = max|theta| for the monomial and
    Newton bases, no change for scaled Newton, as Sec. 4.3 states) gives
    the oracle's decisions and solution; column scaling (A D_c y = b,
    x = D_c y) too, with D_c rounded independently on each side, so x is
    held to the residual-implied bound.  (On the 24^2 anisotropic matrix a
    partial-Cholesky kappa lands within rounding of Omega at s = 20, so the
    scalar cases use the 24^2 nonsymmetric stencil, as the basis tests do.)"""
    if grid == "c1":
        c = W.config_c1(24)
        A, rng = c["A"], np.random.default_rng(17)
    else:
        A, rng = W.aniso2d(24)
    b = rng.uniform(-1, 1, A.n)
    x0 = rng.uniform(-0.1, 0.1, A.n)
    _analyze(solver, A)
    kw = dict(m=40 if grid == "c1" else 60, s=s, tol=1e-10, basis=basis)
    ro, _ = O.equilibrated_sgmres(A, b, mode, x0=x0, **kw)
    x, info = solver.solve(b, x0=x0, equilibrate=mode, **kw)
    assert info.converged
    xrel = 1e-9 if mode == "scalar" else max(1e-9, _xrel_from_residuals(A, b, ro.x, 1e-10))
    _compare(ro, x, info, A, b, x0=x0, xrel=xrel)


def test_column_equilibration_rejects_adjoint_and_follows_value_updates(solver):
    A, rng = W.aniso2d(16)
    b = rng.uniform(-1, 1, A.n)
    _analyze(solver, A)
    with pytest.raises(sg.SgError):
        solver.solve_adjoint(b, m=40, s=8, tol=1e-10, equilibrate="column")
    new = W.aniso2d(16, seed=11)[0].val   # same pattern, other conductivities
    solver.update_values(new)
    A2 = W.CSR(A.n, A.rowptr, A.colind, new)
    ro, _ = O.equilibrated_sgmres(A2, b, "column", m=40, s=8, tol=1e-10)
    x, info = solver.solve(b, m=40, s=8, tol=1e-10, equilibrate="column")
    assert info.converged and ro.converged
    _compare(ro, x, info, A2, b, xrel=max(1e-9, _xrel_from_residuals(A2, b, ro.x, 1e-10)))


def test_solve_paper_test1_monomial_s6(solver):
    lam = np.linspace(0.1, 10.0, 10000)
    A = W.diagonal(lam)
    b = np.ones(10000) / 100.0
    _analyze(solver, A)
    ro = O.adaptive_sgmres(A, b, m=100, s=10, tol=1e-10, basis="monomial")
    x, info = solver.solve(b, m=100, s=10, tol=1e-10, basis="monomial")
    assert info.s_hist[0] == 6
    _compare(ro, x, info, A, b)


def test_solve_paper_test3_scaled_newton_s100(solver):
    lam = np.linspace(0.1, 10.0, 10000)
    A = W.diagonal(lam)
    b = np.ones(10000) / 100.0
    _analyze(solver, A)
    ro = O.adaptive_sgmres(A, b, m=100, s=100, tol=1e-10)
    x, info = solver.solve(b, m=100, s=100, tol=1e-10)
    assert info.s_hist[0] == 100
    _compare(ro, x, info, A, b)


def test_solve_s1_matches_mgs_gmres(solver):
    c = W.config_c1(20)
    _analyze(solver, c["A"])
    g = O.mgs_gmres(c["A"], c["b"], m=30, tol=1e-10)
    x, info = solver.solve(c["b"], m=30, s=1, tol=1e-10)
    assert info.iters == g.iters
    assert np.max(np.abs(info.relres_hist - np.array(g.relres_hist))) <= 1e-12


def test_solve_complex_spectrum(solver):
    import scipy.sparse as sp
    rng = np.random.default_rng(9)
    nb = 300
    a, bb = rng.uniform(1.0, 4.0, nb), rng.uniform(0.2, 1.5, nb)
    blocks = [sp.csr_matrix(np.array([[a[k], bb[k]], [-bb[k], a[k]]]))
              for k in range(nb)]
    S = sp.csr_matrix(sp.block_diag(blocks, format="csr"))
    S.sort_indices()
    A = W.CSR(S.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data)
    b = rng.uniform(-1, 1, A.n)
    _analyze(solver, A)
    ro = O.adaptive_sgmres(A, b, m=80, s=12, tol=1e-10)
    x, info = solver.solve(b, m=80, s=12, tol=1e-10)
    assert np.any(np.abs(info.ritz.imag) > 1e-3)
    _compare(ro, x, info, A, b)


def test_solve_random_band_small(solver):
    A, rng = W.random_band(20000, k=24, band=4096)
    xs = W.uniform_vector(A.n, rng)
    b = W.rhs_from_solution(A, xs)
    _analyze(solver, A)
    ro = O.adaptive_sgmres(A, b, m=60, s=0, s_max=40, tol=1e-10)
    x, info = solver.solve(b, m=60, s=0, s_max=40, tol=1e-10)
    _compare(ro, x, info, A, b)


def test_solve_zero_rhs_and_tiny(solver):
    c = W.config_c1(6)
    _analyze(solver, c["A"])
    x, info = solver.solve(np.zeros(36), m=10, s=3)
    assert info.converged and np.all(x == 0) and info.iters == 0
    rng = np.random.default_rng(8)
    import scipy.sparse as sp
    Ad = rng.standard_normal((25, 25)) + 8 * np.eye(25)
    S = sp.csr_matrix(Ad)
    A = W.CSR(25, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data)
    b = rng.standard_normal(25)
    _analyze(solver, A)
    x, info = solver.solve(b, m=25, s=5, tol=1e-13)
    xs = O.dense_solve(A, b)
    assert info.iters <= 25
    assert np.linalg.norm(x - xs) <= np.linalg.cond(Ad) * 1e-14 * np.linalg.norm(xs)


def test_solve_max_iters_reports_noconv(solver):
    c = W.config_c1(32)
    _analyze(solver, c["A"])
    x, info = solver.solve(c["b"], m=20, s=5, tol=1e-14, max_iters=40)
    assert info.status == sg.SG_ENOCONV and not info.converged
    assert info.iters == 40


def test_invariant_subspace_ends_the_solve_exactly(solver):
    """A diagonal matrix with three distinct eigenvalues: the Krylov space
    has dimension 3, the Ritz pre-pass stops early (h_{j+1,j} ~ 0), the
    step size is capped by the Ritz values available, and the solve ends
    with a residual at rounding level, as in the oracle."""
    lam = np.repeat([1.0, 2.5, 4.0], 1000)
    A = W.diagonal(lam)
    b = np.random.default_rng(3).uniform(-1, 1, A.n)
    _analyze(solver, A)
    ro = O.adaptive_sgmres(A, b, m=20, s=8, tol=1e-12)
    x, info = solver.solve(b, m=20, s=8, tol=1e-12)
    assert info.converged and ro.converged
    assert info.s0 == ro.s0 == 3 and info.iters == ro.iters <= 4
    assert np.linalg.norm(x - b / lam) <= 1e-13 * np.linalg.norm(b / lam)


def test_nonfinite_rhs_is_reported_and_the_handle_recovers(solver):
    """Host-side fault injection: a NaN in b gives SG_ENUMERIC (no device
    trap), and the same handle then solves a clean system."""
    c = W.config_c1(16)
    _analyze(solver, c["A"])
    bad = c["b"].copy()
    bad[7] = np.nan
    with pytest.raises(sg.SgError) as e:
        solver.solve(bad, m=20, s=4, tol=1e-10)
    assert e.value.status == sg.SG_ENUMERIC
    x, info = solver.solve(c["b"], m=20, s=4, tol=1e-10)
    assert info.converged


def test_bounded_waits_time_out_and_leave_the_device_usable(solver):
    """Failure detection without a GPU fault: a grid barrier that expects
    one block too many and an mbarrier nothing arrives on both run out
    their 50 ms limit, set their error flags, return, and the context
    keeps working (a solve follows)."""
    import time
    t0 = time.perf_counter()
    gb, mb = sg.probe_bounded_waits(0, 50.0)
    dt = time.perf_counter() - t0
    assert gb and mb
    assert dt < 5.0
    c = W.config_c1(16)
    _analyze(solver, c["A"])
    x, info = solver.solve(c["b"], m=20, s=4, tol=1e-10)
    assert info.converged


def test_analyze_rejects_bad_csr(solver):
    with pytest.raises(sg.SgError):
        solver.analyze(np.array([0, 2, 1], np.int32), np.array([0, 1], np.int32),
                       np.array([1.0, 2.0]))
    with pytest.raises(sg.SgError):
        solver.analyze(np.array([0, 2, 3], np.int32), np.array([1, 0, 5], np.int32),
                       np.array([1.0, 2.0, 3.0]))


@pytest.mark.parametrize("rowptr,colind,what", [
    ([1, 2, 3, 3], [0, 1, 2], "rowptr must start at 0"),
    ([0, 2, 3, 4], [0, 1, 2], "end at nnz"),
    ([0, 2, 1, 3], [0, 1, 2], "non-decreasing"),
    ([0, 2, 9, 3], [0, 1, 2], "non-decreasing"),
    ([0, 2, 2, 3], [0, 3, 2], "out of range"),
    ([0, 2, 2, 3], [0, -1, 2], "out of range"),
    ([0, 2, 2, 3], [1, 0, 2], "sorted"),
    ([0, 2, 2, 3], [1, 1, 2], "sorted"),
])
def test_analyze_device_checks_keep_the_previous_matrix(solver, rowptr, colind, what):
    """The structure of a square CSR matrix is checked on the device after
    its copy (one thread per row; a row whose bounds fail is not read
    further); a rejected matrix names the failed check and leaves the
    previously analysed matrix in place."""
    c = W.config_c1(12)
    op = _analyze(solver, c["A"])
    with pytest.raises(sg.SgError, match=what):
        solver.analyze(np.array(rowptr, np.int32), np.array(colind, np.int32),
                       np.arange(1.0, len(colind) + 1.0))
    x, info = solver.solve(c["b"], m=30, s=4, tol=1e-10)
    assert info.converged
    assert np.linalg.norm(c["b"] - op @ np.asarray(x)) <= 1e-10 * np.linalg.norm(c["b"])


# ------------------------------------------------------------ adjoint path
def test_adjoint_solve_and_grad_values(solver):
    c = W.config_c1(30)
    A = c["A"]
    op = _analyze(solver, A)
    g = np.random.default_rng(4).uniform(-1, 1, A.n)
    AT = op.T.tocsr()
    AT.sort_indices()
    ro = O.adaptive_sgmres(AT, g, m=60, s=8, tol=1e-10)
    lam, info = solver.solve_adjoint(g, m=60, s=8, tol=1e-10)
    _compare(ro, lam, info, AT, g)
    x = np.random.default_rng(5).uniform(-1, 1, A.n)
    dval = host(solver.grad_values(dev(lam), dev(x)))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    assert np.allclose(dval, -lam[rows] * x[A.colind], rtol=0, atol=0)
    # A^T has A's eigenvalues: the adjoint solve from the forward solve's
    # Ritz values (the oracle's forward run's) skips its pre-pass and
    # follows the oracle given the same values
    fwd = O.adaptive_sgmres(A, c["b"], m=60, s=8, tol=1e-10)
    ro2 = O.adaptive_sgmres(AT, g, m=60, s=8, tol=1e-10, ritz=fwd.ritz)
    lam2, info2 = solver.solve_adjoint(g, m=60, s=8, tol=1e-10, ritz=fwd.ritz)
    assert info2.converged
    _compare(ro2, lam2, info2, AT, g)


# ------------------------------------------------------- FP32 basis + IR
def test_fp32_ir_reaches_fp64_accuracy(solver):
    c = W.config_c2(20)
    _analyze(solver, c["A"])
    x, info = solver.solve(c["b"], m=60, s=0, s_min=2, s_max=40, tol=1e-10,
                           precision="fp32_ir")
    assert info.converged and info.final_relres <= 1e-10
    op = O.as_operator(c["A"])
    rel = np.linalg.norm(c["b"] - op @ x) / np.linalg.norm(c["b"])
    assert rel <= 1e-10
    ro = O.adaptive_sgmres(c["A"], c["b"], m=60, s=0, s_min=2, s_max=40, tol=1e-10)
    err = np.linalg.norm(x - ro.x) / np.linalg.norm(ro.x)
    assert err <= 1e-8, err
    assert info.refinements >= 2


@pytest.mark.parametrize("case,k", [
    ("c2_16", 1), ("c2_16", 3), ("c2_16", 4), ("c2_16", 5), ("c2_16", 9),
    ("c2_16", 12), ("c1_45", 12)])
def test_fp32_prepass_ritz_values_follow_fp64_arnoldi(solver, case, k):
    """The FP32 pre-pass (all MGS coefficients of a step from the basis's
    Gram matrix, two grid barriers per step) gives the Ritz values of the
    FP64 MGS-Arnoldi oracle to FP32 accuracy.  16^3 = 4096 rows leaves CTAs
    with no rows; 45^2 = 2025 rows is not a multiple of 4 or 32.  Compared
    as sets (Leja order can swap near-ties).  Past a dozen steps the Ritz
    values of an FP32 Arnoldi drift from the FP64 ones by more than this
    tolerance whatever the orthogonalisation order (the last Krylov
    directions sink below FP32 rounding), so the wide bases are pinned by
    the exact Jacobi-matrix case below."""
    name, size = case.split("_")
    c = W.config_c2(int(size)) if name == "c2" else W.config_c1(int(size))
    _analyze(solver, c["A"])
    _, info = solver.solve(c["b"], m=40, s=k, tol=1e-10, precision="fp32_ir", max_iters=k)
    q = c["b"] / np.linalg.norm(c["b"])
    H, steps = O.arnoldi_mgs(O.as_operator(c["A"]), q, k)
    ref = O.ritz_values(H, steps)
    got = info.ritz
    assert got.size == ref.size
    scale = np.max(np.abs(ref))
    for z in ref:
        assert np.min(np.abs(got - z)) <= 2e-5 * scale, (z, got)


@pytest.mark.parametrize("precision,n,k", [
    ("fp32_ir", 2025, 33), ("fp32_ir", 4096, 100), ("fp32_ir", 884_737, 40),
    ("fp32_ir", 2025, 165), ("fp64", 2025, 70)])
def test_prepass_reproduces_jacobi_matrix(solver, precision, n, k):
    """Arnoldi from the head of a symmetric tridiagonal chain reproduces the
    chain's leading k x k block exactly (every entry, coupling and norm is
    exact in FP32 and FP64), so the pre-pass's Ritz values must equal the
    eigenvalues of that block to rounding, at any basis width.  The chain
    rows are spread over the whole matrix (stride 7919), so every CTA's
    partial sums and the cross-CTA reductions carry the nonzeros; the cases
    span more basis vectors than warps, several 4096-row chunks per CTA
    (884,737 rows, not a multiple of 4), and a basis past the 161 vectors of
    the two-barrier step (165)."""
    A, a, b = W.jacobi_chain(n)
    _analyze(solver, A)
    rhs = np.zeros(n)
    rhs[0] = 1.0
    _, info = solver.solve(rhs, m=max(40, k), s=k, tol=1e-10, precision=precision,
                           max_iters=k)
    T = np.diag(a[:k]) + np.diag(b[:k - 1], 1) + np.diag(b[:k - 1], -1)
    ref = np.linalg.eigvalsh(T)
    got = info.ritz
    assert got.size == k
    assert np.max(np.abs(got.imag)) <= 1e-12 * np.max(np.abs(ref))
    assert np.allclose(np.sort(got.real), ref, rtol=0, atol=1e-11 * np.max(np.abs(ref)))


ARNOLDI_CASES = {
    # one CTA (2025 rows), two CTAs of 2048 rows, 16 CTAs, and 151 CTAs
    # whose last one holds a ragged 1603 rows (rows per CTA rounded to 32)
    "stencil2d_45": lambda: W.stencil2d(45, 45),
    "stencil2d_64": lambda: W.stencil2d(64, 64),
    "convdiff3d_32": lambda: W.stencil3d_convdiff(32),
    "randband_400003": lambda: W.random_band(400_003, k=24, band=4096)[0],
}


@pytest.mark.parametrize("name", list(ARNOLDI_CASES))
@pytest.mark.parametrize("k", [1, 12])
def test_arnoldi_hessenberg_matches_oracle(solver, name, k):
    """sg_arnoldi (the Ritz pre-pass, Sec. 3.4) against the oracle's
    MGS-Arnoldi, entry by entry.  Two runs of MGS-Arnoldi that differ only
    in rounding order have Hessenberg columns j that differ by about
    u kappa(K_{j+2}) ||A||, K the normalised Krylov matrix [q, Aq, ...]
    (a first-order perturbation of its QR factor); the tolerance is 8 times
    that, and at least 1e-12 ||A||_1.  The first columns are thus held to
    a few ulps of ||A||, where a wrong projection would show at O(1)."""
    A = ARNOLDI_CASES[name]()
    op = _analyze(solver, A)
    q = np.random.default_rng(31).uniform(-1, 1, A.n)
    q /= np.linalg.norm(q)
    H, steps = solver.arnoldi(dev(q), k)
    Ho, so = O.arnoldi_mgs(op, q, k)
    assert steps == so == k
    anorm = abs(op).sum(axis=0).max()
    K = [q]
    for _ in range(k):
        v = op @ K[-1]
        K.append(v / np.linalg.norm(v))
    K = np.column_stack(K)
    for j in range(k):
        tol = max(8 * 2.0 ** -53 * np.linalg.cond(K[:, :j + 2]) * anorm, 1e-12 * anorm)
        assert np.all(np.abs(H[:, j] - Ho[:, j]) <= tol), (j, np.abs(H[:, j] - Ho[:, j]).max(), tol)


@pytest.mark.parametrize("n,k", [(2025, 70), (884_737, 40)])
def test_arnoldi_reproduces_jacobi_matrix_exactly(solver, n, k):
    """From the head of a symmetric tridiagonal chain, FP64 Arnoldi is
    Lanczos on a Jacobi matrix: every projection, coupling and norm is exact,
    so H equals the chain's leading block entry for entry (884,737 rows
    spread the chain over every CTA of the resident step)."""
    A, a, b = W.jacobi_chain(n)
    _analyze(solver, A)
    q = np.zeros(n)
    q[0] = 1.0
    H, steps = solver.arnoldi(dev(q), k)
    assert steps == k
    T = np.diag(a[:k]) + np.diag(b[:k - 1], 1) + np.diag(b[:k - 1], -1)
    assert np.array_equal(H[:k, :k], T) and H[k, k - 1] == b[k - 1]
    assert np.all(H[k, :k - 1] == 0.0)


def test_arnoldi_stops_at_an_invariant_subspace(solver):
    """A diagonal matrix with 5 distinct eigenvalues: the Krylov space of
    any start vector has dimension 5, so the pre-pass stops after 5 steps
    (h_65 below 1e-12 of ||A v_5||), like the oracle."""
    lam = np.repeat([1.0, 2.0, 3.5, 5.0, 8.0], 600)
    A = W.diagonal(lam)
    op = _analyze(solver, A)
    q = np.random.default_rng(5).uniform(-1, 1, A.n)
    q /= np.linalg.norm(q)
    _, steps = solver.arnoldi(dev(q), 9)
    _, so = O.arnoldi_mgs(op, q, 9)
    assert steps == so == 5


def test_arnoldi_rejects_bad_arguments(solver):
    A = W.stencil2d(8, 8)
    _analyze(solver, A)
    q = dev(np.ones(A.n) / 8.0)
    with pytest.raises(sg.SgError):
        solver.arnoldi(q, 0)
    with pytest.raises(sg.SgError):
        solver.arnoldi(q, 3, precision=7)


# ------------------------------------------------------ full-size workload
@pytest.mark.slow
def test_full_size_c2_sampled_and_converged(solver):
    c = W.config_c2()
    A = c["A"]
    op = _analyze(solver, A)
    rng = np.random.default_rng(31)
    x = rng.uniform(-1, 1, A.n)
    y = host(solver.spmv_newton(dev(x), 1.3, 2.1))
    rows = rng.choice(A.n, 2000, replace=False)
    for r in rows:
        a, e = A.rowptr[r], A.rowptr[r + 1]
        ref = (np.dot(A.val[a:e], x[A.colind[a:e]]) - 1.3 * x[r]) / 2.1
        assert abs(y[r] - ref) <= 1e-14 * (np.abs(A.val[a:e]) @ np.abs(x[A.colind[a:e]]) + 2)
    xs, info = solver.solve(c["b"], m=c["m"], s=0, s_min=c["s_min"],
                            s_max=c["s_max"], tol=c["tol"])
    assert info.converged
    rel = np.linalg.norm(c["b"] - op @ xs) / np.linalg.norm(c["b"])
    assert rel <= 1e-10
    assert c["s_min"] <= info.s0 <= c["s_max"]
    h = info.relres_hist
    k = 0
    for n_c in info.cycle_iters:
        seg = h[k:k + n_c]
        assert np.all(np.diff(seg) <= 1e-12 * seg[:-1])
        k += n_c


# ------------------------------------------------------------ gradients
def test_autograd_matches_dense_gradient_and_fd(solver):
    """Autograd through the solver (forward solve, adjoint solve, sampled
    outer product) against the oracle's dense gradient (1e-6 relative) and
    against central differences of the exact loss (dense LU) along 16 seeded
    directions with h = 1e-6."""
    from paper_2303_08953_gb300.autograd import sparse_solve
    A, rng = W.aniso2d(24)
    b = rng.uniform(-1, 1, A.n)
    xt = rng.uniform(-1, 1, A.n)
    solver.analyze_csr(A)
    opts = dict(m=600, s=8, tol=1e-13)
    vals = dev(A.val).requires_grad_(True)
    bt = dev(b).requires_grad_(True)
    x = sparse_solve(vals, bt, solver, **opts)
    L = 0.5 * ((x - dev(xt)) ** 2).sum()
    L.backward()
    L0, dv, db, _ = O.loss_gradients(A, b, xt)
    assert abs(L.item() - L0) <= 1e-9 * abs(L0)
    gv, gb = host(vals.grad), host(bt.grad)
    assert np.linalg.norm(gv - dv) <= 1e-6 * np.linalg.norm(dv)
    assert np.linalg.norm(gb - db) <= 1e-6 * np.linalg.norm(db)
    h = 1e-6
    for k in range(16):
        d = np.random.default_rng(100 + k).standard_normal(A.nnz)
        e = np.random.default_rng(200 + k).standard_normal(A.n)
        Ap = W.CSR(A.n, A.rowptr, A.colind, A.val + h * d)
        Am = W.CSR(A.n, A.rowptr, A.colind, A.val - h * d)
        fd = (O.loss_gradients(Ap, b + h * e, xt)[0]
              - O.loss_gradients(Am, b - h * e, xt)[0]) / (2 * h)
        an = gv @ d + gb @ e
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (k, fd, an)
