"""Pins of the CPU oracle against what the paper and the mathematics fix:
closed-form spectra, hand-computed small cases, invariants (Arnoldi
relation, orthogonality, GMRES monotonicity), textbook special cases (s = 1
is CGS2-GMRES, m >= N terminates, dense LU agreement) and the values the
paper prints for its worked examples (tests/golden/paper_pins.json).

The last group plants mistakes in the oracle (on the CPU) and checks that
some pin catches each of them.
"""
import json
import math
import os

import numpy as np
import scipy.sparse as sp
import pytest

import workloads as W
from oracle import sgmres_oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_pins.json")))


# ------------------------------------------------------------ generators
def test_generator_nnz_closed_forms():
    A = W.stencil2d(64, 64)
    assert A.n == 4096 and A.nnz == 5 * 4096 - 4 * 64 == 20224
    B = W.stencil3d_convdiff(16)
    assert B.nnz == 7 * 16 ** 3 - 6 * 16 ** 2
    C, _ = W.vardiff3d(12)
    assert C.nnz == 7 * 12 ** 3 - 6 * 12 ** 2
    D, _ = W.aniso2d(20)
    assert D.nnz == 5 * 400 - 4 * 20
    E, _ = W.random_band(50000, k=24, band=4096)
    assert E.nnz == 25 * 50000


def test_generator_row_sums_and_structure():
    A = W.stencil3d_convdiff(8).to_scipy()
    # interior row: 6 - 3*1.2 - 3*0.8 = 0; a corner row (0,0,0) has only
    # the three downwind neighbours: 6 - 3*0.8
    rs = np.asarray(A.sum(axis=1)).ravel()
    i_int = 3 + 8 * 3 + 64 * 3
    assert rs[i_int] == pytest.approx(0.0, abs=1e-14)
    assert rs[0] == pytest.approx(6 - 2.4)
    S = W.stencil2d(5, 4).to_scipy().toarray()
    assert S[6, 5] == -1.1 and S[6, 7] == -0.9      # west / east
    assert S[6, 1] == -1.1 and S[6, 11] == -0.9     # south / north
    D, _ = W.aniso2d(16)
    Ds = D.to_scipy()
    assert abs(Ds - Ds.T).max() == 0.0
    # diagonal = sum of 4 edge conductivities >= |off-diagonal row sum|
    d = Ds.diagonal()
    off = np.asarray(abs(Ds).sum(axis=1)).ravel() - d
    assert np.all(d >= off - 1e-12)
    E, _ = W.random_band(20000, k=24, band=4096)
    Es = E.to_scipy()
    d = Es.diagonal()
    off = np.asarray(abs(Es).sum(axis=1)).ravel() - np.abs(d)
    assert np.allclose(d, 1.1 * off)
    rows = np.repeat(np.arange(E.n), 25)
    assert np.all(np.abs(E.colind.astype(np.int64) - rows) <= 4096)
    assert np.all(np.diff(E.colind.reshape(-1, 25), axis=1) > 0)
    C, _ = W.vardiff3d(6, skew=0.1)
    Cs = C.to_scipy()
    K = (Cs - Cs.T) * 0.5
    nz = K.data[np.abs(K.data) > 0]
    assert np.allclose(np.abs(nz), 0.1)


def _stencil2d_eigs(nx, ny, d, w, e, s, n_):
    kx = np.arange(1, nx + 1)
    ky = np.arange(1, ny + 1)
    ex = 2 * math.sqrt(w * e) * np.cos(kx * np.pi / (nx + 1))
    ey = 2 * math.sqrt(s * n_) * np.cos(ky * np.pi / (ny + 1))
    return np.sort((d + ex[:, None] + ey[None, :]).ravel())


def test_stencil_spectrum_closed_form():
    """Separable nonsymmetric stencil with positive off-diagonal products:
    eigenvalues d + 2 sqrt(ac) cos(k pi/(n+1)) summed over the axes."""
    A = W.stencil2d(7, 5)
    ev = np.sort(np.linalg.eigvals(A.to_scipy().toarray()).real)
    assert np.allclose(ev, _stencil2d_eigs(7, 5, 4.0, -1.1, -0.9, -1.1, -0.9),
                       atol=1e-12)


def test_arnoldi_ritz_values_full_space():
    """k = N Arnoldi steps: the Ritz values are the eigenvalues."""
    A = W.stencil2d(4, 3)
    op = O.as_operator(A)
    q = np.random.default_rng(5).uniform(-1, 1, A.n)
    H, steps = O.arnoldi_mgs(op, q / np.linalg.norm(q), A.n)
    assert steps == A.n
    rv = np.sort(O.ritz_values(H, steps).real)
    ex = _stencil2d_eigs(4, 3, 4.0, -1.1, -0.9, -1.1, -0.9)
    assert np.allclose(rv, ex, atol=1e-10)


def test_arnoldi_reproduces_jacobi_matrix():
    """Arnoldi from the unit vector at the head of a symmetric tridiagonal
    chain is Lanczos on a Jacobi matrix: the basis is the chain's unit
    vectors, H is the leading block of the matrix itself (entries exact),
    and the Ritz values are the eigenvalues of that k x k block."""
    A, a, b = W.jacobi_chain(2025)
    q = np.zeros(A.n)
    q[0] = 1.0
    k = 40
    H, steps = O.arnoldi_mgs(O.as_operator(A), q, k)
    assert steps == k
    T = np.diag(a[:k]) + np.diag(b[:k - 1], 1) + np.diag(b[:k - 1], -1)
    assert np.array_equal(H[:k, :k], T) and H[k, k - 1] == b[k - 1]
    rv = np.sort(O.ritz_values(H, steps).real)
    assert np.allclose(rv, np.linalg.eigvalsh(T), rtol=0, atol=1e-12)


def test_mgs_coefficients_from_the_gram_matrix():
    """The FP32 pre-pass step takes all MGS coefficients of a step at once,
    h = (I + L)^-1 V^T w with L the strict lower triangle of V^T V.  That is
    exactly what MGS computes one projection at a time, h_k = v_k . (w -
    sum_{q<k} h_q v_q), for any basis, orthonormal or not: checked here in
    FP64 on a deliberately non-orthogonal basis, where a dropped or
    transposed Gram term would show at O(1)."""
    rng = np.random.default_rng(11)
    n, k = 500, 12
    V = rng.standard_normal((n, k))
    V /= np.linalg.norm(V, axis=0)
    V[:, 5] += 0.3 * V[:, 2]  # far from orthogonal
    w = rng.standard_normal(n)
    h_mgs = np.zeros(k)
    r = w.copy()
    for q in range(k):
        h_mgs[q] = V[:, q] @ r
        r -= h_mgs[q] * V[:, q]
    G = V.T @ V
    L = np.tril(G, -1)
    h_gram = np.linalg.solve(np.eye(k) + L, V.T @ w)
    assert np.allclose(h_gram, h_mgs, rtol=0, atol=1e-12 * np.linalg.norm(w))
    # the update with those coefficients is MGS's residual
    assert np.allclose(w - V @ h_gram, r, rtol=0, atol=1e-12 * np.linalg.norm(w))


def test_ritz_values_inside_field_of_values():
    """Ritz values lie in the field of values of A: their real parts are
    bounded by the extreme eigenvalues of the symmetric part (A + A^T)/2
    (for a non-normal A they may leave the spectral interval)."""
    A = W.stencil2d(16, 16)
    op = O.as_operator(A)
    q = np.ones(A.n) / 16.0
    H, steps = O.arnoldi_mgs(op, q, 10)
    Ad = op.toarray()
    fov = np.linalg.eigvalsh(0.5 * (Ad + Ad.T))
    rv = O.ritz_values(H, steps)
    assert np.all(rv.real >= fov[0] - 1e-10)
    assert np.all(rv.real <= fov[-1] + 1e-10)


# ------------------------------------------------------- Leja / gamma / E
def test_leja_real_hand_example():
    # |.| max -> 4; farthest from 4 -> 1; |x-4||x-1| ties (2 vs 3) -> larger
    # real part first -> 3; then 2.
    out = O.leja_order(np.array([2.0, 4.0, 1.0, 3.0]))
    assert np.array_equal(out.real, [4.0, 1.0, 3.0, 2.0])


def test_leja_complex_pair_adjacent():
    th = np.array([1 - 2j, 3.0, -2.0, 1 + 2j])
    out = O.leja_order(th)
    # start 3 (|3| largest); |-2-3| = 5 > |1+2i-3| = 2.83 -> -2; then pair
    assert np.allclose(out, [3.0, -2.0, 1 + 2j, 1 - 2j])


def test_scaling_coefficients_closed_form():
    th = np.array([4.0, 1.0, 1 + 2j, 1 - 2j])
    tbar = (4 + 1 + 1 + 1) / 4.0
    g = O.scaling_coefficients(th)
    assert np.allclose(g, [abs(tbar - 4), abs(tbar - 1), abs(tbar - 1 - 2j),
                           abs(tbar - 1 + 2j)])
    # degenerate: one Ritz value -> gamma = 0 -> replaced by 1
    assert O.scaling_coefficients(np.array([2.5]))[0] == 1.0
    # symmetric triple: the middle one has gamma 0 -> mean of the others
    g3 = O.scaling_coefficients(np.array([1.0, 2.0, 3.0]))
    assert np.allclose(g3, [1.0, 1.0, 1.0])


def test_estimator_two_values_by_hand():
    eps = 2.0 ** -53
    t1, t2 = 3.0, 1.0
    tbar = 2.0
    rho21 = abs(t2 - t1) / abs(tbar - t1)
    E = np.array([[eps, eps], [1.0, eps * rho21]])
    lg = O.estimator_log2_E(np.array([t1, t2]), eps)
    assert np.allclose(np.exp2(lg), E, rtol=1e-14, atol=0)
    nrm = O.estimator_column_norms(np.array([t1, t2]), eps)
    assert np.allclose(nrm, np.linalg.norm(E, axis=0), rtol=1e-14)


def test_estimator_three_values_by_hand():
    eps = 1e-3
    th = np.array([5.0, -1.0, 2.0])
    tbar = 2.0
    rho = lambda i, k: abs(th[i] - th[k]) / abs(tbar - th[k])
    E = np.empty((3, 3))
    for i in range(3):
        for j in range(3):
            ks = [k for k in range(j) if not (j > i and k == i)]
            pr = np.prod([rho(i, k) for k in ks]) if ks else 1.0
            E[i, j] = pr * (eps if j >= i else 1.0)
    assert np.allclose(np.exp2(O.estimator_log2_E(th, eps)), E, rtol=1e-13)


# Four real Ritz values in a Leja order with mean 0, so that
# rho(i,k) = |theta_i - theta_k| / |theta_k| takes the values 1/2, 1, 3/2, 2
# and 3.  E of Eq. (auxiliarymatrix) written out entry by entry by hand
# (rows i, columns j, both 1-based in the comments):
#   column 1: eps (i=1, j=i), then 1, 1, 1 (j < i: empty products)
#   column 2: eps (i=1 > ... j > i, product over k<2, k!=1: empty),
#             2 eps (i=2: rho(2,1)), 1/2 (rho(3,1)), 3/2 (rho(4,1))
#   column 3: 2 eps (rho(1,2)), 2 eps (rho(2,1)),
#             3/4 eps (rho(3,1) rho(3,2)), 3/4 (rho(4,1) rho(4,2))
#   column 4: 2 eps (rho(1,2) rho(1,3) = 2 * 1), 6 eps (rho(2,1) rho(2,3)),
#             3/4 eps (rho(3,1) rho(3,2)), 3/2 eps (rho(4,1..3) = 3/2*1/2*2)
LEJA4 = np.array([4.0, -4.0, 2.0, -2.0])


def _leja4_norms_by_hand(eps):
    return np.array([math.sqrt(3.0 + eps ** 2),
                     math.sqrt(0.25 + 2.25 + 5.0 * eps ** 2),
                     math.sqrt(0.5625 + 8.5625 * eps ** 2),
                     eps * math.sqrt(4.0 + 36.0 + 0.5625 + 2.25)])


def test_estimator_four_values_norms_by_hand():
    assert np.array_equal(O.leja_order(LEJA4[[2, 0, 3, 1]]).real, LEJA4)
    for eps in (0.1, 1e3, 2.0 ** -53):
        assert np.allclose(O.estimator_column_norms(LEJA4, eps),
                           _leja4_norms_by_hand(eps), rtol=1e-14, atol=0)


# (eps, Omega_est, s_min, s_max, s0*): s0* is the largest j such that every
# column l <= j has ||E_l|| < Omega_est (Sec. 3.5, first-crossing reading),
# then clamped to [s_min, s_max].
#   eps = 1e3: norms 1000.0015, 2236.07, 2926.17, 6543.09 (increasing)
#   eps = 0.1: norms 1.7349, 1.5969, 0.8053, 0.6543 (decreasing)
ESTIMATOR_EXACT = [
    (1e3, 2500.0, 1, None, 2),     # crossing at column 3
    (1e3, 3000.0, 1, None, 3),     # crossing at column 4
    (1e3, 2236.0, 1, None, 1),     # column 2 just above Omega_est
    (1e3, 2237.0, 1, None, 2),     # ... and just below
    (1e3, 7000.0, 1, None, 4),     # no crossing: every column
    (1e3, 7000.0, 1, 3, 3),        # clamped from above
    (1e3, 900.0, 1, None, 1),      # crossing at column 1: clamped to s_min
    (1e3, 900.0, 3, None, 3),      # clamped from below
    (1e3, 2500.0, 3, 4, 3),        # s_min above the crossing wins
    (0.1, 1.70, 1, None, 1),       # first column fails, later ones pass:
    (0.1, 1.70, 2, None, 2),       #   the first crossing decides, not the
    (0.1, 1.75, 1, None, 4),       #   last column below Omega_est
]


@pytest.mark.parametrize("eps,omega,smin,smax,want", ESTIMATOR_EXACT)
def test_estimator_first_crossing_and_clamp_exact(eps, omega, smin, smax, want):
    """Exact pin of the index s0* returns: any off-by-one (counting the
    crossing column, 0- vs 1-based j) or a last-below reading fails."""
    norms = _leja4_norms_by_hand(eps)
    # the thresholds sit clear of the norms, so rounding cannot move s0*
    assert np.min(np.abs(norms - omega)) > 1e-5 * omega
    s0, _ = O.estimate_step_size(LEJA4, omega_est=omega, eps=eps,
                                 s_min=smin, s_max=smax)
    assert s0 == want


@pytest.mark.parametrize("key", ["test8_estimator_uniform",
                                 "test8_estimator_lmax2000"])
def test_estimator_paper_test8(key):
    """Soft pin (paper's Test 8): the estimator's s0* and the column where
    kappa(V_1:j) passes 1e8, with Ritz values from a 200-step Arnoldi
    pre-pass from a ones start vector."""
    gd = GOLD[key]
    lam = np.linspace(1.0, 200.0, gd["n"])
    lam[-1] = gd["lam_max"]
    op = O.as_operator(W.diagonal(lam))
    q = np.ones(gd["n"]) / math.sqrt(gd["n"])
    H, steps = O.arnoldi_mgs(op, q, gd["n"])
    ritz = O.leja_order(O.ritz_values(H, steps))
    s0, _ = O.estimate_step_size(ritz, GOLD["omega"]["omega_est"])
    assert abs(s0 - gd["s0_star"]) <= gd["s0_star_tol"]
    th, gm = O.basis_shifts(O.BASIS_SCALED_NEWTON, ritz,
                            O.scaling_coefficients(ritz))
    kmax = min(gd["kappa_cross"] + gd["kappa_cross_tol"] + 2, gd["n"] - 1)
    V, _ = O.mpk(op, q, kmax, th, gm)
    cross = next(j for j in range(1, kmax + 2)
                 if np.linalg.cond(V[:, :j]) > 1e8)
    assert abs(cross - gd["kappa_cross"]) <= gd["kappa_cross_tol"]


# ------------------------------------------------------- partial Cholesky
def test_partial_cholesky_matches_cholesky_when_well_conditioned():
    X = np.random.default_rng(1).standard_normal((200, 12))
    G = X.T @ X
    p, R, kap = O.partial_cholesky(G)
    assert p == 12
    assert np.allclose(R, np.linalg.cholesky(G).T, rtol=1e-12, atol=1e-12)
    assert kap[0] == 1.0


def test_partial_cholesky_stops_at_nonpositive_pivot():
    G = np.diag([4.0, 1.0, -1.0, 1.0])
    p, R, _ = O.partial_cholesky(G)
    assert p == 2 and np.allclose(R, np.diag([2.0, 1.0]))
    # a singular Gram: column 3 equals column 1 -> pivot 0
    X = np.random.default_rng(2).standard_normal((50, 3))
    X[:, 2] = X[:, 0]
    p, _, _ = O.partial_cholesky(X.T @ X)
    assert p == 2
    # first pivot <= 0: nothing kept (happy breakdown)
    p, _, _ = O.partial_cholesky(np.zeros((3, 3)))
    assert p == 0


def test_partial_cholesky_kappa_ramp():
    """R = diag(10^0 .. 10^9): ICE is exact on a diagonal factor, kappa_j =
    10^(j-1), and the first column with kappa > 1e7 is excluded."""
    R = np.diag(10.0 ** np.arange(10))
    p, Rp, kap = O.partial_cholesky(R.T @ R, omega=1e7)
    assert p == 8
    assert np.allclose(kap, 10.0 ** np.arange(9), rtol=1e-12)
    p, _, _ = O.partial_cholesky(R.T @ R, omega=1e7, cond="svd")
    assert p == 8


def test_ice_bounds_svd():
    """ICE never overestimates (its Delta is a lower bound of sigma_max and
    its delta an upper bound of sigma_min) and stays within 10x of the SVD
    value "generally" (Sec. 3.2): here at the 95th percentile of random
    triangular factors, with a median near 1."""
    rng = np.random.default_rng(3)
    ratios = []
    for trial in range(30):
        n = 25
        R = np.triu(rng.standard_normal((n, n))) + np.diag(
            np.exp(rng.uniform(-4, 4, n)))
        est = O.ICE(R[0, 0])
        for j in range(1, n):
            k = est.update(R[:j, j], R[j, j])
            sv = np.linalg.svd(R[:j + 1, :j + 1], compute_uv=False)
            ktrue = sv[0] / sv[-1]
            assert k <= ktrue * (1 + 1e-10)
            ratios.append(ktrue / k)
    assert np.percentile(ratios, 95) < 10.0
    assert np.median(ratios) < 1.5


# --------------------------------------------------------------- MPK
def test_mpk_diagonal_closed_form_with_pair():
    """On a diagonal A, V_{j+1} is a polynomial in the eigenvalues; a
    conjugate pair (a +- ib) contributes ((lam - a)^2 + b^2)/(g1 g2)."""
    lam = np.linspace(0.5, 3.0, 40)
    op = O.as_operator(W.diagonal(lam))
    q = np.random.default_rng(4).uniform(-1, 1, 40)
    th = np.array([2.0, 1 + 0.5j, 1 - 0.5j, 0.7])
    gm = np.array([1.3, 0.9, 0.9, 1.7])
    V, B = O.mpk(op, q, 4, th, gm)
    assert np.allclose(V[:, 1], (lam - 2.0) * q / 1.3)
    assert np.allclose(V[:, 2], (lam - 2.0) * (lam - 1.0) * q / (1.3 * 0.9))
    assert np.allclose(V[:, 3], (lam - 2.0) * ((lam - 1.0) ** 2 + 0.25) * q
                       / (1.3 * 0.9 * 0.9))
    assert np.allclose(V[:, 4], (lam - 2.0) * ((lam - 1.0) ** 2 + 0.25)
                       * (lam - 0.7) * q / (1.3 * 0.9 * 0.9 * 1.7))
    assert np.allclose(op @ V[:, :4], V @ B, atol=1e-13)


def test_mpk_change_of_basis_general_matrix():
    A = W.stencil2d(10, 10)
    op = O.as_operator(A)
    q = np.ones(A.n) / 10.0
    H, st = O.arnoldi_mgs(op, q, 12)
    rz = O.leja_order(O.ritz_values(H, st))
    th, gm = O.basis_shifts(O.BASIS_SCALED_NEWTON, rz,
                            O.scaling_coefficients(rz))
    V, B = O.mpk(op, q, 12, th, gm)
    assert np.linalg.norm(op @ V[:, :12] - V @ B) < 1e-13 * np.linalg.norm(V)


# ----------------------------------------------------------- block QR
def test_block_qr_reproduces_block_and_is_orthonormal():
    rng = np.random.default_rng(6)
    Q, _ = np.linalg.qr(rng.standard_normal((300, 7)))
    X = rng.standard_normal((300, 9))
    bq = O.block_qr(Q, X)
    assert bq.p1 == 9 and bq.p2 == 9
    Qall = np.hstack([Q, bq.Qk])
    assert O.loss_of_orthogonality(Qall) < 1e-13
    recon = Q @ bq.R_top + bq.Qk @ bq.R_kk
    assert np.allclose(recon, X, atol=1e-12)
    assert np.allclose(np.tril(bq.R_kk, -1), 0.0)
    assert np.all(np.diag(bq.R_kk) > 0)


def test_block_qr_truncates_rank_deficient_block():
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((300, 3)))
    X = rng.standard_normal((300, 6))
    X[:, 4] = X[:, 1] + 1e-12 * rng.standard_normal(300)
    bq = O.block_qr(Q, X)
    assert bq.p2 == 4
    assert O.loss_of_orthogonality(np.hstack([Q, bq.Qk])) < 1e-13


# ------------------------------------------------------------- solver
def test_s1_is_mgs_gmres_on_stencil():
    """s = 1: partial CholQR is a norm and the block QR is CGS2, so the
    residual history equals MGS-GMRES to rounding (Sec. 3.3)."""
    c = W.config_c1(32)
    g = O.mgs_gmres(c["A"], c["b"], m=40, tol=1e-10)
    r = O.adaptive_sgmres(c["A"], c["b"], m=40, s=1, tol=1e-10)
    assert r.iters == g.iters and r.restarts == g.restarts
    a, b = np.array(r.relres_hist), np.array(g.relres_hist)
    assert np.max(np.abs(a - b)) <= 1e-12
    assert np.max(np.abs(a[:40] - b[:40]) / b[:40]) <= 1e-10


def test_s1_is_mgs_gmres_on_diagonal():
    lam = np.linspace(0.1, 10, 2000)
    b = np.random.default_rng(0).uniform(-1, 1, 2000)
    g = O.mgs_gmres(W.diagonal(lam), b, m=50, tol=1e-10)
    r = O.adaptive_sgmres(W.diagonal(lam), b, m=50, s=1, tol=1e-10)
    a, bb = np.array(r.relres_hist), np.array(g.relres_hist)
    assert a.size == bb.size and np.max(np.abs(a - bb)) <= 1e-12


def test_c1_converges_with_invariants():
    c = W.config_c1()
    r = O.adaptive_sgmres(c["A"], c["b"], m=c["m"], s=c["s"], tol=c["tol"],
                          diagnostics=True)
    assert r.converged and r.final_relres <= 1e-10
    assert max(r.loo) <= 1e-12            # LOO O(eps) at stable s
    assert max(r.arnoldi_res) <= 1e-12    # A Q_j = Q_{j+1} H_j
    # residual norms never increase inside a cycle (GMRES optimality)
    h = np.array(r.relres_hist)
    k = 0
    for n_c in r.cycle_iters:
        seg = h[k:k + n_c]
        assert np.all(np.diff(seg) <= 1e-13 * seg[:-1])
        k += n_c
    assert k == h.size
    # the implicit estimate at the end of the last cycle equals the true one
    op = O.as_operator(c["A"])
    assert np.linalg.norm(c["b"] - op @ r.x) / np.linalg.norm(c["b"]) \
        == pytest.approx(r.final_relres, rel=1e-10)
    assert h[-1] == pytest.approx(r.final_relres, rel=1e-3)


def test_residuals_monotone_within_cycle():
    c = W.config_c1(24)
    r = O.adaptive_sgmres(c["A"], c["b"], m=200, s=8, tol=1e-10)
    assert r.restarts == 0
    h = np.array(r.relres_hist)
    assert np.all(np.diff(h) <= 1e-13 * h[:-1])


def test_tiny_system_matches_dense_lu_and_terminates():
    """m >= N: GMRES reaches the exact solution within N columns."""
    rng = np.random.default_rng(8)
    n = 30
    Ad = rng.standard_normal((n, n)) + 8 * np.eye(n)
    import scipy.sparse as sp
    A = sp.csr_matrix(Ad)
    b = rng.standard_normal(n)
    xs = O.dense_solve(A, b)
    r = O.adaptive_sgmres(A, b, m=n, s=5, tol=1e-13)
    assert r.converged and r.iters <= n
    kappa = np.linalg.cond(Ad)
    assert np.linalg.norm(r.x - xs) <= kappa * 1e-14 * np.linalg.norm(xs)


def test_complex_spectrum_system():
    """2x2 rotation blocks: eigenvalues a +- ib, so the Ritz values come in
    conjugate pairs and the pair recurrence is exercised."""
    rng = np.random.default_rng(9)
    nb = 200
    a = rng.uniform(1.0, 4.0, nb)
    bb = rng.uniform(0.2, 1.5, nb)
    import scipy.sparse as sp
    blocks = [np.array([[a[k], bb[k]], [-bb[k], a[k]]]) for k in range(nb)]
    A = sp.csr_matrix(sp.block_diag(blocks, format="csr"))
    b = rng.uniform(-1, 1, 2 * nb)
    r = O.adaptive_sgmres(A, b, m=80, s=12, tol=1e-10, diagnostics=True)
    assert np.any(np.abs(r.ritz.imag) > 1e-3)
    assert r.converged and max(r.loo) < 1e-12 and max(r.arnoldi_res) < 1e-12
    assert np.linalg.norm(r.x - O.dense_solve(A, b)) < 1e-8 * np.linalg.norm(r.x)


def test_zero_rhs():
    c = W.config_c1(8)
    r = O.adaptive_sgmres(c["A"], np.zeros(64), m=10, s=3)
    assert r.converged and np.all(r.x == 0) and r.iters == 0


def test_paper_test1_monomial_adapts_to_6():
    """Paper Test 1: monomial basis with s0 = 10 adapts to s = 6."""
    gd = GOLD["test1_diag_monomial"]
    lam = np.linspace(gd["lam_lo"], gd["lam_hi"], gd["n"])
    b = np.ones(gd["n"]) / math.sqrt(gd["n"])
    r = O.adaptive_sgmres(W.diagonal(lam), b, m=100, s=gd["s0"], tol=1e-10,
                          basis=O.BASIS_MONOMIAL, diagnostics=True)
    full = [q for q, se in zip(r.s_hist, r.s_eff_hist)]
    assert full[0] == gd["adapted_s"]
    assert all(q == gd["adapted_s"] for q, se in zip(r.s_hist, r.s_eff_hist)
               if se >= gd["adapted_s"])
    assert max(r.loo) < 1e-12


def test_paper_test3_scaled_newton_keeps_100():
    """Paper Test 3: scaled Newton with s0 = 100 keeps s = 100."""
    gd = GOLD["test3_diag_scaled_newton"]
    lam = np.linspace(gd["lam_lo"], gd["lam_hi"], gd["n"])
    b = np.ones(gd["n"]) / math.sqrt(gd["n"])
    r = O.adaptive_sgmres(W.diagonal(lam), b, m=100, s=gd["s0"], tol=1e-10)
    assert r.s_hist[0] == gd["adapted_s"] and r.p1_hist[0] == gd["adapted_s"]


def test_estimator_drives_first_block():
    c = W.config_c2(12)
    r = O.adaptive_sgmres(c["A"], c["b"], m=60, s=0, tol=1e-10, s_min=4,
                          s_max=30, diagnostics=True)
    assert 4 <= r.s0 <= 30 and r.converged
    assert max(r.loo) < 1e-12


# ------------------------------------------------------ equilibration
def test_column_scaling_gives_unit_columns():
    """Eq. (equil) with D_r = I: every non-empty column of A D_c has unit
    2-norm; an empty column keeps the factor 1."""
    A, _ = W.random_band(3001, k=6, band=200)
    op = O.as_operator(A).tolil()
    op[:, 7] = 0.0                      # an empty column
    op = op.tocsr()
    op.eliminate_zeros()
    d = O.column_scaling(op)
    norms = np.linalg.norm((op @ sp.diags(d)).toarray(), axis=0)
    assert d[7] == 1.0 and norms[7] == 0.0
    keep = np.arange(op.shape[1]) != 7
    assert np.all(np.abs(norms[keep] - 1.0) <= 4e-16 * 8)


def test_scalar_scaling_normalises_the_ritz_values():
    """Scalar equilibration divides A by alpha = max |theta|: the same
    pre-pass on A / alpha gives Ritz values of largest modulus 1."""
    c = W.config_c1(24)
    alpha = O.scalar_scaling(c["A"], c["b"], k=12)
    op = O.as_operator(c["A"]) / alpha
    r = c["b"] / np.linalg.norm(c["b"])
    H, steps = O.arnoldi_mgs(op, r, 12)
    assert abs(np.max(np.abs(O.ritz_values(H, steps))) - 1.0) <= 1e-12


def test_equilibration_follows_the_papers_observations():
    """Sec. 4.3 on the explicitly scaled matrix A / alpha: the scaled
    Newton basis is insensitive to scalar scaling (its gamma is relative),
    the monomial basis gains a larger adapted step from the normalised
    spectrum, and the constant-gamma form the paper states as equivalent
    makes the same step-size decisions.  Every equilibrated solve reaches
    tol on the original system."""
    A, rng = W.aniso2d(32)
    b = rng.uniform(-1, 1, A.n)
    op = O.as_operator(A)
    kw = dict(m=60, s=20, tol=1e-10)
    alpha = O.scalar_scaling(A, b, k=20)
    assert alpha > 100
    r0 = O.adaptive_sgmres(A, b, basis="scaled_newton", **kw)
    r1 = O.adaptive_sgmres(op / alpha, b / alpha, basis="scaled_newton", **kw)
    assert r0.s_hist == r1.s_hist and r0.iters == r1.iters
    m0 = O.adaptive_sgmres(A, b, basis="monomial", **kw)
    m1 = O.adaptive_sgmres(op / alpha, b / alpha, basis="monomial", **kw)
    assert max(m1.s_hist) > max(m0.s_hist)
    m2, alpha2 = O.equilibrated_sgmres(A, b, "scalar", basis="monomial", **kw)
    assert abs(alpha2 - alpha) <= 1e-12 * alpha
    assert m2.s_hist[:len(m1.s_hist) // 2] == m1.s_hist[:len(m1.s_hist) // 2]
    c1, d = O.equilibrated_sgmres(A, b, "column", basis="scaled_newton", **kw)
    for r in (r1, m1, m2, c1):
        assert r.converged
        assert np.linalg.norm(b - op @ r.x) <= 1.01e-10 * np.linalg.norm(b)


# ------------------------------------------------------ adjoint gradient
def test_loss_gradients_match_central_differences():
    """dL/dvalues and dL/db of L = 0.5||A^-1 b - x_t||^2 against central
    differences along 16 seeded random directions (h = 1e-6)."""
    A, rng = W.aniso2d(8)
    b = rng.uniform(-1, 1, A.n)
    xt = rng.uniform(-1, 1, A.n)
    L0, dv, db, _ = O.loss_gradients(A, b, xt)
    h = 1e-6
    for k in range(16):
        d = np.random.default_rng(100 + k).standard_normal(A.nnz)
        e = np.random.default_rng(200 + k).standard_normal(A.n)
        Ap = W.CSR(A.n, A.rowptr, A.colind, A.val + h * d)
        Am = W.CSR(A.n, A.rowptr, A.colind, A.val - h * d)
        fd = (O.loss_gradients(Ap, b + h * e, xt)[0]
              - O.loss_gradients(Am, b - h * e, xt)[0]) / (2 * h)
        an = dv @ d + db @ e
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3)


def test_sparse_loss_matches_dense_and_central_differences():
    """The sparse-LU form of the loss and gradient agrees with the dense
    one (itself pinned by central differences above), and its perturbed
    losses give central differences that match its own gradient."""
    A, rng = W.aniso2d(20)
    b = rng.uniform(-1, 1, A.n)
    xt = rng.uniform(-1, 1, A.n)
    L0, dv, db, x0 = O.loss_gradients(A, b, xt)
    S = O.SparseLoss(A, b, xt)
    L1, dv1, db1, x1 = S.gradients()
    assert abs(L1 - L0) <= 1e-12 * abs(L0)
    assert np.linalg.norm(dv1 - dv) <= 1e-10 * np.linalg.norm(dv)
    assert np.linalg.norm(db1 - db) <= 1e-10 * np.linalg.norm(db)
    h = 1e-6
    for k in range(4):
        d = np.random.default_rng(100 + k).standard_normal(A.nnz)
        e = np.random.default_rng(200 + k).standard_normal(A.n)
        fd = (S.loss(h * d, h * e) - S.loss(-h * d, -h * e)) / (2 * h)
        fd_dense = (O.loss_gradients(W.CSR(A.n, A.rowptr, A.colind, A.val + h * d), b + h * e, xt)[0]
                    - O.loss_gradients(W.CSR(A.n, A.rowptr, A.colind, A.val - h * d), b - h * e, xt)[0]) / (2 * h)
        an = dv1 @ d + db1 @ e
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3)
        assert abs(fd - fd_dense) <= 1e-6 * max(abs(an), 1e-3)


# ----------------------------------------------- planted-mistake checks
def _pair_pin_fails():
    try:
        test_mpk_diagonal_closed_form_with_pair()
    except AssertionError:
        return True
    return False


def test_planted_pair_sign_is_caught(monkeypatch):
    orig = O.mpk

    def bad(A, q, s, theta, gamma):
        # plant: drop the b^2 term of the second step of a pair
        V, B = orig(A, q, s, theta, gamma)
        for j in range(s):
            if theta[j].imag < 0:
                V[:, j + 1] = (A @ V[:, j] - theta[j].real * V[:, j]) \
                    / gamma[j]
        return V, B
    monkeypatch.setattr(O, "mpk", bad)
    assert _pair_pin_fails()


def test_planted_hessenberg_term_is_caught(monkeypatch):
    orig = O.assemble_hessenberg

    def bad(H, i, R_top, R_kk, B):
        # plant: forget the previous-columns correction
        q = R_kk.shape[0]
        Rbar = np.zeros((i + q, q + 1))
        Rbar[i - 1, 0] = 1.0
        Rbar[:i, 1:] = R_top
        Rbar[i:, 1:] = R_kk
        M = Rbar @ B[:q + 1, :q]
        T = Rbar[i - 1:i + q - 1, :q]
        import scipy.linalg as sla
        H[:i + q, i - 1:i - 1 + q] = sla.solve_triangular(
            T, M.T, trans="T", lower=False).T
    monkeypatch.setattr(O, "assemble_hessenberg", bad)
    c = W.config_c1(16)
    r = O.adaptive_sgmres(c["A"], c["b"], m=40, s=6, tol=1e-10,
                          diagnostics=True, max_iters=200)
    assert (not r.converged) or max(r.arnoldi_res) > 1e-10


def test_planted_ice_sign_is_caught(monkeypatch):
    orig = O.ICE.update

    def bad(self, v, gam):
        return orig(self, -v, gam) if len(v) > 1 else orig(self, v, gam)
    monkeypatch.setattr(O.ICE, "update", bad)
    failed = False
    try:
        test_ice_bounds_svd()
    except AssertionError:
        failed = True
    assert failed


def test_planted_transposed_gram_is_caught(monkeypatch):
    orig = O.block_qr

    def bad(Q, X, omega=O.OMEGA, cond="ice"):
        out = orig(Q, X, omega, cond)
        out.R_top = out.R_top[:, ::-1].copy()   # plant: columns swapped
        return out
    monkeypatch.setattr(O, "block_qr", bad)
    c = W.config_c1(16)
    r = O.adaptive_sgmres(c["A"], c["b"], m=40, s=6, tol=1e-10,
                          diagnostics=True, max_iters=200)
    assert (not r.converged) or max(r.arnoldi_res) > 1e-10


def _estimator_pin_fails():
    for case in ESTIMATOR_EXACT:
        try:
            test_estimator_first_crossing_and_clamp_exact(*case)
        except AssertionError:
            return True
    return False


@pytest.mark.parametrize("plant", ["count_crossing", "last_below",
                                   "no_lower_clamp"])
def test_planted_estimator_index_is_caught(monkeypatch, plant):
    """Plants in the estimator's index (on the CPU): counting the crossing
    column itself, taking the last column below Omega_est, and dropping the
    clamp to s_min.  The exact pin catches each."""
    def bad(theta, omega_est=O.OMEGA_EST, eps=O.EPS64, s_min=1, s_max=None):
        norms = O.estimator_column_norms(theta, eps)
        below = [j for j in range(norms.size) if norms[j] < omega_est]
        if plant == "count_crossing":
            s0 = next((j + 1 for j in range(norms.size)
                       if not norms[j] < omega_est), norms.size)
        elif plant == "last_below":
            s0 = below[-1] + 1 if below else 0
        else:
            s0 = next((j for j in range(norms.size)
                       if not norms[j] < omega_est), norms.size)
            return (min(s0, s_max) if s_max is not None else s0), norms
        if s_max is not None:
            s0 = min(s0, s_max)
        return max(s0, s_min), norms
    monkeypatch.setattr(O, "estimate_step_size", bad)
    assert _estimator_pin_fails()


# ----------------------------------------------- Ritz residuals, supplied Ritz values
def test_ritz_residual_bounds_the_eigenvalue_distance():
    """For a symmetric matrix every Ritz value lies within its Ritz-pair
    residual of an eigenvalue (|theta - lambda| <= ||A z - theta z|| for a
    unit z, Sec. 3.4's Ritz pairs); converged ones have tiny residuals."""
    lam = np.linspace(1.0, 50.0, 400)
    lam[-1] = 100.0                      # an isolated eigenvalue converges first
    op = O.as_operator(W.diagonal(lam))
    q = np.random.default_rng(4).uniform(-1, 1, lam.size)
    H, steps = O.arnoldi_mgs(op, q / np.linalg.norm(q), 30)
    theta, res = O.ritz_residuals(H, steps)
    assert np.all(np.abs(theta.imag) < 1e-12)
    for t, r in zip(theta.real, res):
        assert np.min(np.abs(lam - t)) <= r * (1 + 1e-9) + 1e-12
    # the isolated extreme eigenvalue has converged
    i = np.argmax(theta.real)
    assert res[i] < 1e-6 and abs(theta.real[i] - 100.0) < 1e-6
    # a full Arnoldi on a 12 x 12 stencil: every residual is ~0
    A = O.as_operator(W.stencil2d(4, 3))
    H, steps = O.arnoldi_mgs(A, np.ones(12) / math.sqrt(12), 12)
    _, res = O.ritz_residuals(H, steps)
    assert np.all(res < 1e-6)


def test_supplied_ritz_values_reproduce_the_run():
    """Feeding a run's own (Leja-ordered) Ritz values back in skips the
    pre-pass and repeats every decision and the solution bit for bit."""
    c = W.config_c2(10)
    kw = dict(m=40, s=0, s_min=2, s_max=16, tol=1e-10)
    r1 = O.adaptive_sgmres(c["A"], c["b"], **kw)
    r2 = O.adaptive_sgmres(c["A"], c["b"], ritz=r1.ritz[::-1], **kw)
    assert r2.prepass_H is None and r1.prepass_H is not None
    assert np.array_equal(r2.ritz, r1.ritz)
    assert r2.s0 == r1.s0 and r2.s_hist == r1.s_hist and r2.p1_hist == r1.p1_hist
    assert np.array_equal(r2.x, r1.x)
