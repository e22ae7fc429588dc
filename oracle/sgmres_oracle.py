"""CPU oracle for the adaptive s-step GMRES of Xu, Alonso and Darve,
"A numerically stable communication-avoiding s-step GMRES algorithm"
(arXiv 2303.08953).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain FP64 statement of
what the GPU library computes.  Only the tests, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline leg may import it; the library never does.
It shares no code with the CUDA path.

Every function follows one passage of the paper and names it.  Library
primitives serve as single steps (scipy's CSR product, numpy's matrix
product, LAPACK's eigenvalues / triangular solves / SVD); there is no
blocking or fusion beyond what the paper's algorithms state.

Readings of passages the paper leaves open (each is listed with its reason
in the design notes of the repository):
  * Leja order: start at the Ritz value of largest modulus, then maximise
    the product of distances to the chosen ones; a complex value (imaginary
    part > 0 representative) is followed at once by its conjugate.  Scores
    within a relative 1e-9 count as ties, broken by larger real part, then
    larger imaginary part, then lower index.
  * Complex Ritz pairs (a +- ib) in real arithmetic: two-step recurrence
    V+1 = (A - a)V/g, V+2 = ((A - a)V+1 + (b^2/g) V)/g'.
  * Ritz values: k steps of MGS-Arnoldi from the first normalised residual,
    once per solve (k = s0 when s0 is fixed, s_max when s is estimated);
    the pre-pass vectors are not counted as iterations.  Arnoldi stops early
    when the new subdiagonal falls below 1e-12 of the pre-projection norm.
  * Degenerate scaling coefficient (gamma <= 1e-14 max|theta|, e.g. s = 1):
    replaced by the mean of the non-degenerate ones, or 1 if there are none.
  * Alg. 3's inner sum runs over k < i (standard Cholesky); the stop test is
    a non-positive / non-finite pivot or kappa_j > Omega (strict).
  * Estimator: E exactly as Eq. (auxiliarymatrix) with O(eps) = eps,
    unnormalised column 2-norms; s0* = number of leading columns whose norm
    stays below Omega_est (first crossing), clamped to [s_min, s_max].
  * Hessenberg assembly (Alg. 4 "assemble"): from A V = V B and
    V = Q Rbar, H[:, new] = (Rbar B - [H_old Rbar_top; 0]) T^-1.
  * s carries over restarts and is never increased; a block shortened to fit
    the restart length m does not lower the carried s.
  * Convergence inside a block: the first column whose implicit relative
    residual |g_{j+1}|/beta0 <= tol ends the cycle; the true residual
    decides, otherwise a new cycle starts from the updated x.
  * Happy breakdown (first Cholesky pivot <= 0): the block contributes one
    column with a zero subdiagonal, which makes the least-squares solution
    exact.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

EPS64 = 2.0 ** -53          # unit round-off of FP64 (Sec. 4: eps ~ 2^-53)
OMEGA = 1.0e7               # Omega for partial CholQR (Sec. 4 intro)
OMEGA_EST = 1.0e7           # Omega_est of the estimator (Sec. 4.4.2)

BASIS_SCALED_NEWTON = "scaled_newton"   # Eq. (scalednewton)
BASIS_NEWTON = "newton"                 # Eq. (newton)
BASIS_MONOMIAL = "monomial"             # Eq. (monomial)


# --------------------------------------------------------------- operators
def as_operator(A):
    """CSR (workloads.CSR or scipy) -> scipy CSR matrix (library SpMV)."""
    if sp.issparse(A):
        return A.tocsr()
    if hasattr(A, "to_scipy"):
        return A.to_scipy()
    return sp.csr_matrix(np.asarray(A, dtype=np.float64))


def spmv(A, x):
    """y = A x (CSR product; Sec. 2, the MPK's building block)."""
    return A @ x


# ---------------------------------------------------- Ritz values / shifts
def arnoldi_mgs(A, q1, k):
    """k steps of Arnoldi with modified Gram-Schmidt from unit vector q1
    (the 'classical Arnoldi' pre-pass that supplies Ritz values, Sec. 3.4).

    Returns (H, steps): H is (k+1) x k, ``steps`` the number of completed
    steps (fewer than k after an invariant-subspace breakdown).
    """
    n = q1.size
    Q = np.zeros((n, k + 1))
    H = np.zeros((k + 1, k))
    Q[:, 0] = q1
    for j in range(k):
        w = spmv(A, Q[:, j])
        wnorm0 = np.linalg.norm(w)
        for l in range(j + 1):
            H[l, j] = Q[:, l] @ w
            w = w - H[l, j] * Q[:, l]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= 1e-12 * wnorm0 or not np.isfinite(H[j + 1, j]):
            return H, j + 1
        Q[:, j + 1] = w / H[j + 1, j]
    return H, k


def ritz_values(H, steps):
    """Eigenvalues of the leading steps x steps block of H (Sec. 3.4)."""
    return np.linalg.eigvals(H[:steps, :steps]).astype(np.complex128)


def ritz_residuals(H, steps):
    """Ritz values theta of the leading steps x steps block of H and, for
    each, the residual norm of its Ritz pair, ||A V y - theta V y|| =
    h_{k+1,k} |e_k^T y| for the unit eigenvector y of H_k (the Arnoldi
    relation A V_k = V_{k+1} H_{k+1,k}, Sec. 3.4).  A small residual marks a
    converged Ritz value, one that another run of the pre-pass reproduces
    whatever its rounding."""
    Hk = H[:steps, :steps]
    theta, Y = np.linalg.eig(Hk)
    Y = Y / np.linalg.norm(Y, axis=0)
    hnext = abs(H[steps, steps - 1]) if H.shape[0] > steps else 0.0
    return theta.astype(np.complex128), hnext * np.abs(Y[steps - 1, :])


def _is_tie(a, b):
    return abs(a - b) <= 1e-9 * max(1.0, abs(a), abs(b))


def _better(cand, best, vals):
    """Tie rules of the Leja reading: larger real, then larger imaginary
    part, then lower index."""
    (sc, ic), (sb, ib) = cand, best
    if not _is_tie(sc, sb):
        return sc > sb
    zc, zb = vals[ic], vals[ib]
    if zc.real != zb.real:
        return zc.real > zb.real
    if zc.imag != zb.imag:
        return zc.imag > zb.imag
    return ic < ib


def leja_order(theta):
    """Leja ordering of the Ritz values with conjugate pairs kept adjacent
    (Sec. 3.4, 'Ritz values of A in a Leja ordering').  Returns a complex
    array; a pair appears as (a+ib, a-ib) with b > 0."""
    theta = np.asarray(theta, dtype=np.complex128)
    n = theta.size
    reps = [i for i in range(n) if theta[i].imag >= 0]
    used = np.zeros(n, dtype=bool)
    order = []

    def take(i):
        order.append(i)
        used[i] = True
        if theta[i].imag > 0:
            # its conjugate: the unused value with -imag closest to it
            cands = [j for j in range(n) if not used[j] and theta[j].imag < 0]
            j = min(cands, key=lambda j: abs(theta[j] - np.conj(theta[i])))
            order.append(j)
            used[j] = True

    best = None
    for i in reps:
        c = (abs(theta[i]), i)
        if best is None or _better(c, best, theta):
            best = c
    take(best[1])
    while len(order) < n:
        best = None
        for i in reps:
            if used[i]:
                continue
            d = np.abs(theta[i] - theta[order])
            sc = -math.inf if np.any(d == 0) else float(np.sum(np.log(d)))
            c = (sc, i)
            if best is None or _better(c, best, theta):
                best = c
        take(best[1])
    return theta[order]


def scaling_coefficients(theta):
    """gamma_i = |mean(theta) - theta_i| (Eq. scalingcoeff), with the
    degenerate-gamma reading for gamma ~ 0."""
    theta = np.asarray(theta, dtype=np.complex128)
    tbar = np.mean(theta).real
    gam = np.abs(tbar - theta)
    bad = gam <= 1e-14 * np.max(np.abs(theta)) if theta.size else gam
    if np.any(bad):
        good = gam[~bad]
        gam = gam.copy()
        gam[bad] = np.mean(good) if good.size else 1.0
    return gam


def estimator_log2_E(theta, eps=EPS64):
    """log2 of the auxiliary matrix E (Eq. auxiliarymatrix), s x s, for the
    Leja-ordered Ritz values theta (1-based i, j in the paper; 0-based
    here).  Row i, column j:
      j <  i : prod_{k<j} rho(i,k)
      j == i : eps * prod_{k<j} rho(i,k)
      j >  i : eps * prod_{k<j, k!=i} rho(i,k)
    with rho(i,k) = |theta_i - theta_k| / |tbar - theta_k|."""
    theta = np.asarray(theta, dtype=np.complex128)
    s = theta.size
    tbar = np.mean(theta).real
    lg = np.empty((s, s))
    with np.errstate(divide="ignore"):
        den = np.log2(np.abs(tbar - theta))
        for i in range(s):
            acc = 0.0
            for j in range(s):
                if j < i:
                    lg[i, j] = acc
                    acc += math.log2(abs(theta[i] - theta[j])) - den[j] \
                        if theta[i] != theta[j] else -math.inf
                elif j == i:
                    lg[i, j] = acc + math.log2(eps)
                else:
                    lg[i, j] = acc + math.log2(eps)
                    acc += math.log2(abs(theta[i] - theta[j])) - den[j] \
                        if theta[i] != theta[j] else -math.inf
    return lg


def estimator_column_norms(theta, eps=EPS64):
    """||E_j||_2 for every column j (Sec. 3.5), evaluated from log2 E with
    a per-column scale so that no entry overflows:
    ||E_j|| = 2^mx * sqrt(sum_i (E_ij / 2^mx)^2), mx = max_i log2 E_ij."""
    lg = estimator_log2_E(theta, eps)
    mx = np.max(lg, axis=0)
    with np.errstate(over="ignore", invalid="ignore"):
        sc = np.sqrt(np.sum(np.exp2(2.0 * (lg - mx[None, :])), axis=0))
        return np.exp2(mx) * sc


def estimate_step_size(theta, omega_est=OMEGA_EST, eps=EPS64, s_min=1,
                       s_max=None):
    """s0* = argmax_j { ||E_j|| < Omega_est } (Sec. 3.5), first crossing,
    clamped to [s_min, s_max]."""
    norms = estimator_column_norms(theta, eps)
    s0 = norms.size
    for j in range(norms.size):
        if not norms[j] < omega_est:
            s0 = j
            break
    if s_max is not None:
        s0 = min(s0, s_max)
    return max(s0, s_min), norms


# ------------------------------------------------------------------- MPK
def basis_shifts(basis, theta, gamma):
    """Per-step (shift, scale) parameters of the polynomial basis.
    monomial: theta = 0, gamma = 1 (Eq. monomial); Newton: gamma = 1
    (Eq. newton); scaled Newton: Eq. (scalednewton) with Eq. (scalingcoeff).
    """
    k = len(theta)
    if basis == BASIS_MONOMIAL:
        return np.zeros(k, dtype=np.complex128), np.ones(k)
    if basis == BASIS_NEWTON:
        return np.asarray(theta, dtype=np.complex128), np.ones(k)
    if basis == BASIS_SCALED_NEWTON:
        return np.asarray(theta, dtype=np.complex128), np.asarray(gamma)
    raise ValueError(basis)


def mpk(A, q, s, theta, gamma):
    """Matrix powers kernel in the (scaled) Newton basis (Sec. 2, Eq.
    newtonrecurrence): V_1 = q, V_{j+1} = (A V_j - theta_j V_j)/gamma_j,
    with the real two-step form for a conjugate pair.  Returns V
    (n x (s+1)) and the change-of-basis matrix B ((s+1) x s) with
    A V[:, :s] = V B."""
    n = q.size
    V = np.zeros((n, s + 1))
    B = np.zeros((s + 1, s))
    V[:, 0] = q
    for j in range(s):
        th, g = theta[j], gamma[j]
        a = th.real
        AV = spmv(A, V[:, j])
        if th.imag < 0 and j > 0 and theta[j - 1].imag > 0:
            # second step of a pair: ((A - a)V_j + (b^2/gamma_{j-1}) V_{j-1})
            b2g = th.imag ** 2 / gamma[j - 1]
            V[:, j + 1] = (AV - a * V[:, j] + b2g * V[:, j - 1]) / g
            B[j - 1, j] = -b2g
        else:
            V[:, j + 1] = (AV - a * V[:, j]) / g
        B[j, j] = a
        B[j + 1, j] = g
    return V, B


# --------------------------------------------------- partial Cholesky (Alg 3)
def _sym2_max_eig(a, b, d):
    """Largest eigenvalue of [[a, b], [b, d]] and a unit eigenvector."""
    half = 0.5 * (a - d)
    rad = math.hypot(half, b)
    lam = 0.5 * (a + d) + rad
    if b == 0.0:
        return lam, ((1.0, 0.0) if a >= d else (0.0, 1.0))
    # (b, lam - a) and (lam - d, b) are both eigenvectors; use the longer
    v1 = (b, lam - a)
    v2 = (lam - d, b)
    v = v1 if math.hypot(*v1) >= math.hypot(*v2) else v2
    nv = math.hypot(*v)
    return lam, (v[0] / nv, v[1] / nv)


class ICE:
    """Incremental condition estimator for an upper-triangular factor
    grown one column at a time (Sec. 3.2; Bischof 1990), derived here:

    largest singular value: keep unit x with ||x^T R|| = Delta; the new
    column (v, gam) gives ||[sig x; c]^T R_new||^2 = [sig c] M [sig c]^T,
    M = [[Delta^2 + alpha^2, alpha gam], [alpha gam, gam^2]], alpha = x^T v.
    smallest singular value: keep w = R^-T x with ||w|| = 1/delta; then
    ||[sig x; c]^T R_new^-1||^2 = [sig c] M' [sig c]^T,
    M' = [[1/delta^2 + alpha'^2/gam^2, -alpha'/gam^2], [., 1/gam^2]],
    alpha' = w^T v.  Both maximise over the unit circle (largest
    eigenvalue), kappa = Delta / delta.
    """

    def __init__(self, r11):
        self.x = np.array([1.0])
        self.Delta = abs(r11)
        self.w = np.array([1.0 / r11])
        self.delta = abs(r11)

    def update(self, v, gam):
        alpha = float(self.x @ v)
        nu, (s1, c1) = _sym2_max_eig(self.Delta ** 2 + alpha ** 2,
                                     alpha * gam, gam ** 2)
        self.x = np.concatenate([s1 * self.x, [c1]])
        self.Delta = math.sqrt(nu)
        alpha2 = float(self.w @ v)
        mu, (s2, c2) = _sym2_max_eig(1.0 / self.delta ** 2
                                     + alpha2 ** 2 / gam ** 2,
                                     -alpha2 / gam ** 2, 1.0 / gam ** 2)
        self.w = np.concatenate([s2 * self.w, [(c2 - s2 * alpha2) / gam]])
        self.delta = 1.0 / math.sqrt(mu)
        return self.kappa

    @property
    def kappa(self):
        return self.Delta / self.delta


def partial_cholesky(G, omega=OMEGA, cond="ice"):
    """Alg. 3: column-by-column Cholesky of the s x s Gram matrix G; stop
    before column j when its pivot is not positive (breakdown, Sec. 3.1) or
    when kappa_j > Omega (Sec. 3.2).  Returns (p, R_p, kappas)."""
    s = G.shape[0]
    R = np.zeros((s, s))
    kappas = []
    est = None
    for j in range(s):
        for i in range(j):
            R[i, j] = (G[i, j] - R[:i, i] @ R[:i, j]) / R[i, i]
        d = G[j, j] - R[:j, j] @ R[:j, j]
        if not (d > 0.0) or not np.isfinite(d):
            return j, R[:j, :j].copy(), kappas
        R[j, j] = math.sqrt(d)
        if cond == "svd":
            sv = np.linalg.svd(R[:j + 1, :j + 1], compute_uv=False)
            kap = sv[0] / sv[-1]
        elif j == 0:
            est = ICE(R[0, 0])
            kap = est.kappa
        else:
            kap = est.update(R[:j, j], R[j, j])
        kappas.append(kap)
        if kap > omega:
            return j, R[:j, :j].copy(), kappas
    return s, R, kappas


# ------------------------------------------------------ block QR (Alg 4)
@dataclass
class BlockQR:
    p1: int                 # columns kept by the first partial CholQR
    p2: int                 # columns kept by the second (the new s)
    Qk: np.ndarray          # n x p2 new orthonormal columns
    R_top: np.ndarray       # i x p2
    R_kk: np.ndarray        # p2 x p2
    breakdown: bool = False


def block_qr(Q, X, omega=OMEGA, cond="ice"):
    """BCGS2 with partial CholQR (Alg. 4, 'First BCGS' ... 'Combine both
    steps') of the block X against the orthonormal columns Q (n x i)."""
    W = Q.T @ X                                   # first BCGS
    X = X - Q @ W
    p1, Z, _ = partial_cholesky(X.T @ X, omega, cond)   # first partial CholQR
    if p1 == 0:
        return BlockQR(0, 0, np.zeros((Q.shape[0], 0)), W[:, :1],
                       np.zeros((1, 1)), breakdown=True)
    Qk = sla.solve_triangular(Z, X[:, :p1].T, trans="T", lower=False).T
    Rp = Q.T @ Qk                                  # second BCGS
    Qk = Qk - Q @ Rp
    p2, Zt, _ = partial_cholesky(Qk.T @ Qk, omega, cond)  # second CholQR
    if p2 == 0:
        return BlockQR(p1, 0, np.zeros((Q.shape[0], 0)),
                       W[:, :1] + Rp[:, :1] * Z[0, 0], np.zeros((1, 1)),
                       breakdown=True)
    Qk = sla.solve_triangular(Zt, Qk[:, :p2].T, trans="T", lower=False).T
    R_top = W[:, :p2] + Rp[:, :p2] @ Z[:p2, :p2]  # combine both steps
    R_kk = Zt @ Z[:p2, :p2]
    return BlockQR(p1, p2, Qk, R_top, R_kk)


def assemble_hessenberg(H, i, R_top, R_kk, B):
    """New Hessenberg columns i..i+q-1 (1-based) from V = Q Rbar and
    A V[:, :q] = V[:, :q+1] B (Alg. 4 'Assemble upper Hessenberg').
    H holds the unrotated Hessenberg matrix and is updated in place."""
    q = R_kk.shape[0]
    Rbar = np.zeros((i + q, q + 1))
    Rbar[i - 1, 0] = 1.0
    Rbar[:i, 1:] = R_top
    Rbar[i:, 1:] = R_kk
    M = Rbar @ B[:q + 1, :q]
    if i > 1:
        M[:i, :] -= H[:i, :i - 1] @ Rbar[:i - 1, :q]
    T = Rbar[i - 1:i + q - 1, :q]
    Hnew = sla.solve_triangular(T, M.T, trans="T", lower=False).T
    H[:i + q, i - 1:i - 1 + q] = Hnew
    return Hnew


# ---------------------------------------------------------------- Givens
def givens_column(Hr, cs, sn, g, j):
    """Apply the previous rotations to column j of Hr, then make the one
    that annihilates Hr[j+1, j] and update g (Alg. 1 'Apply Givens')."""
    for l in range(j):
        t = cs[l] * Hr[l, j] + sn[l] * Hr[l + 1, j]
        Hr[l + 1, j] = -sn[l] * Hr[l, j] + cs[l] * Hr[l + 1, j]
        Hr[l, j] = t
    a, b = Hr[j, j], Hr[j + 1, j]
    r = math.hypot(a, b)
    if r == 0.0:
        cs[j], sn[j] = 1.0, 0.0
    else:
        cs[j], sn[j] = a / r, b / r
    Hr[j, j] = r
    Hr[j + 1, j] = 0.0
    g[j + 1] = -sn[j] * g[j]
    g[j] = cs[j] * g[j]


# ---------------------------------------------------------------- solvers
@dataclass
class SolveResult:
    x: np.ndarray
    converged: bool
    iters: int = 0
    restarts: int = 0
    s0: int = 0
    s_hist: list = field(default_factory=list)       # p2 per block
    s_eff_hist: list = field(default_factory=list)   # columns generated
    p1_hist: list = field(default_factory=list)
    relres_hist: list = field(default_factory=list)  # implicit, per column
    cycle_relres: list = field(default_factory=list)  # true, per cycle
    cycle_iters: list = field(default_factory=list)   # columns per cycle
    final_relres: float = 0.0
    ritz: np.ndarray = None
    gamma: np.ndarray = None
    prepass_H: np.ndarray = None                     # (k+1) x k, Sec. 3.4
    prepass_steps: int = 0
    est_norms: np.ndarray = None
    loo: list = field(default_factory=list)          # per cycle
    arnoldi_res: list = field(default_factory=list)  # per cycle


def adaptive_sgmres(A, b, x0=None, m=60, s=10, tol=1e-10, *,
                    basis=BASIS_SCALED_NEWTON, omega=OMEGA,
                    omega_est=OMEGA_EST, eps=EPS64, s_min=1, s_max=None,
                    max_iters=None, cond="ice", diagnostics=False,
                    scalar_equil=False, ritz=None):
    """Adaptive s-step GMRES(m) (Alg. 4) with restarts.

    s > 0: fixed initial step size s0 (Ritz pre-pass of s0 steps);
    s == 0: s0* from the estimator (Sec. 3.5) over s_max Ritz values.
    ritz: Ritz values to use instead of running the pre-pass (conjugate
    pairs complete); they are Leja-ordered and used as the pre-pass's
    would be (Sec. 3.4).
    scalar_equil: scalar equilibration A' = A / alpha, alpha = max |theta|
    (Eq. equil), in the equivalent form Sec. 4.3 states: the monomial and
    standard Newton bases take the constant scaling coefficient alpha; the
    scaled Newton basis is unchanged.
    """
    A = as_operator(A)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    if s_max is None:
        s_max = s if s > 0 else m
    if max_iters is None:
        max_iters = 50 * m
    r = b - spmv(A, x)
    beta0 = float(np.linalg.norm(r))
    res = SolveResult(x=x, converged=True)
    if beta0 == 0.0:
        return res
    res.converged = False
    theta = gamma = None
    cur_s = 0
    total = 0
    cycle = 0
    while True:
        beta = float(np.linalg.norm(r))
        Q = np.zeros((n, m + 1))
        Q[:, 0] = r / beta
        H = np.zeros((m + 1, m))
        Hr = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        if theta is None:
            if ritz is None:
                k = s if s > 0 else s_max
                k = min(k, m)
                Hk, steps = arnoldi_mgs(A, Q[:, 0], k)
                res.prepass_H, res.prepass_steps = Hk, steps
                ritz = leja_order(ritz_values(Hk, steps))
            else:
                ritz = leja_order(np.asarray(ritz, dtype=np.complex128))
                steps = ritz.size
            gam_sn = scaling_coefficients(ritz)
            theta, gamma = basis_shifts(basis, ritz, gam_sn)
            if scalar_equil and basis != BASIS_SCALED_NEWTON:
                gamma = np.full(len(gamma), float(np.max(np.abs(ritz))))
            res.ritz, res.gamma = ritz, gamma
            if s > 0:
                cur_s = min(s, steps)
            else:
                cur_s, res.est_norms = estimate_step_size(
                    ritz, omega_est, eps, s_min, min(s_max, steps))
                cur_s = min(cur_s, steps)
            res.s0 = cur_s
        i = 1
        jdone = 0
        stop_cycle = False
        while i <= m and not stop_cycle:
            s_eff = min(cur_s, m + 1 - i)
            V, B = mpk(A, Q[:, i - 1], s_eff, theta, gamma)
            bq = block_qr(Q[:, :i], V[:, 1:], omega, cond)
            res.s_eff_hist.append(s_eff)
            res.p1_hist.append(bq.p1)
            if bq.breakdown:
                q = 1
                assemble_hessenberg(H, i, bq.R_top, bq.R_kk, B)
                res.s_hist.append(0)
            else:
                q = bq.p2
                Q[:, i:i + q] = bq.Qk
                assemble_hessenberg(H, i, bq.R_top, bq.R_kk, B)
                res.s_hist.append(q)
                if q < s_eff:
                    cur_s = q                      # Alg. 4: s = p
            for c in range(q):
                j = i - 1 + c
                Hr[:j + 2, j] = H[:j + 2, j]
                givens_column(Hr, cs, sn, g, j)
                rel = abs(g[j + 1]) / beta0
                res.relres_hist.append(rel)
                jdone = j + 1
                if rel <= tol or bq.breakdown:
                    stop_cycle = True
                    break
            total_cols = total + jdone
            i += q
            if total_cols >= max_iters:
                stop_cycle = True
        # end of cycle: least squares + update (Alg. 4 last two lines)
        y = sla.solve_triangular(Hr[:jdone, :jdone], g[:jdone], lower=False)
        x = x + Q[:, :jdone] @ y
        if diagnostics:
            Qj = Q[:, :jdone + 1]
            res.loo.append(float(np.linalg.norm(
                np.eye(Qj.shape[1]) - Qj.T @ Qj)))
            AQ = np.column_stack([spmv(A, Q[:, c]) for c in range(jdone)])
            Hj = H[:jdone + 1, :jdone]
            res.arnoldi_res.append(float(
                np.linalg.norm(AQ - Qj @ Hj)
                / (sp.linalg.norm(A) * np.linalg.norm(Hj))))
        total += jdone
        r = b - spmv(A, x)
        rel_true = float(np.linalg.norm(r)) / beta0
        res.cycle_relres.append(rel_true)
        res.cycle_iters.append(jdone)
        cycle += 1
        if rel_true <= tol:
            res.converged = True
            break
        if total >= max_iters:
            break
    res.x = x
    res.iters = total
    res.restarts = cycle - 1
    res.final_relres = res.cycle_relres[-1]
    return res


# ------------------------------------------------------------ equilibration
def column_scaling(A):
    """Column equilibration of Eq. (equil), Sec. 4.3: D_r = I and
    D_c = diag(1 / ||A(:, j)||_2) (a column with no entries keeps 1).
    Returns the diagonal of D_c."""
    op = as_operator(A)
    norms = np.sqrt(np.asarray(op.multiply(op).sum(axis=0)).ravel())
    d = np.ones(op.shape[1])
    nz = norms > 0
    d[nz] = 1.0 / norms[nz]
    return d


def scalar_scaling(A, b, x0=None, k=10):
    """Scalar equilibration of Eq. (equil), Sec. 4.3: A' = A / alpha with
    alpha = max |theta| over the Ritz values of the same k-step pre-pass
    the solver runs (from the normalised initial residual)."""
    op = as_operator(A)
    x = np.zeros(b.size) if x0 is None else np.asarray(x0, dtype=np.float64)
    r = b - spmv(op, x)
    Hk, steps = arnoldi_mgs(op, r / np.linalg.norm(r), k)
    return float(np.max(np.abs(ritz_values(Hk, steps))))


def equilibrated_sgmres(A, b, mode, x0=None, **kw):
    """Alg. 4 on the equilibrated system of Eq. (equil):
    'scalar': A' = A / alpha in the equivalent form of Sec. 4.3 (constant
    scaling coefficient alpha for the monomial and Newton bases);
    'column': A' = A D_c, A' y = b, x = D_c y.
    Both keep ||b - A x|| / ||b - A x0|| equal to the scaled system's
    relative residual.  Returns (SolveResult with x in the original
    unknowns, the scaling: alpha or the diagonal of D_c)."""
    op = as_operator(A)
    if mode == "scalar":
        res = adaptive_sgmres(op, b, x0, scalar_equil=True, **kw)
        return res, float(np.max(np.abs(res.ritz)))
    if mode == "column":
        d = column_scaling(op)
        y0 = None if x0 is None else np.asarray(x0, dtype=np.float64) / d
        res = adaptive_sgmres(op @ sp.diags(d), b, y0, **kw)
        res.x = d * res.x
        return res, d
    raise ValueError(mode)


def mgs_gmres(A, b, x0=None, m=60, tol=1e-10, max_iters=None):
    """Standard GMRES(m) with MGS Arnoldi and Givens rotations (the paper's
    baseline, Sec. 4 and Sec. 5).  Same result record as adaptive_sgmres."""
    A = as_operator(A)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    if max_iters is None:
        max_iters = 50 * m
    r = b - spmv(A, x)
    beta0 = float(np.linalg.norm(r))
    res = SolveResult(x=x, converged=True)
    if beta0 == 0.0:
        return res
    res.converged = False
    total = 0
    cycle = 0
    while True:
        beta = float(np.linalg.norm(r))
        Q = np.zeros((n, m + 1))
        Q[:, 0] = r / beta
        Hr = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        jdone = 0
        for j in range(m):
            w = spmv(A, Q[:, j])
            for l in range(j + 1):
                Hr[l, j] = Q[:, l] @ w
                w = w - Hr[l, j] * Q[:, l]
            hnext = np.linalg.norm(w)
            Hr[j + 1, j] = hnext
            if hnext > 0:
                Q[:, j + 1] = w / hnext
            givens_column(Hr, cs, sn, g, j)
            rel = abs(g[j + 1]) / beta0
            res.relres_hist.append(rel)
            jdone = j + 1
            if rel <= tol or hnext == 0 or total + jdone >= max_iters:
                break
        y = sla.solve_triangular(Hr[:jdone, :jdone], g[:jdone], lower=False)
        x = x + Q[:, :jdone] @ y
        total += jdone
        r = b - spmv(A, x)
        rel_true = float(np.linalg.norm(r)) / beta0
        res.cycle_relres.append(rel_true)
        res.cycle_iters.append(jdone)
        cycle += 1
        if rel_true <= tol:
            res.converged = True
            break
        if total >= max_iters:
            break
    res.x = x
    res.iters = total
    res.restarts = cycle - 1
    res.final_relres = res.cycle_relres[-1]
    return res


def dense_solve(A, b):
    """x = A^-1 b by dense LU with partial pivoting (LAPACK), for tiny
    systems."""
    Ad = as_operator(A).toarray()
    return sla.lu_solve(sla.lu_factor(Ad), b)


class SparseLoss:
    """The same loss and adjoint gradient as `loss_gradients` for systems
    too large for dense LU: one sparse LU of A (SuperLU, a library step)
    gives x = A^-1 b and lam = A^-T (x - x_t).  `loss(dval, db)` evaluates
    L at perturbed values A + dA (same pattern) and b + db by iterative
    refinement on A's factors, for central differences at full size."""

    def __init__(self, A, b, x_target):
        import scipy.sparse.linalg as spl
        self.op = as_operator(A)
        self.b = np.asarray(b, dtype=np.float64)
        self.xt = np.asarray(x_target, dtype=np.float64)
        self.lu = spl.splu(self.op.tocsc())
        self.x = self._refine(self.op, self.b)
        r = self.x - self.xt
        self.lam = self._refine(self.op.T.tocsr(), r, trans=True)
        rows = np.repeat(np.arange(self.op.shape[0]), np.diff(self.op.indptr))
        self.dvals = -self.lam[rows] * self.x[self.op.indices]
        self.L = 0.5 * float(r @ r)

    def _refine(self, M, rhs, trans=False, iters=30):
        """Solve M y = rhs (M = A + small dA, or A^T) by iterative
        refinement with A's LU factors, until the correction stops
        shrinking."""
        solve = (lambda v: self.lu.solve(v, trans="T")) if trans else self.lu.solve
        y = solve(rhs)
        prev = np.inf
        for _ in range(iters):
            dy = solve(rhs - M @ y)
            y = y + dy
            nd = np.linalg.norm(dy)
            if nd <= 1e-17 * np.linalg.norm(y) or nd >= 0.5 * prev:
                break
            prev = nd
        return y

    def gradients(self):
        """(L, dL/dvalues, dL/db = lam, x)."""
        return self.L, self.dvals, self.lam, self.x

    def loss(self, dval, db):
        """L at values A.val + dval and right-hand side b + db."""
        op = self.op.copy()
        op.data = op.data + dval
        x = self._refine(op, self.b + db)
        r = x - self.xt
        return 0.5 * float(r @ r)


def loss_of_orthogonality(Q):
    """||I - Q^T Q||_F (Sec. 2.2, Eq. LOO)."""
    return float(np.linalg.norm(np.eye(Q.shape[1]) - Q.T @ Q))


def loss_gradients(A, b, x_target):
    """Dense reference for the adjoint gradient of L = 0.5 ||x - x_t||^2
    with x = A^-1 b (the differentiation workload): lam = A^-T (x - x_t),
    dL/db = lam, dL/dA_ij = -lam_i x_j on A's stored pattern.  Returns
    (L, dL/dvalues, dL/db, x)."""
    op = as_operator(A)
    Ad = op.toarray()
    lu = sla.lu_factor(Ad)
    x = sla.lu_solve(lu, b)
    r = x - x_target
    lam = sla.lu_solve(lu, r, trans=1)
    rows = np.repeat(np.arange(op.shape[0]), np.diff(op.indptr))
    dvals = -lam[rows] * x[op.indices]
    return 0.5 * float(r @ r), dvals, lam, x

