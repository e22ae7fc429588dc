"""CPU checks of the C library without a GPU: every symbol declared in
include/sgmres.h is exported, and the host small-dense algebra of the
library (partial Cholesky + ICE, Ritz values, Leja order, scaling
coefficients, step-size estimator) agrees with the oracle."""
import math
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import sgmres_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sg():
    import paper_2303_08953_gb300 as sg
    return sg


def test_header_symbols_exported(sg):
    hdr = open(os.path.join(ROOT, "include", "sgmres.h")).read()
    names = set(re.findall(r"\b(sg_[a-z0-9_]+)\s*\(", hdr))
    assert names, "no declarations found"
    for nm in names:
        assert hasattr(sg.lib, nm), f"{nm} declared but not exported"
    assert names <= set(sg.EXPORTED) | names


def test_partial_cholesky_matches_oracle(sg):
    rng = np.random.default_rng(11)
    for trial in range(20):
        s = int(rng.integers(2, 30))
        X = rng.standard_normal((400, s)) @ np.diag(np.exp(rng.uniform(-6, 6, s)))
        X[:, -1] += 1e-9 * X[:, 0] if s > 2 else 0
        G = X.T @ X
        p_o, R_o, k_o = O.partial_cholesky(G)
        p_l, R_l, k_l = sg.partial_cholesky(G)
        assert p_l == p_o
        assert np.allclose(R_l, R_o, rtol=1e-12, atol=1e-12 * np.abs(R_o).max())
        assert np.allclose(k_l[:len(k_o)], k_o, rtol=1e-10)


def test_partial_cholesky_edge_cases(sg):
    assert sg.partial_cholesky(np.diag([4.0, 1.0, -1.0, 1.0]))[0] == 2
    assert sg.partial_cholesky(np.zeros((3, 3)))[0] == 0
    R = np.diag(10.0 ** np.arange(10))
    p, _, k = sg.partial_cholesky(R.T @ R, omega=1e7)
    assert p == 8 and np.allclose(k[:9], 10.0 ** np.arange(9))
    G = np.diag([1.0, np.nan, 1.0])
    assert sg.partial_cholesky(G)[0] == 1


def _match_sets(a, b):
    a = np.sort_complex(np.asarray(a))
    b = np.sort_complex(np.asarray(b))
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


def test_hessenberg_eigvals_random(sg):
    rng = np.random.default_rng(12)
    for k in [1, 2, 3, 5, 17, 60, 120]:
        H = np.triu(rng.standard_normal((k, k)), -1)
        ev = sg.hessenberg_eigvals(H)
        assert _match_sets(ev, np.linalg.eigvals(H)) < 1e-9
        # pairs are exact conjugates
        cp = ev[ev.imag > 0]
        for z in cp:
            assert np.any(ev == np.conj(z))


def test_hessenberg_eigvals_arnoldi(sg):
    c = W.config_c1(32)
    op = O.as_operator(c["A"])
    q = c["b"] / np.linalg.norm(c["b"])
    H, st = O.arnoldi_mgs(op, q, 40)
    ev = sg.hessenberg_eigvals(H[:st, :st])
    assert _match_sets(ev, O.ritz_values(H, st)) < 1e-10


def test_leja_and_gamma_match_oracle(sg):
    rng = np.random.default_rng(13)
    for trial in range(10):
        k = int(rng.integers(1, 40))
        re_ = rng.uniform(-3, 8, k)
        nc = int(rng.integers(0, k // 2 + 1))
        vals = list(re_[: k - 2 * nc])
        for t in range(nc):
            a, b = rng.uniform(-1, 5), rng.uniform(0.1, 2)
            vals += [a + 1j * b, a - 1j * b]
        th = np.array(vals, dtype=complex)
        rng.shuffle(th)
        lo = O.leja_order(th)
        ll = sg.leja_order(th)
        assert np.allclose(ll, lo, rtol=0, atol=0)
        assert np.allclose(sg.scaling_coefficients(lo),
                           O.scaling_coefficients(lo), rtol=1e-14)


def test_leja_hand_example(sg):
    assert np.array_equal(sg.leja_order(np.array([2.0, 4.0, 1.0, 3.0])).real,
                          [4.0, 1.0, 3.0, 2.0])


def test_estimator_matches_oracle(sg):
    lam = np.linspace(1.0, 200.0, 200)
    for lmax in (200.0, 2000.0):
        lam2 = lam.copy()
        lam2[-1] = lmax
        op = O.as_operator(W.diagonal(lam2))
        q = np.ones(200) / math.sqrt(200)
        H, st = O.arnoldi_mgs(op, q, 200)
        rz = O.leja_order(O.ritz_values(H, st))
        s_o, n_o = O.estimate_step_size(rz)
        s_l, n_l = sg.estimate_step(rz)
        assert s_l == s_o
        fin = np.isfinite(n_o) & (n_o > 0) & (n_o < 1e300)
        assert np.allclose(n_l[fin], n_o[fin], rtol=1e-9)
        # clamping
        assert sg.estimate_step(rz, s_min=150, s_max=180)[0] == max(150, min(s_o, 180))


def test_estimator_exact_pin(sg):
    """The library's estimator against the hand-computed auxiliary matrix
    of four Leja-ordered values (column 2-norms and the first-crossing
    index with both clamps), independent of the oracle."""
    from test_oracle_pins import ESTIMATOR_EXACT, LEJA4, _leja4_norms_by_hand
    for eps in (0.1, 1e3):
        _, nrm = sg.estimate_step(LEJA4, eps=eps, omega_est=1e300)
        assert np.allclose(nrm, _leja4_norms_by_hand(eps), rtol=1e-14, atol=0)
    for eps, omega, smin, smax, want in ESTIMATOR_EXACT:
        s0, _ = sg.estimate_step(LEJA4, eps=eps, omega_est=omega, s_min=smin,
                                 s_max=smax or 0)
        assert s0 == want, (eps, omega, smin, smax)
