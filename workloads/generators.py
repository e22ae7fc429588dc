"""Generators for the five synthetic workloads and the small diagonal test
matrices of the paper's stability study (Sec. 4.1, 4.2.1, 4.4.1).

Randomness: numpy's PCG64 generator (``numpy.random.default_rng(seed)``),
drawn in the order documented per function, so one seed gives one system on
every machine.  Every matrix is returned in CSR form with int32 row pointers
and column indices (columns sorted within each row) and float64 values.
Grid unknowns are numbered lexicographically with x fastest:
``i = ix + nx*iy (+ nx*ny*iz)``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """Compressed sparse row matrix (square, ``n`` rows)."""
    n: int
    rowptr: np.ndarray  # int32, n+1
    colind: np.ndarray  # int32, nnz
    val: np.ndarray     # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.colind, self.rowptr),
                             shape=(self.n, self.n))


def _assemble(n, rows, cols, vals):
    """Build a CSR from coordinate triplets (no duplicates allowed)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    vals = np.asarray(vals, dtype=np.float64)[order]
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    assert rowptr[-1] < 2**31, "int32 CSR requires nnz < 2^31"
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), vals)


def _grid_stencil(shape, diag, offdiag):
    """Constant-coefficient stencil on a box grid with Dirichlet boundary.

    ``shape`` = (nx, ny[, nz]); ``offdiag`` maps (axis, +1/-1) to the value
    of the coupling to the neighbour in that direction.
    """
    dims = len(shape)
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for ax in range(dims):
        coords.append(rem % shape[ax])
        rem //= shape[ax]
    strides = [int(np.prod(shape[:ax])) for ax in range(dims)]
    rows, cols, vals = [idx], [idx], [np.full(n, float(diag))]
    for (ax, sgn), v in offdiag.items():
        ok = coords[ax] + sgn >= 0 if sgn < 0 else coords[ax] + sgn < shape[ax]
        r = idx[ok]
        rows.append(r)
        cols.append(r + sgn * strides[ax])
        vals.append(np.full(r.size, float(v)))
    return _assemble(n, np.concatenate(rows), np.concatenate(cols),
                     np.concatenate(vals))


def stencil2d(nx=64, ny=64, diag=4.0, west=-1.1, south=-1.1, east=-0.9,
              north=-0.9) -> CSR:
    """2D 5-point nonsymmetric stencil (west = -x neighbour, south = -y)."""
    return _grid_stencil((nx, ny), diag, {(0, -1): west, (1, -1): south,
                                           (0, +1): east, (1, +1): north})


def stencil3d_convdiff(n=128, diag=6.0, upwind=-1.2, downwind=-0.8) -> CSR:
    """3D 7-point convection-diffusion: on each axis the coupling to the
    -1 neighbour (upwind for a flow in the +axis direction) is ``upwind``,
    to the +1 neighbour ``downwind``."""
    off = {}
    for ax in range(3):
        off[(ax, -1)] = upwind
        off[(ax, +1)] = downwind
    return _grid_stencil((n, n, n), diag, off)


def vardiff3d(n=192, sigma=1.5, shift=1e-3, skew=0.1, seed=2):
    """3D 7-point variable-coefficient diffusion with a convection skew.

    Draw order (one PCG64 stream, ``seed``): g for the x faces, shape
    (n, n, n+1) indexed [iz, iy, face_x]; then y faces (n, n+1, n); then z
    faces (n+1, n, n); each g ~ N(0, sigma^2), conductivity k = exp(g).
    Boundary faces (Dirichlet) add to the diagonal only.  Off-diagonal of an
    interior face between i and i+e: a[i, i+e] = -k - skew,
    a[i+e, i] = -k + skew.  Diagonal = sum of the 6 face conductivities +
    ``shift``.  Returns (CSR, rng) so the caller can keep drawing from the
    same stream (right-hand side).
    """
    rng = np.random.default_rng(seed)
    kx = np.exp(sigma * rng.standard_normal((n, n, n + 1)))
    ky = np.exp(sigma * rng.standard_normal((n, n + 1, n)))
    kz = np.exp(sigma * rng.standard_normal((n + 1, n, n)))
    N = n ** 3
    diag = (kx[:, :, :-1] + kx[:, :, 1:] + ky[:, :-1, :] + ky[:, 1:, :]
            + kz[:-1, :, :] + kz[1:, :, :]).reshape(-1) + shift
    idx = np.arange(N, dtype=np.int64).reshape(n, n, n)
    rows, cols, vals = [idx.reshape(-1)], [idx.reshape(-1)], [diag]
    for face, sl_lo, sl_hi, stride in (
            (kx[:, :, 1:-1], (slice(None), slice(None), slice(0, -1)),
             (slice(None), slice(None), slice(1, None)), 1),
            (ky[:, 1:-1, :], (slice(None), slice(0, -1), slice(None)),
             (slice(None), slice(1, None), slice(None)), n),
            (kz[1:-1, :, :], (slice(0, -1), slice(None), slice(None)),
             (slice(1, None), slice(None), slice(None)), n * n)):
        lo = idx[sl_lo].reshape(-1)
        hi = idx[sl_hi].reshape(-1)
        k = face.reshape(-1)
        rows += [lo, hi]
        cols += [hi, lo]
        vals += [-k - skew, -k + skew]
    A = _assemble(N, np.concatenate(rows), np.concatenate(cols),
                  np.concatenate(vals))
    return A, rng


def aniso2d(n=1024, ratio=10.0, seed=3):
    """2D 5-point anisotropic diffusion with random edge conductivities.

    Draw order (PCG64, ``seed``): g for the x edges, shape (n, n+1) indexed
    [iy, edge_x]; then the y edges, shape (n+1, n); g ~ N(0, 1).  Edge
    conductivity: x edges ``ratio*exp(g)``, y edges ``exp(g)``.  Boundary
    edges (Dirichlet) add to the diagonal only; the matrix is symmetric with
    diagonal = sum of the 4 edge conductivities.  Returns (CSR, rng).
    """
    rng = np.random.default_rng(seed)
    kx = ratio * np.exp(rng.standard_normal((n, n + 1)))
    ky = np.exp(rng.standard_normal((n + 1, n)))
    N = n * n
    diag = (kx[:, :-1] + kx[:, 1:] + ky[:-1, :] + ky[1:, :]).reshape(-1)
    idx = np.arange(N, dtype=np.int64).reshape(n, n)
    rows, cols, vals = [idx.reshape(-1)], [idx.reshape(-1)], [diag]
    lo, hi = idx[:, :-1].reshape(-1), idx[:, 1:].reshape(-1)
    k = kx[:, 1:-1].reshape(-1)
    rows += [lo, hi]; cols += [hi, lo]; vals += [-k, -k]
    lo, hi = idx[:-1, :].reshape(-1), idx[1:, :].reshape(-1)
    k = ky[1:-1, :].reshape(-1)
    rows += [lo, hi]; cols += [hi, lo]; vals += [-k, -k]
    A = _assemble(N, np.concatenate(rows), np.concatenate(cols),
                  np.concatenate(vals))
    return A, rng


def random_band(N=4_194_304, k=24, band=4096, dominance=1.1, seed=4,
                chunk=1 << 20):
    """Unstructured random sparse matrix.

    Row i gets ``k`` distinct off-diagonal columns drawn uniformly from
    [max(0, i-band), min(N-1, i+band)] without i, values N(0, 1), and the
    diagonal ``dominance`` x the row's off-diagonal absolute sum.
    Draw order (PCG64, ``seed``), rows in chunks of ``chunk``: 2k candidate
    offsets per row; the first k distinct valid ones are kept (rows that get
    fewer, vanishingly rare, redraw 4k candidates); then N(0,1) values for
    the kept entries in row-major order.  Returns (CSR, rng).
    """
    assert N >= k + 1
    rng = np.random.default_rng(seed)
    nnz = N * (k + 1)
    assert nnz < 2**31
    colind = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    for r0 in range(0, N, chunk):
        r1 = min(N, r0 + chunk)
        rows = np.arange(r0, r1, dtype=np.int64)
        lo = np.maximum(0, rows - band)
        hi = np.minimum(N - 1, rows + band)
        picked = _pick_distinct(rng, rows, lo, hi, k, 2 * k)
        bad = np.where(picked[:, -1] < 0)[0]
        if bad.size:
            picked[bad] = _pick_distinct(rng, rows[bad], lo[bad], hi[bad],
                                         k, 4 * k)
            assert (picked[:, -1] >= 0).all()
        offv = rng.standard_normal((r1 - r0, k))
        dg = dominance * np.abs(offv).sum(axis=1)
        cols = np.concatenate([picked, rows[:, None]], axis=1)
        vals = np.concatenate([offv, dg[:, None]], axis=1)
        order = np.argsort(cols, axis=1, kind="stable")
        cols = np.take_along_axis(cols, order, axis=1)
        vals = np.take_along_axis(vals, order, axis=1)
        colind[r0 * (k + 1):r1 * (k + 1)] = cols.reshape(-1)
        val[r0 * (k + 1):r1 * (k + 1)] = vals.reshape(-1)
    rowptr = (np.arange(N + 1, dtype=np.int64) * (k + 1)).astype(np.int32)
    return CSR(N, rowptr, colind, val), rng


def _pick_distinct(rng, rows, lo, hi, k, ncand):
    width = (hi - lo + 1)[:, None]
    cand = lo[:, None] + np.floor(rng.random((rows.size, ncand)) * width
                                  ).astype(np.int64)
    valid = cand != rows[:, None]
    order = np.argsort(cand, axis=1, kind="stable")
    srt = np.take_along_axis(cand, order, axis=1)
    dup_sorted = np.zeros_like(valid)
    dup_sorted[:, 1:] = srt[:, 1:] == srt[:, :-1]
    dup = np.empty_like(valid)
    np.put_along_axis(dup, order, dup_sorted, axis=1)
    valid &= ~dup
    rank = np.cumsum(valid, axis=1)
    keep = valid & (rank <= k)
    out = np.full((rows.size, k), -1, dtype=np.int64)
    rr, cc = np.nonzero(keep)
    out[rr, rank[rr, cc] - 1] = cand[rr, cc]
    return out


def diagonal(eigs) -> CSR:
    """Diagonal matrix with the given diagonal (the paper's test matrices)."""
    eigs = np.asarray(eigs, dtype=np.float64)
    n = eigs.size
    return CSR(n, np.arange(n + 1, dtype=np.int32),
               np.arange(n, dtype=np.int32), eigs.copy())


def jacobi_chain(n, stride=7919):
    """Symmetric tridiagonal (Jacobi) matrix laid along the row chain
    r_i = (i * stride) mod n (stride coprime to n), so consecutive chain
    rows sit far apart: A[r_i, r_i] = a_i = 2 + (i mod 5)/4 and
    A[r_i, r_{i+1}] = A[r_{i+1}, r_i] = b_i = 1 (i even) or 1/2 (i odd).
    Every entry and every b_i^2 is exact in FP32.  Returns (A, a, b); the
    chain starts at row r_0 = 0."""
    import math
    if math.gcd(stride, n) != 1:
        raise ValueError("stride must be coprime to n")
    i = np.arange(n, dtype=np.int64)
    r = (i * stride) % n
    a = 2.0 + (i % 5) / 4.0
    b = np.where(i[:-1] % 2 == 0, 1.0, 0.5)
    rows = np.concatenate([r, r[:-1], r[1:]])
    cols = np.concatenate([r, r[1:], r[:-1]])
    vals = np.concatenate([a, b, b])
    return _assemble(n, rows, cols, vals), a, b


def uniform_vector(n, rng) -> np.ndarray:
    """n draws from U(-1, 1)."""
    return rng.uniform(-1.0, 1.0, n)


def rhs_from_solution(A: CSR, xstar: np.ndarray) -> np.ndarray:
    """b = A x* through scipy's CSR product (input construction only)."""
    return A.to_scipy() @ xstar


# ---------------------------------------------------------------- configs
def config_c1(n=64):
    """2D 5-pt nonsymmetric stencil, n x n (default 64x64, N=4096);
    x* ~ U(-1,1) seed 0; b = A x*; m=60, s0=10 fixed, tol 1e-10."""
    A = stencil2d(n, n)
    xs = uniform_vector(A.n, np.random.default_rng(0))
    return dict(name=f"c1_stencil2d_{n}x{n}", A=A, xstar=xs,
                b=rhs_from_solution(A, xs), m=60, s=10, s_min=1, s_max=10,
                tol=1e-10)


def config_c2(n=128):
    """3D 7-pt convection-diffusion n^3 (default 128^3, N=2,097,152);
    x* ~ U(-1,1) seed 1; m=240, s auto in [20,120], tol 1e-10."""
    A = stencil3d_convdiff(n)
    xs = uniform_vector(A.n, np.random.default_rng(1))
    return dict(name=f"c2_convdiff3d_{n}^3", A=A, xstar=xs,
                b=rhs_from_solution(A, xs), m=240, s=0, s_min=20, s_max=120,
                tol=1e-10)


def config_c3(n=192):
    """3D variable-coefficient diffusion n^3 (default 192^3); x* from the
    seed-2 stream after the conductivities; m=200, s <= 60."""
    A, rng = vardiff3d(n)
    xs = uniform_vector(A.n, rng)
    return dict(name=f"c3_vardiff3d_{n}^3", A=A, xstar=xs,
                b=rhs_from_solution(A, xs), m=200, s=0, s_min=1, s_max=60,
                tol=1e-10)


def config_c4(n=1024):
    """2D anisotropic diffusion n^2 (default 1024^2); from the seed-3 stream
    after the conductivities: x* ~ U(-1,1) (b = A x*), then the loss target
    x_t ~ U(-1,1); m=120, s auto."""
    A, rng = aniso2d(n)
    xs = uniform_vector(A.n, rng)
    xt = uniform_vector(A.n, rng)
    return dict(name=f"c4_aniso2d_{n}^2", A=A, xstar=xs, xtarget=xt,
                b=rhs_from_solution(A, xs), m=120, s=0, s_min=1, s_max=120,
                tol=1e-10)


def config_c5(N=4_194_304):
    """Random banded sparse matrix, N rows, 24 off-diagonals within +-4096;
    x* from the seed-4 stream after the values, then the loss target
    x_t ~ U(-1,1) of the adjoint run; m=120, s auto."""
    A, rng = random_band(N)
    xs = uniform_vector(A.n, rng)
    xt = uniform_vector(A.n, rng)
    return dict(name=f"c5_randband_{N}", A=A, xstar=xs, xtarget=xt,
                b=rhs_from_solution(A, xs), m=120, s=0, s_min=1, s_max=120,
                tol=1e-10)


CONFIGS = dict(c1=config_c1, c2=config_c2, c3=config_c3, c4=config_c4,
               c5=config_c5)
