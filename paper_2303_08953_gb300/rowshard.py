"""Row-partitioned adaptive s-step GMRES: Alg. 4 with the rows of A, b, x
and of every Krylov vector split into consecutive blocks, one per process
(the paper's parallel layout, Sec. 5).

Per process and per block of s columns (Sec. 2.2):
  * matrix powers kernel: s SpMVs on the local row block, each after a halo
    exchange of the entries of the input vector that other processes own;
  * BCGS2 with partial CholQR: every tall-skinny product (W = Q^T X, the
    Gram X^T X, R' = Q^T Q_k, the second Gram) is a local partial summed by
    one allreduce -- four per block;
  * the small algebra (partial Cholesky with ICE, triangular inverses,
    combination of the two passes, Hessenberg assembly, Givens rotations,
    the step-size decisions) is replicated on every process from the same
    reduced numbers, so every process takes the same decisions.
The Ritz pre-pass is MGS-Arnoldi with one allreduce per projection
(Sec. 3.4).  Communication goes through torch.distributed: NCCL between
GPUs (device tensors), or gloo (host tensors; device tensors are staged
through host memory).

Local arithmetic is delegated to an `ops` object; `DeviceOps` runs it in
the library's CUDA kernels on this process's GPU.  The host small algebra
is the library's (sg_host_* calls).  Nothing here computes on its own: this
module orders the steps, moves buffers and calls the collectives.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch
import torch.distributed as dist

from . import (Solver, SgError, SG_EINVAL, basis, combine_r, assemble_hessenberg,
               estimate_step, gather, givens_column, givens_solve, halo_plan,
               hessenberg_eigvals, leja_order, partial_cholesky,
               scaling_coefficients, upper_inverse)


# ---------------------------------------------------------------- comm
class Comm:
    """The process group's collectives; gloo gets host copies of device
    tensors (it has no device all-to-all)."""

    def __init__(self, group=None):
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.stage = dist.get_backend(group) == "gloo"

    def allreduce(self, t):
        if self.stage and t.is_cuda:
            h = t.cpu()
            dist.all_reduce(h, group=self.group)
            t.copy_(h)
        else:
            dist.all_reduce(t, group=self.group)
        return t

    def alltoall(self, out, inp, out_splits, in_splits):
        if self.stage and (out.is_cuda or inp.is_cuda):
            ho = torch.empty(out.shape, dtype=out.dtype)
            dist.all_to_all_single(ho, inp.cpu(), out_splits, in_splits, group=self.group)
            out.copy_(ho)
        else:
            dist.all_to_all_single(out, inp, out_splits, in_splits, group=self.group)
        return out

    def allgather_ints(self, values):
        t = torch.tensor(values, dtype=torch.int64)
        outs = [torch.empty_like(t) for _ in range(self.world)]
        dist.all_gather(outs, t, group=self.group)
        return [o.tolist() for o in outs]


# ---------------------------------------------------------------- partition
def row_partition(n, world):
    """Consecutive row blocks [bounds[r], bounds[r+1]) of near-equal size."""
    return [(n * r) // world for r in range(world + 1)]


@dataclass
class RowBlock:
    """This process's rows [lo, hi) in local numbering and its halo
    exchange plan (sg_host_halo_plan)."""
    lo: int
    hi: int
    n: int
    rowptr: np.ndarray
    colind: np.ndarray            # local columns: [own rows; halo]
    val: np.ndarray
    halo: np.ndarray              # global columns of the halo, sorted
    recv_counts: list = field(default_factory=list)   # halo entries per owner
    send_counts: list = field(default_factory=list)   # own entries per peer
    send_idx: np.ndarray = None   # local rows packed for the peers, in order

    @property
    def rows(self):
        return self.hi - self.lo

    @property
    def ncols(self):
        return self.rows + self.halo.size


def make_row_block(rowptr, colind, val, lo, hi, n, comm):
    """Rows [lo, hi) of a global CSR (rowptr of the block starting at 0,
    global column indices) and the exchange lists agreed with the peers."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    loc, halo = halo_plan(rp, ci, lo, hi)
    bounds = [b[0] for b in comm.allgather_ints([lo])] + [n]
    owners = np.searchsorted(np.asarray(bounds[1:]), halo, side="right")
    recv = np.bincount(owners, minlength=comm.world).astype(np.int64).tolist()
    # tell every owner which of its rows this process needs
    counts = comm.allgather_ints(recv)
    send = [counts[q][comm.rank] for q in range(comm.world)]
    req = torch.as_tensor(halo.astype(np.int64))
    got = torch.empty(sum(send), dtype=torch.int64)
    dist.all_to_all_single(got, req, send, recv, group=comm.group)
    send_idx = (got.numpy() - lo).astype(np.int32)
    if send_idx.size and (send_idx.min() < 0 or send_idx.max() >= hi - lo):
        raise SgError(SG_EINVAL, "halo request outside the owner's rows")
    return RowBlock(lo, hi, n, rp, loc, np.ascontiguousarray(val, dtype=np.float64), halo,
                    recv, send, send_idx)


# ---------------------------------------------------------------- local ops
class DeviceOps:
    """Local kernels of one process on its GPU, through the library: the
    row block is ingested with sg_analyze_rows; vectors are float64 CUDA
    tensors, a block of k vectors a (k, rows) tensor (column-major n x k)."""

    def __init__(self, block: RowBlock, device=0):
        self.dev = torch.device("cuda", device)
        self.solver = Solver(device)
        self.solver.analyze_rows(block.rowptr, block.colind, block.val, block.ncols)
        self.rows = block.rows
        self.send_idx = torch.as_tensor(block.send_idx, device=self.dev)

    def zeros(self, *shape):
        return torch.zeros(shape, dtype=torch.float64, device=self.dev)

    def tensor(self, a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=self.dev)

    def spmv(self, x_ext, y, theta=0.0, gamma=1.0, z=None, c=0.0):
        self.solver.spmv_newton(x_ext, theta, gamma, z, c, out=y)

    def residual(self, b, x_ext, r):
        self.solver.residual(b, x_ext, out=r)

    def dot(self, Q, X, sym=False):
        """Local partial of Q^T X as an (s, i) tensor (column-major i x s)."""
        return self.solver.block_dot(Q, X, sym=sym)

    def update(self, Q, W, X, alpha=-1.0, beta=1.0, upper=False):
        """X = beta X + alpha Q W on the local rows (W an (s, i) tensor)."""
        self.solver.block_update(Q, W, X, alpha=alpha, beta=beta, upper=upper)

    def pack(self, v, out):
        gather(self.send_idx, v, out)

    def close(self):
        self.solver.close()


# ---------------------------------------------------------------- solver
@dataclass
class ShardInfo:
    converged: bool = False
    s0: int = 0
    iters: int = 0
    restarts: int = 0
    final_relres: float = 0.0
    s_hist: list = field(default_factory=list)
    s_eff_hist: list = field(default_factory=list)
    p1_hist: list = field(default_factory=list)
    relres_hist: list = field(default_factory=list)
    cycle_relres: list = field(default_factory=list)
    cycle_iters: list = field(default_factory=list)
    ritz: np.ndarray = None
    gamma: np.ndarray = None
    allreduces: int = 0
    exchanges: int = 0


class RowShardedSolver:
    """Alg. 4 with restarts over a row-partitioned system (see the module
    docstring).  `ops` provides the local kernels (DeviceOps on a GPU)."""

    def __init__(self, block: RowBlock, ops, comm: Comm):
        self.b, self.ops, self.comm = block, ops, comm
        self.rows = block.rows
        self.ext = ops.zeros(block.ncols)
        self.sendbuf = ops.zeros(max(1, int(block.send_idx.size)))
        self.tmp = ops.zeros(block.rows)
        self.info = None

    # ---- communication steps
    def _exchange(self, v):
        """ext = [v; entries of v owned by the peers that this block's rows
        reference] (the SpMV input)."""
        blk = self.b
        self.ext[:self.rows].copy_(v)
        ns = int(blk.send_idx.size)
        if ns:
            self.ops.pack(v, self.sendbuf[:ns])
        self.comm.alltoall(self.ext[self.rows:], self.sendbuf[:ns], blk.recv_counts,
                           blk.send_counts)
        self.info.exchanges += 1
        return self.ext

    def _reduce(self, t):
        self.info.allreduces += 1
        return self.comm.allreduce(t)

    def _dot(self, Q, X, sym=False):
        """Q^T X summed over all processes, as an (i, s) host array."""
        W = self.ops.dot(Q, X, sym=sym)
        self._reduce(W)
        return W.cpu().numpy().T.copy(order="F")

    def _norm(self, v):
        return math.sqrt(self._dot(v[None, :], v[None, :])[0, 0])

    def _scale(self, src, dst, a):
        """dst = a src (through a scratch vector when they are the same)."""
        out = self.tmp if src.data_ptr() == dst.data_ptr() else dst
        self.ops.update(src[None, :], self.ops.tensor([[a]]), out[None, :], alpha=1.0,
                        beta=0.0)
        if out is not dst:
            dst.copy_(out)

    # ---- Ritz pre-pass (Sec. 3.4): MGS-Arnoldi, one reduction per projection
    def _prepass(self, q1, k):
        V = self.ops.zeros(k + 1, self.rows)
        V[0].copy_(q1)
        H = np.zeros((k + 1, k), order="F")
        for j in range(k):
            w = V[j + 1]
            self.ops.spmv(self._exchange(V[j]), w)
            wn0 = self._norm(w)
            for l in range(j + 1):
                h = self._dot(V[l][None, :], w[None, :])[0, 0]
                H[l, j] = h
                self.ops.update(V[l][None, :], self.ops.tensor([[h]]), w[None, :])
            hn = self._norm(w)
            H[j + 1, j] = hn
            if not (hn > 1e-12 * wn0) or not math.isfinite(hn):
                return H, j + 1
            self._scale(w, w, 1.0 / hn)
        return H, k

    # ---- Alg. 4 with restarts
    def solve(self, b, x0=None, m=60, s=10, s_min=1, s_max=0, tol=1e-10, max_iters=0,
              omega=1e7, omega_est=1e7, basis_kind="scaled_newton"):
        """b, x0: this process's rows (tensors of the ops' kind).  Returns
        (x rows, ShardInfo); every process returns the same decisions."""
        ops, n = self.ops, self.rows
        self.info = info = ShardInfo()
        x = ops.zeros(n) if x0 is None else x0.clone()
        r = ops.zeros(n)
        max_iters = max_iters if max_iters > 0 else 50 * m
        if s_max <= 0:
            s_max = s if s > 0 else m
        ops.residual(b, self._exchange(x), r)
        beta0 = self._norm(r)
        if beta0 == 0.0:
            info.converged = True
            return x, info
        beta = beta0
        theta = gam = None
        cur_s = total = 0
        Q = ops.zeros(m + 1, n)
        kk = s if s > 0 else s_max
        Vb = ops.zeros(max(kk, 1) + 1, n)
        Yb = ops.zeros(max(kk, 1), n)
        while True:
            self._scale(r, Q[0], 1.0 / beta)
            if theta is None:
                k = min(kk, m)
                Hp, steps = self._prepass(Q[0], k)
                ritz = leja_order(hessenberg_eigvals(Hp[:steps, :steps]))
                gam = scaling_coefficients(ritz)
                theta = ritz
                if basis_kind == "monomial":
                    theta, gam = np.zeros(steps, complex), np.ones(steps)
                elif basis_kind == "newton":
                    gam = np.ones(steps)
                info.ritz, info.gamma = ritz, gam
                if s > 0:
                    cur_s = min(s, steps)
                else:
                    cur_s, _ = estimate_step(ritz, omega_est=omega_est, s_min=s_min,
                                             s_max=min(s_max, steps))
                    cur_s = min(cur_s, steps)
                cur_s = max(cur_s, 1)
                info.s0 = cur_s
            H = np.zeros((m + 1, m), order="F")
            Hr = np.zeros((m + 1, m), order="F")
            cs, sn, g = np.zeros(m), np.zeros(m), np.zeros(m + 1)
            g[0] = beta
            i, jdone, stop = 1, 0, False
            while i <= m and not stop:
                s_eff = min(cur_s, m + 1 - i)
                th, cc, gg, _ = basis(theta, gam, s_eff)
                # matrix powers kernel (Sec. 2), V[0] = Q_i
                Vb[0].copy_(Q[i - 1])
                for j in range(s_eff):
                    z = Vb[j - 1] if cc[j] != 0.0 else None
                    ops.spmv(self._exchange(Vb[j]), Vb[j + 1], th[j], gg[j], z, cc[j])
                X = Vb[1:s_eff + 1]
                Qi = Q[:i]
                # first BCGS and partial CholQR (Alg. 4, Alg. 3)
                W = self._dot(Qi, X)
                ops.update(Qi, ops.tensor(W.T), X)
                G = self._dot(X, X, sym=True)
                p1, Z1, _ = partial_cholesky(G, omega)
                info.s_eff_hist.append(s_eff)
                info.p1_hist.append(p1)
                breakdown = False
                if p1 == 0:
                    breakdown, q = True, 1
                    R_top, R_kk = W[:, :1].copy(order="F"), np.zeros((1, 1), order="F")
                else:
                    Y = Yb[:p1]
                    ops.update(X[:p1], ops.tensor(upper_inverse(Z1, p1).T), Y, alpha=1.0,
                               beta=0.0, upper=True)
                    # second BCGS and partial CholQR
                    Rp = self._dot(Qi, Y)
                    ops.update(Qi, ops.tensor(Rp.T), Y)
                    G2 = self._dot(Y, Y, sym=True)
                    p2, R2, _ = partial_cholesky(G2, omega)
                    if p2 == 0:
                        breakdown, q = True, 1
                        R_top = np.asfortranarray((W[:, 0] + Rp[:, 0] * Z1[0, 0])[:, None])
                        R_kk = np.zeros((1, 1), order="F")
                    else:
                        q = p2
                        R_top, R_kk = combine_r(W, Rp, Z1, R2, q)
                        ops.update(Y[:q], ops.tensor(upper_inverse(R2, q).T), Q[i:i + q],
                                   alpha=1.0, beta=0.0, upper=True)
                _, _, _, Bq = basis(theta, gam, q)
                assemble_hessenberg(H, i, R_top, R_kk, Bq)
                info.s_hist.append(0 if breakdown else q)
                for c in range(q):
                    j = i - 1 + c
                    rel = givens_column(Hr, cs, sn, g, H, j) / beta0
                    info.relres_hist.append(rel)
                    jdone = j + 1
                    if rel <= tol or breakdown:
                        stop = True
                        break
                if not breakdown and q < s_eff:
                    cur_s = q                         # Alg. 4: s = p
                i += q
                if total + jdone >= max_iters:
                    stop = True
            # end of cycle: least squares, x += Q y, true residual
            y = givens_solve(Hr, g, jdone)
            ops.update(Q[:jdone], ops.tensor(y[None, :]), x[None, :], alpha=1.0, beta=1.0)
            ops.residual(b, self._exchange(x), r)
            beta = self._norm(r)
            total += jdone
            rel_true = beta / beta0
            info.cycle_relres.append(rel_true)
            info.cycle_iters.append(jdone)
            if rel_true <= tol or beta == 0.0:
                info.converged = True
                break
            if total >= max_iters:
                break
        info.iters = total
        info.restarts = len(info.cycle_relres) - 1
        info.final_relres = info.cycle_relres[-1]
        return x, info

    def gather(self, x):
        """The whole solution on every process (for checks): host copies of
        every block, padded to the longest for the all-gather."""
        bounds = [v[0] for v in self.comm.allgather_ints([self.b.lo])] + [self.b.n]
        sizes = [hi - lo for lo, hi in zip(bounds[:-1], bounds[1:])]
        pad = torch.zeros(max(sizes), dtype=torch.float64)
        pad[:self.rows].copy_(x.cpu())
        parts = [torch.empty_like(pad) for _ in sizes]
        dist.all_gather(parts, pad, group=self.comm.group)
        return torch.cat([p[:k] for p, k in zip(parts, sizes)])
