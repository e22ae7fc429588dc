"""Row-partitioned solve (Alg. 4 over row blocks, Sec. 5; four reductions
per block, Sec. 2.2) run as gloo ranks on the CPU.

The distributed driver (paper_2303_08953_gb300.rowshard) and the library's
host pieces it calls (halo plan, partial Cholesky, combination of the two
BCGS passes, Hessenberg assembly, Givens rotations, Ritz values, Leja
order, estimator) run as they would on GPUs; only the local dense and
sparse kernels are numpy stand-ins here (HostOps), since the CPU has no
CUDA device.  Every rank must take the oracle's decisions (s0, every
block's p and p', columns per cycle) and the gathered x must match the
oracle's within 1e-9.  A GPU variant runs the same ranks with the CUDA
kernels (tests/test_gpu_rowshard.py).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads as W                       # noqa: E402
from oracle import sgmres_oracle as O       # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


class HostOps:
    """numpy stand-ins for the library's local kernels (same interface as
    rowshard.DeviceOps), on CPU torch tensors."""

    def __init__(self, block):
        import scipy.sparse as sp
        import torch
        self.torch = torch
        self.A = sp.csr_matrix((block.val, block.colind, block.rowptr),
                               shape=(block.rows, block.ncols))
        self.send_idx = torch.as_tensor(block.send_idx.astype(np.int64))

    def zeros(self, *shape):
        return self.torch.zeros(shape, dtype=self.torch.float64)

    def tensor(self, a):
        return self.torch.as_tensor(np.array(a, dtype=np.float64))

    def spmv(self, x_ext, y, theta=0.0, gamma=1.0, z=None, c=0.0):
        xe = x_ext.numpy()
        n = y.shape[0]
        v = self.A @ xe - theta * xe[:n]
        if z is not None and c != 0.0:
            v = v + c * z.numpy()
        y.copy_(self.torch.from_numpy(v / gamma))

    def residual(self, b, x_ext, r):
        r.copy_(b - self.torch.from_numpy(self.A @ x_ext.numpy()))

    def dot(self, Q, X, sym=False):
        return self.torch.from_numpy(X.numpy() @ Q.numpy().T)      # (s, i)

    def update(self, Q, W, X, alpha=-1.0, beta=1.0, upper=False):
        Wm = W.numpy().T                                           # (i, s)
        if upper:
            Wm = np.triu(Wm)
        X.copy_(self.torch.from_numpy(beta * X.numpy() + alpha * (Wm.T @ Q.numpy())))

    def pack(self, v, out):
        out.copy_(v[self.send_idx])


SYSTEMS = {
    "stencil2d_40": (lambda: W.config_c1(40), dict(m=40, s=8, tol=1e-10)),
    "convdiff3d_12_est": (lambda: W.config_c2(12),
                          dict(m=48, s=0, s_min=4, s_max=24, tol=1e-10)),
    "randband_6000": (lambda: W.config_c5(6000), dict(m=30, s=0, s_min=1, s_max=30,
                                                      tol=1e-10)),
}


def _worker(rank, world, port, name, out, device_ops):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2303_08953_gb300 import rowshard as RS
        gen, opts = SYSTEMS[name]
        c = gen()
        A = c["A"]
        bounds = RS.row_partition(A.n, world)
        lo, hi = bounds[rank], bounds[rank + 1]
        a, e = A.rowptr[lo], A.rowptr[hi]
        comm = RS.Comm()
        blk = RS.make_row_block(A.rowptr[lo:hi + 1] - a, A.colind[a:e], A.val[a:e],
                                lo, hi, A.n, comm)
        if device_ops:
            ops = RS.DeviceOps(blk, 0)
            b = ops.tensor(c["b"][lo:hi])
        else:
            ops = HostOps(blk)
            b = torch.as_tensor(c["b"][lo:hi].copy())
        sv = RS.RowShardedSolver(blk, ops, comm)
        x, info = sv.solve(b, **opts)
        xg = sv.gather(x).numpy()
        out[rank] = dict(x=xg, s0=info.s0, s_hist=list(info.s_hist),
                         p1_hist=list(info.p1_hist), s_eff_hist=list(info.s_eff_hist),
                         iters=info.iters, restarts=info.restarts,
                         cycle_iters=list(info.cycle_iters),
                         cycle_relres=list(info.cycle_relres),
                         relres_hist=list(info.relres_hist), converged=info.converged,
                         allreduces=info.allreduces, exchanges=info.exchanges,
                         halo=int(blk.halo.size))
        if device_ops:
            ops.close()
    finally:
        dist.destroy_process_group()


def run_ranks(name, world, device_ops=False):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, name, out, device_ops))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
        assert p.exitcode == 0
    return [out[r] for r in range(world)]


def check_against_oracle(name, res):
    gen, opts = SYSTEMS[name]
    c = gen()
    ro = O.adaptive_sgmres(c["A"], c["b"], **opts)
    for r in res:
        assert r["converged"] and ro.converged
        assert r["s0"] == ro.s0
        assert r["s_hist"] == list(ro.s_hist)
        assert r["p1_hist"] == list(ro.p1_hist)
        assert r["s_eff_hist"] == list(ro.s_eff_hist)
        assert r["iters"] == ro.iters and r["restarts"] == ro.restarts
        assert r["cycle_iters"] == list(ro.cycle_iters)
        co = np.array(ro.cycle_relres)
        assert np.all(np.abs(np.array(r["cycle_relres"]) - co) <= np.maximum(1e-8 * co, 1e-13))
        ho = np.array(ro.relres_hist)
        assert np.all(np.abs(np.array(r["relres_hist"]) - ho) <= np.maximum(1e-6 * ho, 1e-13))
        err = np.linalg.norm(r["x"] - ro.x) / np.linalg.norm(ro.x)
        assert err <= 1e-9, err
    return ro


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_two_ranks_match_the_single_rank_oracle(name):
    res = run_ranks(name, 2)
    ro = check_against_oracle(name, res)
    # both ranks agree exactly (replicated small algebra on reduced sums)
    assert np.array_equal(res[0]["x"], res[1]["x"])
    assert res[0]["relres_hist"] == res[1]["relres_hist"]
    assert all(r["halo"] > 0 for r in res)
    # four reductions per block (W, Gram, R', Gram) besides the pre-pass's
    # and the residual norms
    blocks = len(ro.s_hist)
    k = res[0]["s0"] if SYSTEMS[name][1]["s"] > 0 else None
    assert res[0]["allreduces"] >= 4 * blocks
    if k is not None:
        pre = sum(j + 3 for j in range(k))        # ||w||, j+1 projections, ||w'||
        assert res[0]["allreduces"] == 4 * blocks + pre + 1 + len(ro.cycle_relres)


def test_three_ranks_uneven_blocks():
    res = run_ranks("stencil2d_40", 3)
    check_against_oracle("stencil2d_40", res)


def test_halo_plan_matches_brute_force():
    """sg_host_halo_plan against the definition: the sorted distinct
    columns outside [lo, hi) and every entry renumbered."""
    import paper_2303_08953_gb300 as sg
    A = W.config_c5(3000)["A"]
    for lo, hi in [(0, 1000), (1000, 2500), (2500, 3000), (0, 3000)]:
        a, e = A.rowptr[lo], A.rowptr[hi]
        cols = A.colind[a:e]
        loc, halo = sg.halo_plan(A.rowptr[lo:hi + 1] - a, cols, lo, hi)
        want = np.unique(cols[(cols < lo) | (cols >= hi)])
        assert np.array_equal(halo, want)
        own = (cols >= lo) & (cols < hi)
        assert np.array_equal(loc[own], cols[own] - lo)
        assert np.array_equal(halo[loc[~own] - (hi - lo)], cols[~own])
