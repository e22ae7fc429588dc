"""Benchmark: time to relative residual 1e-10 of the adaptive s-step GMRES
on the 3D 7-point convection-diffusion system (128^3 grid, N = 2,097,152,
nnz = 14,581,760; m = 240, scaled Newton basis, s estimated in [20, 120]).

One step = one complete solve from x0 = 0 (Ritz pre-pass, estimator, every
block and restart) with A and b resident in HBM.  The FP64 solve gives
`value`; the FP32-basis + FP64-refinement solve and the forward + adjoint
pair are reported beside it on the same system.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (under torchrun): every rank solves its own copy (replicas), the
reported time is the max over ranks.  --impl reference times the CPU oracle
on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# The headline metric covers three forms of the solve and the SpMV roofline;
# `value` is the FP64 solve, the other parts ride on the same line
# (fp32_ir, fwd_adjoint, roofline_spmv).
METRIC = "time to relres 1e-10: FP64 vs FP32-basis+IR, fwd+adjoint; % HBM roofline"
VALUE_IS = ("seconds per FP64 adaptive s-step GMRES solve to relres 1e-10; the FP32-basis+IR "
            "and forward+adjoint times are in fp32_ir / fwd_adjoint, the SpMV % of HBM in "
            "roofline_spmv, the FP32-basis block kernels' rooflines in roofline_fp32")
GRID = 128
SOLVE_KW = dict(m=240, s=0, s_min=20, s_max=120, tol=1e-10)
FP64_ALU_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12   # 152 SMs x 2.07 GHz x 4 flop/clk


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--grid", type=int, default=GRID)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--case", default=None,
                   choices=["solve-fp64", "solve-fp32ir", "spmv", "dot64",
                            "upd64", "dot32", "gram32", "upd32"],
                   help="run one small workload for a profiler and exit")
    return p.parse_args()


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ------------------------------------------------------------ clocks
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
                "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                "clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,"
                "clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, dev_index):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(dev_index)], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ helpers
def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    """Slowest rank's value (the whole job is done when the last rank is);
    works for NCCL (CUDA tensor) and gloo (CPU tensor) process groups."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(grid):
    import workloads as W
    c = W.config_c2(grid)
    A = c["A"]
    return c, {"workload": f"convdiff3d_{grid}^3", "n": int(A.n),
               "nnz": int(A.nnz), "m": SOLVE_KW["m"], "s": "auto[20,120]",
               "basis": "scaled_newton", "tol": SOLVE_KW["tol"],
               "x0": "zero", "l2": "inputs larger than L2 (A 175 MB, Q 4 GB)"}


# DRAM bytes per row of the FP64 block dot (i = 107, s = 106) from one ncu
# capture at n = 2^20: read 2,291,351,000 + write 5,751,296 bytes.
DOT64_DRAM_BYTES_PER_ROW = (2_291_351_000 + 5_751_296) / (1 << 20)


# DRAM bytes per row of the FP32 tensor-core block dot (W = Q^T X) and
# update (X -= Q W) at i = 107, s = 106, from ncu captures at n = 2^20:
# dot read 893,510,656 + write 3,351,552; update read 893,552,896 + write
# 395,420,928.
TCDOT_DRAM_BYTES_PER_ROW = (893_510_656 + 3_351_552) / (1 << 20)
TCUPD_DRAM_BYTES_PER_ROW = (893_552_896 + 395_420_928) / (1 << 20)
# FP32 pipe: 152 SMs x 128 lanes x 2.07 GHz (FADD / FMUL / FFMA each one op)
FP32_ALU_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12
# FP32 instructions per exact Gram product: product, FMA remainder, the six
# additions of the two-sum, two additions into the compensation
GRAM_OPS_PER_PRODUCT = 10


def spmv_bytes(A):
    return 12 * A.nnz + 4 * (A.n + 1) + 8 * A.n + 8 * A.n


# ------------------------------------------------------------ CPU oracle
# Krylov columns the 128^3 solve takes to reach 1e-10 (the oracle and the
# library take identical step-size decisions, so both need this many).
FULL_SOLVE_COLUMNS = 649
SAMPLE = dict(m=240, s=20, tol=1e-10, max_iters=60)


def cpu_oracle_sample(c):
    """The oracle, as it stands, on a bounded sample of the same solve:
    s fixed at 20 (20-step Ritz pre-pass), stopped after 60 Krylov
    columns (3 blocks).  Returns (seconds, columns)."""
    from oracle import sgmres_oracle as O
    t0 = time.perf_counter()
    r = O.adaptive_sgmres(c["A"], c["b"], **SAMPLE)
    return time.perf_counter() - t0, r.iters


def sample_text(dt, its, full):
    return (f"oracle FP64 solve of the same system with s fixed at 20 "
            f"(20-step Ritz pre-pass) stopped after {its} Krylov columns: "
            f"{dt:.2f} s, scaled by columns to the full solve's {full}")


def oracle_threads():
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count()


# ------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import paper_2303_08953_gb300 as sg
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c, cfg = workload(args.grid)
    A = c["A"]
    solver = sg.Solver(local)
    solver.analyze_csr(A)
    b = torch.as_tensor(c["b"], dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2
    stream = torch.cuda.current_stream()

    def one(**kw):
        x, info = solver.solve(b, **SOLVE_KW, **kw)
        return x, info

    launches = [0]

    def timed(kw, steps, warm):
        for _ in range(warm):
            one(**kw)
        torch.cuda.synchronize()
        barrier(world)
        times, info = [], None
        l0 = sg.kernel_launches()
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, info = one(**kw)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        launches[0] = (sg.kernel_launches() - l0) // max(1, steps)
        barrier(world)
        return times, x, info

    # ---- headline: FP64 solve
    clocks = ClockSampler(local)
    times, x, info = timed({}, args.steps, args.warmup)
    n_launch = launches[0]
    clk = clocks.stop()
    ms_step = max_over_ranks(sum(times) / len(times), world)
    xs = c["xstar"]
    err = float(np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs))
    out = {
        "metric": METRIC, "value": ms_step / 1e3, "unit": "s", "value_is": VALUE_IS,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded generator, x* ~ U(-1,1) seed 1, b = A x*)",
        "config": cfg,
        "solve": {"converged": info.converged, "iters": info.iters,
                  "restarts": info.restarts, "s0": info.s0,
                  "s_hist_first": [int(v) for v in info.s_hist[:6]],
                  "final_relres": info.final_relres, "x_err_vs_xstar": err,
                  "phase_ms": {k: round(v, 2) for k, v in info.times_ms.items()},
                  "step_ms_all": [round(t, 2) for t in times],
                  "median_ms": round(float(np.median(times)), 2),
                  "min_ms": round(float(np.min(times)), 2)},
        "gpu_launches": int(n_launch),
        "clocks": clk,
    }

    # ---- variants on the same system
    if not args.no_variants:
        t32, x32, i32 = timed({"precision": "fp32_ir"}, args.steps, 1)
        e32 = float(np.linalg.norm(x32.cpu().numpy() - xs) / np.linalg.norm(xs))
        out["fp32_ir"] = {
            "time_s": max_over_ranks(sum(t32) / len(t32), world) / 1e3,
            "iters": i32.iters, "refinements": i32.refinements,
            "s0": i32.s0, "final_relres": i32.final_relres,
            "x_err_vs_xstar": e32,
            "x_err_vs_fp64": float(np.linalg.norm(x32.cpu().numpy()
                                                  - x.cpu().numpy())
                                   / np.linalg.norm(x.cpu().numpy())),
            "phase_ms": {k: round(v, 2) for k, v in i32.times_ms.items()}}
        # loss L = 0.5 ||x - x_t||^2 with x_t ~ U(-1,1) drawn after x* from
        # x*'s seeded stream (the differentiation workloads' loss); a target
        # of x* itself would make dL/dx the forward error, which lies in a
        # few slow eigenmodes and gives an ill-conditioned adjoint Krylov
        # basis from its first columns
        import workloads as W
        rng_t = np.random.default_rng(1)
        W.uniform_vector(len(xs), rng_t)
        xt = torch.as_tensor(W.uniform_vector(len(xs), rng_t), device=dev)
        fa = []
        for prec in ("fp32_ir", "fp64"):
            ts = []
            for k in range(max(1, args.steps // 2) + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                xf, inf1 = solver.solve(b, precision=prec, **SOLVE_KW)
                g = xf - xt   # dL/dx
                lam, inf2 = solver.solve_adjoint(g, precision=prec, **SOLVE_KW)
                dval = solver.grad_values(lam, xf)
                torch.cuda.synchronize()
                if k:
                    ts.append(time.perf_counter() - t0)
            fa.append({"precision": prec,
                       "time_s": max_over_ranks(sum(ts) / len(ts), world),
                       "fwd_iters": inf1.iters, "adj_iters": inf2.iters,
                       "fwd_relres": inf1.final_relres,
                       "adj_relres": inf2.final_relres,
                       "adj_s0": inf2.s0, "adj_refinements": inf2.refinements,
                       "adj_fp64_iters": inf2.fp64_iters,
                       "adj_phase_ms": {k: round(v, 2) for k, v in inf2.times_ms.items()}})
        out["fwd_adjoint"] = fa

    # ---- roofline of the dominant kernel (FP64 block dot, FP64 pipe)
    n = A.n
    i_blk, s_blk = 107, 106
    Q = torch.randn(i_blk, n, dtype=torch.float64, device=dev)
    X = torch.randn(s_blk, n, dtype=torch.float64, device=dev)
    for _ in range(2):
        solver.block_dot(Q, X)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        solver.block_dot(Q, X)
    e1.record(stream)
    torch.cuda.synchronize()
    t_dot = e0.elapsed_time(e1) / reps / 1e3
    flops = 2.0 * n * i_blk * s_blk
    ach = flops / t_dot / 1e12
    out["roofline"] = {
        "kernel": f"block_dot FP64 (W = Q^T X, i={i_blk}, s={s_blk})",
        "bound": "alu", "achieved": round(ach, 4),
        "peak": round(FP64_ALU_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
        "frac": round(ach / FP64_ALU_PEAK_TFLOPS, 4),
        "traffic": int(round(DOT64_DRAM_BYTES_PER_ROW * n)),
        "traffic_source": "ncu dram__bytes_read+write of dot_tile_kernel at "
                          "n = 2^20 (same i, s), scaled by rows to this n "
                          "(profiles/dot_tile_fp64_n1M_i107_s106.md)",
        "peak_source": "derived: 152 SMs x 2.07 GHz x 4 FP64 flop/clk/SM "
                       "(nominal 1.25 TFLOP/s FP64)"}
    del Q, X
    # secondary: the MPK's SpMV against HBM
    xv = torch.rand(n, dtype=torch.float64, device=dev)
    yv = torch.empty_like(xv)
    for _ in range(5):
        solver.spmv_newton(xv, 0.3, 1.1, out=yv)
    torch.cuda.synchronize()
    reps = 50
    e0.record(stream)
    for _ in range(reps):
        solver.spmv_newton(xv, 0.3, 1.1, out=yv)
    e1.record(stream)
    torch.cuda.synchronize()
    t_sp = e0.elapsed_time(e1) / reps / 1e3
    pk = measured_peaks()
    hbm = pk["hbm_gbs"] if pk else 6800.0
    gbs = spmv_bytes(A) / t_sp / 1e9
    out["roofline_spmv"] = {
        "kernel": "spmv_newton FP64 (one MPK step)", "bound": "hbm",
        "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
        "frac": round(gbs / hbm, 4), "traffic": None,
        "peak_source": "MEASURED_PEAKS.json hbm_gbs" if pk else "fallback"}

    # the FP32-basis path's block kernels at the same block shape
    def event_ms(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    Q32 = torch.randn(i_blk, n, dtype=torch.float32, device=dev)
    X32 = torch.randn(s_blk, n, dtype=torch.float32, device=dev)
    W64 = torch.randn(s_blk, i_blk, dtype=torch.float64, device=dev)
    t_tcd = event_ms(lambda: solver.block_dot32(Q32, X32)) / 1e3
    t_tcu = event_ms(lambda: solver.block_update32(Q32, W64, X32)) / 1e3
    t_gram = event_ms(lambda: solver.block_dot32(X32, X32, sym=True)) / 1e3
    del Q32, X32, W64
    b_tcd = 4.0 * n * (i_blk + s_blk)
    b_tcu = 4.0 * n * (i_blk + 2 * s_blk)
    ops_gram = GRAM_OPS_PER_PRODUCT * n * s_blk * (s_blk + 1) / 2.0
    hbm_src = "MEASURED_PEAKS.json hbm_gbs" if pk else "fallback"
    out["roofline_fp32"] = [
        {"kernel": f"tc_dot FP32 basis (W = Q^T X on tcgen05, 3xTF32, i={i_blk}, s={s_blk})",
         "bound": "hbm", "achieved": round(b_tcd / t_tcd / 1e9, 1), "peak": hbm,
         "unit": "GB/s", "frac": round(b_tcd / t_tcd / 1e9 / hbm, 4),
         "traffic": int(round(TCDOT_DRAM_BYTES_PER_ROW * n)), "peak_source": hbm_src},
        {"kernel": f"tc_update FP32 basis (X -= Q W on tcgen05, 3xTF32, i={i_blk}, s={s_blk})",
         "bound": "hbm", "achieved": round(b_tcu / t_tcu / 1e9, 1), "peak": hbm,
         "unit": "GB/s", "frac": round(b_tcu / t_tcu / 1e9 / hbm, 4),
         "traffic": int(round(TCUPD_DRAM_BYTES_PER_ROW * n)), "peak_source": hbm_src},
        {"kernel": f"gram_exact FP32 basis (X^T X, exact products, s={s_blk})",
         "bound": "alu", "achieved": round(ops_gram / t_gram / 1e12, 2),
         "peak": round(FP32_ALU_PEAK_TOPS, 2), "unit": "T FP32-op/s",
         "frac": round(ops_gram / t_gram / 1e12 / FP32_ALU_PEAK_TOPS, 4), "traffic": None,
         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz"}]

    # ---- end to end through the public API from host buffers
    rp, ci, va = A.rowptr, A.colind, A.val
    bh = np.asarray(c["b"])
    e2e_t = []
    for k in range(3):
        s2 = sg.Solver(local)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2.analyze(rp, ci, va)
        xh, ih = s2.solve(bh, **SOLVE_KW)
        t1 = time.perf_counter()
        s2.close()
        if k:
            e2e_t.append(t1 - t0)
    h2d = rp.nbytes + ci.nbytes + va.nbytes + bh.nbytes + 8 * A.n
    out["e2e"] = {"value": max_over_ranks(sum(e2e_t) / len(e2e_t), world),
                  "unit": "s", "h2d_bytes_per_step": int(h2d),
                  "d2h_bytes_per_step": int(8 * A.n),
                  "includes": "sg_analyze (CSR ingest from host) + sg_solve "
                              "(b host->device, x device->host)"}

    # ---- CPU baseline (oracle, rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, its = cpu_oracle_sample(c)
        out["cpu_baseline"] = {
            "value": dt * info.iters / max(its, 1), "unit": "s",
            "cores": oracle_threads(), "kind": "oracle",
            "sample": sample_text(dt, its, info.iters)}
    if rank == 0:
        print(json.dumps(out))
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------ reference
def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c, cfg = workload(args.grid)
    from oracle import sgmres_oracle as O
    for _ in range(args.warmup):   # short warm-up: imports, page-in, BLAS
        O.adaptive_sgmres(c["A"], c["b"], m=20, s=4, tol=1e-10, max_iters=8)
    times, its = [], 0
    for _ in range(args.steps):
        dt, its = cpu_oracle_sample(c)
        times.append(dt)
    dt = sum(times) / len(times)
    val = dt * FULL_SOLVE_COLUMNS / max(its, 1)
    out = {"impl": "reference", "metric": METRIC, "value": val, "value_is": VALUE_IS,
           "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * val,
           "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": cfg,
           "cpu_baseline": {"value": val, "unit": "s",
                            "cores": oracle_threads(), "kind": "oracle",
                            "sample": sample_text(dt, its, FULL_SOLVE_COLUMNS)},
           "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ------------------------------------------------------------ profiler cases
def run_case(args):
    """One small workload per kernel family, for ncu (see profiles/)."""
    import torch
    import paper_2303_08953_gb300 as sg
    import workloads as W
    solver = sg.Solver(0)
    dev = torch.device("cuda:0")
    name = args.case
    if name.startswith("solve"):
        c = W.config_c2(args.grid)
        solver.analyze_csr(c["A"])
        b = torch.as_tensor(c["b"], device=dev)
        prec = "fp64" if name == "solve-fp64" else "fp32_ir"
        x, info = solver.solve(b, precision=prec, **SOLVE_KW)
        print(name, info.converged, info.iters, info.final_relres)
    elif name == "spmv":
        c = W.config_c2(args.grid)
        A = c["A"]
        solver.analyze_csr(A)
        x = torch.rand(A.n, dtype=torch.float64, device=dev)
        y = torch.empty_like(x)
        for _ in range(4):
            solver.spmv_newton(x, 0.3, 1.1, out=y)
    else:
        # block kernels on n = 2^20 rows, i = 107, s = 106 (the solve's
        # second-block shape)
        n, i, s = 1 << 20, 107, 106
        fp = torch.float64 if name.endswith("64") else torch.float32
        solver.analyze_csr(W.config_c1(8)["A"])
        solver.n = n
        Q = torch.randn(i, n, dtype=torch.float64, device=dev)
        X = torch.randn(s, n, dtype=torch.float64, device=dev)
        if name == "dot64":
            for _ in range(3):
                solver.block_dot(Q, X)
        elif name == "upd64":
            Wt = torch.randn(s, i, dtype=torch.float64, device=dev)
            for _ in range(3):
                solver.block_update(Q, Wt, X)
        else:
            Q32, X32 = Q.to(fp), X.to(fp)
            Wt = torch.randn(s, i, dtype=torch.float64, device=dev)
            for _ in range(3):
                if name == "dot32":
                    solver.block_dot32(Q32, X32)
                elif name == "upd32":
                    solver.block_update32(Q32, Wt, X32)
                else:
                    solver.block_dot32(X32, X32, sym=True)
    torch.cuda.synchronize()
    solver.close()


if __name__ == "__main__":
    a = parse()
    if a.case:
        run_case(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
