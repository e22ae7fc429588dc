"""Benchmark: time to relative residual 1e-10 of the adaptive s-step GMRES.

Headline workload: the unstructured random-band system, N = 4,194,304 rows
with 24 off-diagonal entries per row at distinct offsets within +-4096 and
a 1.1x dominant diagonal (nnz = 104,857,600), m = 120, scaled Newton basis,
s estimated from a 120-step Ritz pre-pass, tol 1e-10.

One step = one complete solve from x0 = 0 (Ritz pre-pass, estimator, every
block and restart) with A and b resident in HBM.  The FP64 solve gives
`value`; the FP32-basis + FP64-refinement solve and the forward + adjoint
pair (loss 0.5 ||x - x_t||^2) are reported beside it on the same system,
and the 128^3 convection-diffusion system (m = 240, s in [20, 120]) as a
secondary line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config c5|c2|c3] [--with-c3]

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

# workloads: generator, solver options, bench label
WORKLOADS = {
    "c5": dict(label="randband_4194304_k24_band4096",
               opts=dict(m=120, s=0, s_min=1, s_max=120, tol=1e-10),
               s_desc="auto[1,120]", seed=4),
    "c2": dict(label="convdiff3d_128^3",
               opts=dict(m=240, s=0, s_min=20, s_max=120, tol=1e-10),
               s_desc="auto[20,120]", seed=1),
    "c1": dict(label="stencil2d_64^2",
               opts=dict(m=60, s=10, tol=1e-10),
               s_desc="10", seed=0),
    "c3": dict(label="vardiff3d_192^3",
               opts=dict(m=200, s=0, s_min=1, s_max=60, tol=1e-10, max_iters=20000),
               s_desc="auto[1,60]", seed=2),
}
FP64_ALU_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12   # 152 SMs x 2.07 GHz x 4 flop/clk
# The FP32 Gram on the tensor cores multiplies six 8-bit digit slices of
# each value pairwise, levels 0..7: 30 digit-pair products per FP32 product,
# so 30 n s (s + 1) FP16 tensor flops for the n s (s + 1) flops of the upper
# triangle
GRAM32_DIGIT_PAIRS = 30
PREPASS_STEPS = 120


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default="c5", choices=list(WORKLOADS))
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--no-secondary", action="store_true")
    p.add_argument("--with-c3", action="store_true",
                   help="also time the 192^3 mixed-precision system (minutes)")
    p.add_argument("--case", default=None,
                   choices=["solve-fp64", "solve-fp32ir", "prepass64", "prepass32",
                            "spmv", "dot64", "gram64", "upd64", "dot32", "gram32", "upd32"],
                   help="run one small workload for a profiler and exit")
    p.add_argument("--rows", type=int, default=None,
                   help="rows of the --case workload (random band recipe)")
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


def make_workload(name, rows=None):
    """The seeded system of workload `name` (rows: a smaller instance of the
    random-band recipe) and the bench line's config record."""
    import workloads as W
    spec = WORKLOADS[name]
    if name == "c5":
        c = W.config_c5(rows) if rows else W.config_c5()
    elif name == "c2":
        c = W.config_c2(128)
    elif name == "c1":
        c = W.config_c1(64)
    else:
        c = W.config_c3(192)
    A = c["A"]
    cfg = {"workload": spec["label"] if not rows else f"randband_{rows}_k24_band4096",
           "n": int(A.n), "nnz": int(A.nnz), "m": spec["opts"]["m"],
           "s": spec["s_desc"], "basis": "scaled_newton", "tol": spec["opts"]["tol"],
           "x0": "zero", "precision_of_value": "fp64",
           "l2": f"inputs larger than L2 (A {(12 * A.nnz + 4 * A.n) / 1e6:.0f} MB)"}
    return c, cfg, dict(spec["opts"])


def spmv_bytes(A):
    """Bytes of one FP64 SpMV in the stored format: values + column indices
    (2-byte offsets from a per-32-row-slice base when every slice's columns
    span fewer than 65535, as the library stores them, else 4 bytes), row or
    slice pointers, x read once, y written once."""
    rp = np.asarray(A.rowptr, dtype=np.int64)
    ci = np.asarray(A.colind, dtype=np.int64)
    nsl = (A.n + 31) // 32
    first = rp[np.minimum(np.arange(nsl) * 32, A.n)]
    last = rp[np.minimum(np.arange(nsl) * 32 + 32, A.n)]
    lo = np.full(nsl, np.iinfo(np.int64).max)
    hi = np.full(nsl, -1)
    nz = last > first
    sl = np.repeat(np.arange(nsl), last - first)
    np.minimum.at(lo, sl, ci)
    np.maximum.at(hi, sl, ci)
    narrow = bool(np.all((hi[nz] - lo[nz]) < 0xFFFF))
    idx = 2 if narrow else 4
    return (8 + idx) * A.nnz + (8 if narrow else 4) * (nsl + 1) + 8 * A.n + 8 * A.n


def mgs_flops(A, k):
    """FP64 flops of the MGS launches of a k-step pre-pass (Sec. 3.4): per
    step j, j+1 projections (dot and update, 4 N each), the norm of w (2 N)
    and its scaling (N)."""
    return sum(4 * A.n * (j + 1) + 3 * A.n for j in range(k))


def mgs_bytes(A, k):
    """Algorithmic HBM bytes of the same MGS launches: w and the j+1 basis
    vectors read once, the new vector written once."""
    return sum(8 * A.n * (j + 3) for j in range(k))


# DRAM bytes of one MGS launch per row and per vector it streams (j + 2
# vectors read at step j), from the ncu capture of step j = 58 at
# 2,097,152 rows: 1,007,194,000 + 3,276,544 bytes over 60 vectors
# (profiles/arnoldi_mgs_resident_fp64_randband_2M_j58.md).
MGS_DRAM_BYTES_PER_ROW_VECTOR = (1_006_732_000 + 3_225_344) / 2_097_152 / 60


# ------------------------------------------------------------ CPU oracle
# The oracle's complete solve of the headline workload takes minutes on the
# host (it is plain numpy, one projection at a time), so the CPU baseline is
# a complete oracle solve of the same recipe with fewer rows, scaled by rows
# to the full system.  Every oracle operation of the solve (CSR product,
# dot, update, Gram, triangular solve) costs O(rows) at fixed decisions.
SAMPLE_ROWS = 262_144


def cpu_oracle_sample(name):
    """(seconds, effective threads, oracle result, rows) of one complete
    oracle solve of the workload recipe at SAMPLE_ROWS rows (c5) or of the
    workload itself (c2/c3 are not sampled this way)."""
    from oracle import sgmres_oracle as O
    c, _, opts = make_workload(name, rows=SAMPLE_ROWS if name == "c5" else None)
    t0, c0 = time.perf_counter(), os.times()
    r = O.adaptive_sgmres(c["A"], c["b"], **opts)
    dt, c1 = time.perf_counter() - t0, os.times()
    cpu = (c1.user - c0.user) + (c1.system - c0.system)
    return dt, cpu / dt if dt > 0 else 1.0, r, int(c["A"].n)


def sample_text(dt, rows, full_rows, r):
    return (f"complete oracle FP64 solve (oracle/sgmres_oracle.py adaptive_sgmres, "
            f"Ritz pre-pass + estimator + every block) of the same random-band recipe "
            f"at {rows} rows: {dt:.1f} s, {r.iters} Krylov columns, s0 {r.s0}, "
            f"blocks {list(map(int, r.s_hist))}, relres {r.final_relres:.2e}; "
            f"scaled by rows x{full_rows / rows:g} to the {full_rows}-row system")


# ------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import paper_2303_08953_gb300 as sg
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c, cfg, opts = make_workload(args.config)
    A = c["A"]
    solver = sg.Solver(local)
    solver.analyze_csr(A)
    b = torch.as_tensor(c["b"], dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2
    stream = torch.cuda.current_stream()
    launches = [0]

    def timed(fn, steps, warm):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        times, res = [], None
        l0 = sg.kernel_launches()
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        launches[0] = (sg.kernel_launches() - l0) // max(1, steps)
        barrier(world)
        return times, res

    def solve(prec="fp64", sv=solver, rhs=b, o=opts):
        return sv.solve(rhs, precision=prec, **o)

    # ---- headline: FP64 solve
    clocks = ClockSampler(local)
    times, (x, info) = timed(solve, args.steps, args.warmup)
    n_launch = launches[0]
    clk = clocks.stop()
    ms_step = max_over_ranks(sum(times) / len(times), world)
    xs = c["xstar"]
    xh = x.cpu().numpy()
    err = float(np.linalg.norm(xh - xs) / np.linalg.norm(xs))
    out = {
        "metric": METRIC, "value": ms_step / 1e3, "unit": "s", "value_is": VALUE_IS,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": f"synthetic (seeded generator, seed {WORKLOADS[args.config]['seed']}; "
                f"x* ~ U(-1,1), b = A x*)",
        "config": cfg,
        "solve": {"converged": info.converged, "iters": info.iters,
                  "restarts": info.restarts, "s0": info.s0,
                  "s_hist_first": [int(v) for v in info.s_hist[:8]],
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
        t32, (x32, i32) = timed(lambda: solve("fp32_ir"), args.steps, 1)
        x32h = x32.cpu().numpy()
        out["fp32_ir"] = {
            "time_s": max_over_ranks(sum(t32) / len(t32), world) / 1e3,
            "iters": i32.iters, "refinements": i32.refinements,
            "fp64_iters": i32.fp64_iters, "s0": i32.s0,
            "final_relres": i32.final_relres,
            "x_err_vs_xstar": float(np.linalg.norm(x32h - xs) / np.linalg.norm(xs)),
            "x_err_vs_fp64": float(np.linalg.norm(x32h - xh) / np.linalg.norm(xh)),
            "phase_ms": {k: round(v, 2) for k, v in i32.times_ms.items()}}
        # loss L = 0.5 ||x - x_t||^2 with the workload's target x_t ~ U(-1,1)
        # (drawn after x* from its seeded stream)
        xt = torch.as_tensor(c["xtarget"], device=dev)
        fa = []
        for prec in ("fp32_ir", "fp64"):
            def pair(prec=prec):
                # the adjoint reuses the forward solve's Ritz values (A^T
                # has A's eigenvalues) instead of its own pre-pass
                xf, inf1 = solver.solve(b, precision=prec, **opts)
                lam, inf2 = solver.solve_adjoint(xf - xt, precision=prec, ritz=inf1.ritz,
                                                 **opts)
                solver.grad_values(lam, xf)
                return inf1, inf2
            ts, (inf1, inf2) = timed(pair, max(1, args.steps // 2), 1)
            fa.append({"precision": prec,
                       "time_s": max_over_ranks(sum(ts) / len(ts), world) / 1e3,
                       "fwd_iters": inf1.iters, "adj_iters": inf2.iters,
                       "fwd_relres": inf1.final_relres,
                       "adj_relres": inf2.final_relres,
                       "adj_s0": inf2.s0, "adj_refinements": inf2.refinements,
                       "adj_fp64_iters": inf2.fp64_iters,
                       "adj_phase_ms": {k: round(v, 2) for k, v in inf2.times_ms.items()}})
        out["fwd_adjoint"] = fa

    # ---- roofline of the dominant kernel: the resident FP64 MGS launch of
    # the Ritz pre-pass (Sec. 3.4; one launch per step, after that step's
    # SpMV).  Its mean launch time is the pre-pass time, timed with CUDA
    # events over the 240 launches of one pre-pass, minus its 120 SpMVs at
    # the SpMV's own event-timed rate (below)
    n = A.n
    xv = torch.rand(n, dtype=torch.float64, device=dev)
    yv = torch.empty_like(xv)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(5):
        solver.spmv_newton(xv, 0.3, 1.1, out=yv)
    torch.cuda.synchronize()
    reps = 30
    e0.record(stream)
    for _ in range(reps):
        solver.spmv_newton(xv, 0.3, 1.1, out=yv)
    e1.record(stream)
    torch.cuda.synchronize()
    t_sp = e0.elapsed_time(e1) / reps / 1e3
    q = b / torch.linalg.vector_norm(b)
    solver.arnoldi(q, PREPASS_STEPS)
    torch.cuda.synchronize()
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        solver.arnoldi(q, PREPASS_STEPS)
    e1.record(stream)
    torch.cuda.synchronize()
    t_pre = e0.elapsed_time(e1) / reps / 1e3
    t_launch = (t_pre - PREPASS_STEPS * t_sp) / PREPASS_STEPS
    fl = mgs_flops(A, PREPASS_STEPS) / PREPASS_STEPS
    by = mgs_bytes(A, PREPASS_STEPS) / PREPASS_STEPS
    vec = sum(j + 2 for j in range(PREPASS_STEPS)) / PREPASS_STEPS
    pk = measured_peaks()
    hbm = pk["hbm_gbs"] if pk else 6800.0
    hbm_src = "MEASURED_PEAKS.json hbm_gbs" if pk else "fallback"
    ach = fl / t_launch / 1e12
    out["roofline"] = {
        "kernel": f"arnoldi_mgs_resident_kernel FP64 (MGS phases of one Ritz pre-pass step, "
                  f"w in shared memory; mean of the {PREPASS_STEPS} launches of one pre-pass)",
        "bound": "alu", "achieved": round(ach, 4),
        "peak": round(FP64_ALU_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
        "frac": round(ach / FP64_ALU_PEAK_TFLOPS, 4),
        "traffic": int(round(MGS_DRAM_BYTES_PER_ROW_VECTOR * n * vec)),
        "traffic_source": "ncu dram__bytes_read+write of the launch at step j = 58, 2,097,152 "
                          "rows, per row and streamed vector, scaled to this n and the mean "
                          "step (profiles/arnoldi_mgs_resident_fp64_randband_2M_j58.md)",
        "launch_ms": round(t_launch * 1e3, 4),
        "prepass_ms": round(t_pre * 1e3, 2),
        "algorithmic_flops_per_launch": int(fl),
        "algorithmic_bytes_per_launch": int(by),
        "hbm_frac": round(by / t_launch / 1e9 / hbm, 4),
        "peak_source": "derived: 152 SMs x 2.07 GHz x 4 FP64 flop/clk/SM "
                       "(nominal 1.25 TFLOP/s FP64)"}

    # secondary: the MPK's SpMV against HBM (timed above)
    gbs = spmv_bytes(A) / t_sp / 1e9
    out["roofline_spmv"] = {
        "kernel": "spmv_newton FP64 (one MPK step)", "bound": "hbm",
        "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
        "frac": round(gbs / hbm, 4), "traffic": None, "peak_source": hbm_src}
    del xv, yv

    # the block kernels at the 128^3 system's second-block shape
    # (i = 107, s = 106) on 2^21 rows
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
    nb, i_blk, s_blk = 1 << 21, 107, 106
    solver.n = nb
    Q64 = torch.randn(i_blk, nb, dtype=torch.float64, device=dev)
    X64 = torch.randn(s_blk, nb, dtype=torch.float64, device=dev)
    W64u = torch.randn(s_blk, i_blk, dtype=torch.float64, device=dev)
    t_dot = event_ms(lambda: solver.block_dot(Q64, X64)) / 1e3
    t_g64 = event_ms(lambda: solver.block_dot(X64, X64, sym=True)) / 1e3
    t_u64 = event_ms(lambda: solver.block_update(Q64, W64u, X64)) / 1e3
    del Q64, X64, W64u
    Q32 = torch.randn(i_blk, nb, dtype=torch.float32, device=dev)
    X32 = torch.randn(s_blk, nb, dtype=torch.float32, device=dev)
    W64 = torch.randn(s_blk, i_blk, dtype=torch.float64, device=dev)
    t_tcd = event_ms(lambda: solver.block_dot32(Q32, X32)) / 1e3
    t_tcu = event_ms(lambda: solver.block_update32(Q32, W64, X32)) / 1e3
    t_gram = event_ms(lambda: solver.block_dot32(X32, X32, sym=True)) / 1e3
    del Q32, X32, W64
    solver.n = A.n
    # FP64 products on the tensor cores from exact 8-bit digit slices: 36
    # digit-pair products (levels 0..7 of 8 x 8 digits) per FP64 product, so
    # 72 n i s FP16 tensor flops for 2 n i s FP64 flops
    f_dot = 2.0 * nb * i_blk * s_blk
    f_g64 = 2.0 * nb * s_blk * s_blk
    tpk = pk["bf16_tflops"] if pk else 1900.0
    tpk_src = "MEASURED_PEAKS.json bf16_tflops (FP16 runs at the BF16 rate)" if pk else "fallback"

    def tc_entry(name, f64, t):
        ach = 36.0 * f64 / t / 1e12
        return {"kernel": name, "bound": "tensor", "achieved": round(ach, 1), "peak": tpk,
                "unit": "TFLOP/s", "frac": round(ach / tpk, 4), "peak_source": tpk_src,
                "fp64_equivalent_tflops": round(f64 / t / 1e12, 3),
                "fp64_pipe_peak_tflops": round(FP64_ALU_PEAK_TFLOPS, 4),
                "ms": round(t * 1e3, 3)}
    out["roofline_block_fp64"] = [
        tc_entry(f"oz_dot: block_dot FP64 (W = Q^T X, i={i_blk}, s={s_blk}, n=2^21)", f_dot, t_dot),
        tc_entry(f"oz_dot: Gram FP64 (X^T X, s={s_blk}, n=2^21)", f_g64, t_g64),
        tc_entry(f"oz_update: block_update FP64 (X -= Q W, i={i_blk}, s={s_blk}, n=2^21)",
                 f_dot, t_u64)]
    b_tcd = 4.0 * nb * (i_blk + s_blk)
    b_tcu = 4.0 * nb * (i_blk + 2 * s_blk)
    f_gram = float(nb) * s_blk * (s_blk + 1)
    out["roofline_fp32"] = [
        {"kernel": f"tc_dot FP32 basis (W = Q^T X on tcgen05, 3xTF32, i={i_blk}, s={s_blk})",
         "bound": "hbm", "achieved": round(b_tcd / t_tcd / 1e9, 1), "peak": hbm,
         "unit": "GB/s", "frac": round(b_tcd / t_tcd / 1e9 / hbm, 4), "peak_source": hbm_src},
        {"kernel": f"tc_update FP32 basis (X -= Q W on tcgen05, 3xTF32, i={i_blk}, s={s_blk})",
         "bound": "hbm", "achieved": round(b_tcu / t_tcu / 1e9, 1), "peak": hbm,
         "unit": "GB/s", "frac": round(b_tcu / t_tcu / 1e9 / hbm, 4), "peak_source": hbm_src},
        {"kernel": f"oz_gram32: Gram FP32 basis (X^T X on tcgen05 from exact 8-bit digit "
                   f"slices, s={s_blk}, n=2^21)",
         "bound": "tensor", "achieved": round(GRAM32_DIGIT_PAIRS * f_gram / t_gram / 1e12, 1),
         "peak": tpk, "unit": "TFLOP/s",
         "frac": round(GRAM32_DIGIT_PAIRS * f_gram / t_gram / 1e12 / tpk, 4),
         "peak_source": tpk_src,
         "fp32_equivalent_tflops": round(f_gram / t_gram / 1e12, 3),
         "hbm_frac": round(4.0 * nb * s_blk / t_gram / 1e9 / hbm, 4),
         "ms": round(t_gram * 1e3, 3)}]

    # ---- end to end through the public API from host buffers
    rp, ci, va = A.rowptr, A.colind, A.val
    bh = np.asarray(c["b"])
    e2e_t = []
    for k in range(3):
        s2 = sg.Solver(local)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2.analyze(rp, ci, va)
        s2.solve(bh, **opts)
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
    solver.close()
    del b
    torch.cuda.empty_cache()

    # ---- secondary systems (same FP64 / FP32-IR solves)
    sec = []
    names = [] if args.no_secondary else [nm for nm in ("c2", "c1") if nm != args.config]
    if args.with_c3 and args.config != "c3":
        names.append("c3")
    for nm in names:
        c2, cfg2, o2 = make_workload(nm)
        s2 = sg.Solver(local)
        s2.analyze_csr(c2["A"])
        b2 = torch.as_tensor(c2["b"], dtype=torch.float64, device=dev)
        reps = {"c3": 1, "c1": 10}.get(nm, 3)
        rec = {"config": cfg2}
        for prec in ("fp64", "fp32_ir"):
            ts, (xx, ii) = timed(lambda: solve(prec, s2, b2, o2), reps, 1 if nm != "c3" else 0)
            rec[prec] = {"time_s": max_over_ranks(sum(ts) / len(ts), world) / 1e3,
                         "iters": ii.iters, "s0": ii.s0, "refinements": ii.refinements,
                         "fp64_iters": ii.fp64_iters, "final_relres": ii.final_relres,
                         "converged": ii.converged,
                         "phase_ms": {k: round(v, 2) for k, v in ii.times_ms.items()}}
        sec.append(rec)
        s2.close()
        del b2
    if sec:
        out["secondary"] = sec

    # ---- CPU baseline (oracle, rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.config == "c5":
        dt, thr, r, rows = cpu_oracle_sample(args.config)
        out["cpu_baseline"] = {
            "value": dt * A.n / rows, "unit": "s",
            "cores": int(round(thr)), "cores_available": len(os.sched_getaffinity(0)),
            "kind": "oracle", "sample": sample_text(dt, rows, A.n, r)}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------ reference
def run_reference(args):
    """The CPU oracle on the bench's workload, rank 0 only: each step is one
    complete oracle solve of the workload recipe at SAMPLE_ROWS rows, and
    `value` scales the mean step time by rows to the full system."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import sgmres_oracle as O
    import workloads as W
    _, cfg, _ = make_workload(args.config)
    if args.config != "c5":
        print(json.dumps({"impl": "reference",
                          "unavailable": "the reference arm samples the random-band "
                                         "recipe (--config c5) only"}))
        return
    c1 = W.config_c1(32)
    for _ in range(args.warmup):   # short warm-up: imports, page-in, BLAS
        O.adaptive_sgmres(c1["A"], c1["b"], m=20, s=4, tol=1e-10, max_iters=8)
    times, thr, r, rows = [], [], None, SAMPLE_ROWS
    for _ in range(args.steps):
        dt, th, r, rows = cpu_oracle_sample(args.config)
        times.append(dt)
        thr.append(th)
    dt = sum(times) / len(times)
    scale = cfg["n"] / rows
    val = dt * scale
    out = {"impl": "reference", "metric": METRIC, "value": val, "value_is": VALUE_IS,
           "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * dt,
           "ms_per_step_is": "measured wall time of one step (the sampled solve)",
           "value_scale_by_rows": scale,
           "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": cfg,
           "cpu_baseline": {"value": val, "unit": "s",
                            "cores": int(round(statistics.median(thr))),
                            "cores_available": len(os.sched_getaffinity(0)),
                            "kind": "oracle",
                            "sample": sample_text(dt, rows, cfg["n"], r)},
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
    if name in ("solve-fp64", "solve-fp32ir", "prepass64", "prepass32", "spmv"):
        if args.config == "c5":
            c, _, opts = make_workload("c5", rows=args.rows)
        else:
            c, _, opts = make_workload(args.config)
        A = c["A"]
        solver.analyze_csr(A)
        b = torch.as_tensor(c["b"], device=dev)
        if name.startswith("solve"):
            prec = "fp64" if name == "solve-fp64" else "fp32_ir"
            x, info = solver.solve(b, precision=prec, **opts)
            print(name, info.converged, info.iters, info.final_relres)
        elif name.startswith("prepass"):
            q = b / torch.linalg.vector_norm(b)
            prec = "fp64" if name == "prepass64" else "fp32_ir"
            H, steps = solver.arnoldi(q, 64, precision=prec)
            print(name, steps, float(np.abs(H).max()))
        else:
            x = torch.rand(A.n, dtype=torch.float64, device=dev)
            y = torch.empty_like(x)
            for _ in range(4):
                solver.spmv_newton(x, 0.3, 1.1, out=y)
    else:
        # block kernels on n = 2^20 rows, i = 107, s = 106 (the 128^3
        # solve's second-block shape)
        n, i, s = 1 << 20, 107, 106
        fp = torch.float64 if name.endswith("64") else torch.float32
        solver.analyze_csr(W.config_c1(8)["A"])
        solver.n = n
        Q = torch.randn(i, n, dtype=torch.float64, device=dev)
        X = torch.randn(s, n, dtype=torch.float64, device=dev)
        if name == "dot64":
            for _ in range(3):
                solver.block_dot(Q, X)
        elif name == "gram64":
            for _ in range(3):
                solver.block_dot(X, X, sym=True)
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
