"""Writes the oracle's decisions and solution samples for the full-size
workloads to tests/golden/fullsize_<config>.json.

It calls only the CPU oracle (oracle/) and the seeded input generators
(workloads/); nothing here comes from the GPU library.  The GPU test
tests/test_gpu_fullsize.py::test_full_size_decisions_match_oracle compares
the library's FP64 solve, given these Ritz values, with these values:
identical step-size decisions and iteration counts (Alg. 4, Sec. 3.5),
per-cycle true residuals, and the solution on sampled entries, its 2-norm
and seeded linear functionals; and the library's own pre-pass with the
converged Ritz values listed here (those with a small Ritz-pair residual).

    python tests/golden/make_fullsize_golden.py c5      # 4.19M-row random band
    python tests/golden/make_fullsize_golden.py c2      # 128^3 convection-diffusion
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as W                      # noqa: E402
from oracle import sgmres_oracle as O      # noqa: E402

# solver options of each workload (the configurations' m, s range, tol)
OPTS = {
    "c2": dict(m=240, s=0, s_min=20, s_max=120, tol=1e-10),
    "c5": dict(m=120, s=0, s_min=1, s_max=120, tol=1e-10),
}
N_SAMPLES = 1024          # sampled solution entries
N_FUNCTIONALS = 8         # seeded Gaussian functionals u_k . x
SAMPLE_SEED = 20230315


def sample_indices(n):
    """Indices of the sampled entries (stored in the golden file)."""
    rng = np.random.default_rng(SAMPLE_SEED)
    return np.sort(rng.choice(n, size=N_SAMPLES, replace=False))


def functional_vector(n, k):
    """u_k ~ N(0, 1)^n from the PCG64 stream seeded (SAMPLE_SEED, k)."""
    return np.random.default_rng([SAMPLE_SEED, k]).standard_normal(n)


def functionals(x):
    return [float(functional_vector(x.size, k) @ x) for k in range(N_FUNCTIONALS)]


def main(name):
    c = W.CONFIGS[name]()
    opts = OPTS[name]
    t0 = time.perf_counter()
    r = O.adaptive_sgmres(c["A"], c["b"], **opts)
    dt = time.perf_counter() - t0
    idx = sample_indices(c["A"].n)
    theta, rres = O.ritz_residuals(r.prepass_H, r.prepass_steps)
    out = {
        "_about": (f"Oracle (oracle/sgmres_oracle.py, FP64 adaptive s-step GMRES, "
                   f"Alg. 4) on workload {c['name']} with {opts}; written by "
                   f"tests/golden/make_fullsize_golden.py in {dt:.0f} s"),
        "config": name, "opts": opts, "n": int(c["A"].n), "nnz": int(c["A"].nnz),
        "converged": bool(r.converged), "iters": int(r.iters),
        "restarts": int(r.restarts), "s0": int(r.s0),
        "s_hist": [int(v) for v in r.s_hist],
        "s_eff_hist": [int(v) for v in r.s_eff_hist],
        "p1_hist": [int(v) for v in r.p1_hist],
        "cycle_iters": [int(v) for v in r.cycle_iters],
        "cycle_relres": [float(v) for v in r.cycle_relres],
        "relres_hist": [float(v) for v in r.relres_hist],
        "ritz_re": [float(v) for v in np.real(r.ritz)],
        "ritz_im": [float(v) for v in np.imag(r.ritz)],
        # every Ritz value of the pre-pass with its Ritz-pair residual norm
        # (small: converged, reproduced by any rounding of the pre-pass)
        "prepass_ritz_re": [float(v) for v in np.real(theta)],
        "prepass_ritz_im": [float(v) for v in np.imag(theta)],
        "prepass_ritz_residual": [float(v) for v in rres],
        "x_norm": float(np.linalg.norm(r.x)),
        "x_err_vs_xstar": float(np.linalg.norm(r.x - c["xstar"]) / np.linalg.norm(c["xstar"])),
        "sample_seed": SAMPLE_SEED,
        "x_idx": [int(v) for v in idx],
        "x_sample": [float(v) for v in r.x[idx]],
        "x_functionals": functionals(r.x),
        "oracle_seconds": dt,
    }
    path = os.path.join(HERE, f"fullsize_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print(path, f"{dt:.1f} s", r.iters, r.s0, r.s_hist[:8], r.cycle_relres)


if __name__ == "__main__":
    for nm in sys.argv[1:] or ["c5"]:
        main(nm)
