"""Writes the float64 oracle's trajectory on the two large synthetic workloads.

The GPU tests and the benchmark compare the library's relative errors with
these files; no value in them comes from the GPU.  Only the oracle (oracle/)
computes, on inputs from the seeded generator (synth/).  Each file holds the
oracle's relative error ||A - W H||_F / ||A||_F (the "Error" of the Section 4
tables) after every 10th sweep, with the host, the threads and the wall times
of the QB and of the sweeps (error evaluations excluded).

  python tests/golden/make_oracle_reference.py scale
      -> tests/golden/oracle_rhals_fp32_50000x20000_k50.json: randomized HALS
         (Algorithm 1) and deterministic HALS (Section 3.1), 200 sweeps each
  python tests/golden/make_oracle_reference.py precision
      -> tests/golden/oracle_rhals_bf16sketch_100000x50000_k100.json:
         randomized HALS, 300 sweeps (A is 20 GB as float32, 40 GB as float64)
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import philox  # noqa: E402
from oracle import rhals as R  # noqa: E402

EVERY = 10
ROWS = 8192  # row block of the error evaluation (bounds the temporary of A - W H)


def threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        return os.cpu_count() or 1


def rel_err_blocked(A64, W, H, a2):
    """||A - W H||_F / ||A||_F as the sum of the NMF objective over row blocks."""
    e2 = 0.0
    for r in range(0, A64.shape[0], ROWS):
        e2 += R.objective(A64[r:r + ROWS], W[r:r + ROWS], H)
    return float(np.sqrt(e2 / a2))


def run_rhals(A64, w, a2):
    t0 = time.perf_counter()
    Q, B = R.rqb(A64, philox.omega(w.n, w.l, w.seed), w.q)
    t_qb = time.perf_counter() - t0
    W, H = philox.init_factors(w.m, w.n, w.k, w.seed)
    Wt = None
    hist, t_sw = [], 0.0
    for _ in range(w.iters // EVERY):
        t0 = time.perf_counter()
        W, H, Wt, _ = R.rhals_sweeps(Q, B, W, H, EVERY, Wt=Wt)
        t_sw += time.perf_counter() - t0
        hist.append(rel_err_blocked(A64, W, H, a2))
        print(f"  rhals sweep {len(hist) * EVERY}: {hist[-1]:.8g}  ({t_sw:.1f}s)", flush=True)
    return {"rel_err_every_10": hist, "qb_s": t_qb, "sweeps_s": t_sw, "solve_s": t_qb + t_sw}


def run_hals(A64, w, a2):
    W, H = philox.init_factors(w.m, w.n, w.k, w.seed)
    hist, t_sw = [], 0.0
    for _ in range(w.iters // EVERY):
        t0 = time.perf_counter()
        W, H, _ = R.hals_sweeps(A64, W, H, EVERY)
        t_sw += time.perf_counter() - t0
        hist.append(rel_err_blocked(A64, W, H, a2))
        print(f"  hals sweep {len(hist) * EVERY}: {hist[-1]:.8g}  ({t_sw:.1f}s)", flush=True)
    return {"rel_err_every_10": hist, "sweeps_s": t_sw, "solve_s": t_sw}


def main(which: str, out_dir: str = HERE):
    w = {"scale": synth.SCALE, "precision": synth.PRECISION}[which]
    t0 = time.perf_counter()
    A = synth.lowrank(w)
    t_gen = time.perf_counter() - t0
    A64 = A.astype(np.float64)
    del A
    a2 = float(sum(np.sum(A64[r:r + ROWS] ** 2) for r in range(0, w.m, ROWS)))
    rec = {"workload": w.name, "m": w.m, "n": w.n, "k": w.k, "p": w.p, "q": w.q, "iters": w.iters,
           "sigma": w.sigma, "seed": w.seed, "check_every": EVERY,
           "host": {"machine": platform.machine(), "cpus": os.cpu_count(), "blas_threads": threads()},
           "generate_s": t_gen, "writer": "tests/golden/make_oracle_reference.py (float64 oracle only)"}
    print(f"{w.name}: A generated in {t_gen:.1f}s", flush=True)
    rec["rhals"] = run_rhals(A64, w, a2)
    if which == "scale":
        rec["hals"] = run_hals(A64, w, a2)
    path = os.path.join(out_dir, f"oracle_{w.name}.json")
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    print(f"wrote {path}")


if __name__ == "__main__":
    main(sys.argv[1], *(sys.argv[2:3]))
