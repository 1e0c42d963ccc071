"""Benchmark: randomized HALS time to a target relative error on one GB300.

Workload (default): A = W0 H0 + 0.02 |z|, 100000 x 50000 float32 (20 GB), W0 ~
Exp(1) (rank 100), 30% of H0 zero; k = 100, p = 20, q = 2, up to 300 sweeps
(the synthetic stand-in for the Section 4.4 experiments at scale).

Metric: wall time of one rHALS solve (QB + sweeps) in the measured form
(default: BF16 sketch) until the relative error ||A - WH||/||A|| reaches the
target 1.001 x the final error of the FP32 form after all sweeps.  The runs
are deterministic (fixed-order reductions), so the number of sweeps t* at which
the target is first reached (checked every 10 sweeps in an untimed calibration
run) is fixed; every timed step is then exactly rnmf(iters = t*).

Other workloads (one JSON line each, same keys):
  --workload adjoint: forward + backward of T = 50 unrolled compressed sweeps on
      4096 x 2048 (k = 16, l = 26), loss <G, W_T H_T>; metric: seconds per step.
  --workload batch: 512 ragged problems (m in [256, 8192], n in [128, 4096],
      k in [4, 32], p = 10, q = 2, 100 sweeps) in one captured graph; metric:
      problems per second.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]
Under torchrun (N > 1) every rank solves its own replica (the path does not shard).
"""
from __future__ import annotations

import argparse
import hashlib
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

import synth  # noqa: E402

WORKLOADS = {"precision": synth.PRECISION, "scale": synth.SCALE, "small": synth.SMALL, "adjoint": synth.ADJOINT,
             "batch": None, "streamed": synth.PRECISION}
FORMS = {"fp32": 0, "bf16": 1, "split3": 2}
METRIC = "rHALS time to target rel. error (s), BF16-sketch vs FP32 form; % of roofline"
METRIC_ADJOINT = "adjoint of T=50 unrolled compressed sweeps: forward + backward time (s)"
METRIC_BATCH = "batched ragged rHALS throughput (problems/s)"
METRIC_STREAMED = "rHALS with A in host memory, column-blocked QB (Algorithm 2): solve time (s)"
METRIC_SCALE = "rHALS vs deterministic HALS at scale: FP32 rHALS solve time (s), 200 sweeps"
CHECK_EVERY = 10


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def first_reach(hist, target):
    for i, e in enumerate(hist):
        if e <= target:
            return (i + 1) * CHECK_EVERY
    return None


def kernel_source_hash():
    """Hash of the CUDA sources with comments and blank space taken out, so
    that counters stay keyed to the code they were taken on across edits of
    comments only."""
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1711_02037_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            src = open(os.path.join(d, f), encoding="utf-8").read()
            src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
            src = re.sub(r"//[^\n]*", " ", src)
            h.update(f.encode() + b"\0" + " ".join(src.split()).encode())
    return h.hexdigest()[:16]


def roofline(prof: dict, peaks: dict, peak_kind: str, workload: str):
    """Dominant kernel class of the timed region against its roofline."""
    if not prof:
        return None
    name, d = max(prof.items(), key=lambda kv: kv[1]["ms"])
    avg_s = d["ms"] / d["launches"] / 1e3
    bytes_per = d["bytes"] / d["launches"]
    flops_per = d["flops"] / d["launches"]
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tf):
        t = json.load(open(tf)).get(name)
        if t and t.get("source_hash") == kernel_source_hash() and t.get("workload") == workload:
            traffic = t.get("dram_bytes_per_launch")
    if name in ("gemm_ax_fp32", "gemm_atx_fp32", "hals_rows", "gram_f64", "chol_inv", "whalf", "r_tile", "tv_tile"):
        # CUDA-core arithmetic: FP32 FFMA peak = SMs x 128 lanes x 2 flop x max SM clock.  The W half
        # keeps Q on chip (registers, shared memory, L2) and reads it twice per column: its HBM
        # bytes are only Q once and W once per sweep, its work 4 m l k flop per sweep.
        mhz = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
        ach = flops_per / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": traffic, "peak_source": "derived FP32 FFMA (152 SM x 128 x 2 x clock)",
                "launches": d["launches"], "avg_launch_ms": avg_s * 1e3}
    peak = peaks["hbm_gbs"]
    ach = bytes_per / avg_s / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": traffic, "peak_source": f"{peak_kind} hbm_gbs", "launches": d["launches"],
            "avg_launch_ms": avg_s * 1e3, "algorithmic_bytes_per_launch": bytes_per}


def oracle_golden(w):
    """The float64 oracle's stored trajectory of this workload (written by
    tests/golden/make_oracle_reference.py, float64 oracle only), or None."""
    p = os.path.join(ROOT, "tests", "golden", f"oracle_{w.name}.json")
    return json.load(open(p)) if os.path.exists(p) else None


def oracle_full_measured(w):
    """Measured full-size oracle solve time of this workload on a host like this
    one (same machine type and CPU count), from the stored oracle run, or None."""
    import platform
    g = oracle_golden(w)
    if not g:
        return None
    h = g.get("host", {})
    if h.get("machine") != platform.machine() or h.get("cpus") != os.cpu_count():
        return None
    return g["rhals"]["solve_s"]


def cpu_baseline(w, budget_s: float = 25.0, order: int = 0, init: int = 0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload: the same
    recipe scaled down by f in m and n with the same k, p, q, run for s sweeps;
    QB time scaled by 1/f^2 (passes over A), sweep time by iters/(s f) (sweep cost
    is linear in m + n).  f is chosen so that the sample's Q (m f x l float64) no
    longer fits the host caches, as the full one does not.  Returns (seconds
    extrapolated to the full solve, info); info["sample_s"] is the wall time that
    was actually measured."""
    from oracle import rhals as R
    from oracle import philox

    f = 0.3 if w.m * w.n > 1e8 else 1.0
    ms, ns = max(int(w.m * f), w.l + 1), max(int(w.n * f), w.l + 1)
    sw = synth.Workload(w.name + "_sample", ms, ns, w.r, w.k, w.p, w.q, w.iters, w.sigma, w.w0_exp,
                        w.h0_zero_frac, w.seed)
    A = synth.lowrank(sw).astype(np.float64)
    t0 = time.perf_counter()
    Q, B = R.rqb(A, philox.omega(ns, w.l, w.seed), w.q)
    t_qb = time.perf_counter() - t0
    if init == 1:
        from oracle import init_svd
        t0 = time.perf_counter()
        W0, H0 = init_svd.svd_init(Q, B, w.k)
        t_qb += time.perf_counter() - t0
    else:
        W0, H0 = philox.init_factors(ms, ns, w.k, w.seed)
    s = 1
    t0 = time.perf_counter()
    R.rhals_sweeps(Q, B, W0, H0, s, order=order)
    t1 = time.perf_counter() - t0
    s = max(1, min(w.iters, int((budget_s - t_qb) / max(t1, 1e-3))))
    t0 = time.perf_counter()
    R.rhals_sweeps(Q, B, W0, H0, s, order=order)
    t_sw = time.perf_counter() - t0
    full = t_qb / (f * f) + t_sw * (w.iters / s) / f
    extrapolated = f != 1.0 or s != w.iters
    try:
        from threadpoolctl import threadpool_info
        threads = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        threads = os.cpu_count()
    info = {"kind": "oracle", "cores": threads, "extrapolated": extrapolated, "sample_s": t_qb + t_sw + t1,
            "sample": f"FP64 oracle on {ms}x{ns} (same recipe, k={w.k}, p={w.p}, q={w.q}): QB {t_qb:.2f}s, "
                      f"{s} sweeps {t_sw:.2f}s" + (f"; extrapolated to {w.m}x{w.n} x {w.iters} sweeps "
                                                   f"(QB x 1/f^2, sweeps x iters/(s f), f={f})"
                                                   if extrapolated else "")}
    meas = oracle_full_measured(w) if extrapolated and order == 0 and init == 0 else None
    if meas:
        info["measured_full_solve_s"] = meas
        info["extrapolation_over_measured"] = full / meas
    return full, info


def oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        return os.cpu_count()


def cpu_baseline_adjoint(w):
    """The float64 reference gradient (oracle/adjoint.py) of the full workload: one
    forward + backward of T sweeps (it runs in about a second)."""
    from oracle import adjoint as AD
    from oracle import philox
    from oracle import rhals as R

    A = synth.lowrank(w).astype(np.float64)
    Q, _ = R.rqb(A, philox.omega(w.n, w.l, w.seed), w.q)
    W0, H0 = philox.init_factors(w.m, w.n, w.k, w.seed)
    G = synth.cotangent(w.m, w.n).astype(np.float64)
    t0 = time.perf_counter()
    AD.loss_and_grads(A, Q, W0, H0, G, w.iters)
    t = time.perf_counter() - t0
    return t, {"kind": "oracle", "cores": oracle_threads(), "extrapolated": False, "sample_s": t,
               "sample": f"full workload: float64 forward + reverse of {w.iters} sweeps on {w.m}x{w.n} "
                         f"(k={w.k}, l={w.l}), Q fixed"}


def cpu_baseline_batch(ws, budget_s: float = 20.0):
    """The float64 oracle on every 16th problem of the batch (until the budget is
    spent), extrapolated to all problems by the ratio of their m n (k + l) work."""
    from oracle import rhals as R

    work = [w.m * w.n * (w.k + w.l) for w in ws]
    done, t_sum, w_sum = 0, 0.0, 0.0
    for i in range(0, len(ws), 16):
        w = ws[i]
        A = synth.lowrank(w).astype(np.float64)
        t0 = time.perf_counter()
        R.rhals(A, w.k, w.p, w.q, w.iters, w.seed, instance=w.instance)
        t_sum += time.perf_counter() - t0
        w_sum += work[i]
        done += 1
        if t_sum > budget_s:
            break
    full = t_sum * sum(work) / w_sum
    return full, {"kind": "oracle", "cores": oracle_threads(), "extrapolated": done < len(ws), "sample_s": t_sum,
                  "sample": f"float64 oracle on {done} of {len(ws)} problems (every 16th) in {t_sum:.1f}s, "
                            f"extrapolated by total m n (k + l)"}


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    times, walls = [], []
    info = None
    for i in range(args.warmup + args.steps):
        t_step = time.perf_counter()
        if args.workload == "batch":
            bws = synth.batch_workloads()
            v, info = cpu_baseline_batch(bws, budget_s=8.0 if i >= args.warmup else 3.0)
            v = len(bws) / v
        elif args.workload == "adjoint":
            v, info = cpu_baseline_adjoint(w)
        else:
            v, info = cpu_baseline(w, budget_s=8.0 if i >= args.warmup else 3.0,
                                   order=args.extra.get("order", 0), init=args.extra.get("init", 0))
        if i >= args.warmup:
            times.append(v)
            walls.append(time.perf_counter() - t_step)
    val = statistics.mean(times)
    # ms_per_step is the wall time each timed step took (a bounded sample); value is
    # the metric for the whole workload, extrapolated from that sample when it is smaller
    wall_ms = statistics.mean(walls) * 1e3
    if args.workload == "batch":
        out = {"impl": "reference", "metric": METRIC_BATCH, "value": val, "unit": "problems/s", "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall_ms, "extrapolated": True,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": {"workload": "batch_512_ragged", "problems": 512},
               "cpu_baseline": dict(info, value=val, unit="problems/s"),
               "e2e": {"value": val, "unit": "problems/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    else:
        metric = METRIC_ADJOINT if args.workload == "adjoint" else METRIC
        out = {"impl": "reference", "metric": metric, "value": val, "unit": "s", "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall_ms,
               "extrapolated": bool(info.get("extrapolated", False)), "higher_is_better": False,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": w.name, "m": w.m, "n": w.n, "k": w.k, "p": w.p, "q": w.q,
                          "iters": w.iters},
               "cpu_baseline": dict(info, value=val, unit="s"),
               "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="precision", choices=sorted(WORKLOADS))
    ap.add_argument("--form", default="bf16", choices=sorted(FORMS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32-leg", action="store_true")
    ap.add_argument("--iters", type=int, default=None, help="override the sweep count (small probes)")
    ap.add_argument("--problems", type=int, default=512, help="batch workload: the first N problems (small probes)")
    ap.add_argument("--shape", default=None, help="MxN: the workload's recipe on an m x n matrix (small probes)")
    ap.add_argument("--alpha-w", type=float, default=0.0, help="Section 3.4 penalty on ||W||^2")
    ap.add_argument("--alpha-h", type=float, default=0.0, help="Section 3.4 penalty on ||H||^2")
    ap.add_argument("--beta-w", type=float, default=0.0, help="Section 3.4 l1 weight on W")
    ap.add_argument("--beta-h", type=float, default=0.0, help="Section 3.4 l1 weight on H")
    ap.add_argument("--pg-tol", type=float, default=0.0, help="Section 3.3 projected-gradient stopping tolerance")
    ap.add_argument("--pg-every", type=int, default=10, help="sweeps between projected-gradient checks")
    ap.add_argument("--order", default="cyclic", choices=["cyclic", "shuffled", "interleaved"],
                    help="Section 3.2 update order of the sweeps")
    ap.add_argument("--init", default="uniform", choices=["uniform", "svd"],
                    help="initial factors: U[0,1) or NNDSVD of the randomized SVD")
    ap.add_argument("--sweep-products", default="split3", choices=["fp32", "split3"],
                    help="tensor-core forms: the H half's products R, T, V in float32 on CUDA cores or in 3-term "
                         "split BF16 on tensor cores (the FP32 form always takes float32)")
    ap.add_argument("--subspace-report", action="store_true",
                    help="precision workload: compare the QB subspaces of the forms and the sweeps' sensitivity "
                         "to the basis (one JSON object, no timing)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    extra = dict(alpha_W=args.alpha_w, alpha_H=args.alpha_h, beta_W=args.beta_w, beta_H=args.beta_h,
                 pg_tol=args.pg_tol, pg_every=args.pg_every)
    args.extra = {k: v for k, v in extra.items() if v} if (args.pg_tol or args.alpha_w or args.alpha_h or
                                                           args.beta_w or args.beta_h) else {}
    if args.order != "cyclic":
        args.extra["order"] = {"shuffled": 1, "interleaved": 2}[args.order]
    if args.init != "uniform":
        args.extra["init"] = 1
    if args.workload == "batch" and args.impl != "reference":
        return main_batch(args)
    if args.workload == "adjoint" and args.impl != "reference":
        return main_adjoint(args)
    if args.workload == "streamed" and args.impl != "reference":
        return main_streamed(args, w)
    if args.workload == "scale" and args.impl != "reference":
        return main_scale(args, w)
    if args.subspace_report:
        return subspace_report(args, w)
    if args.iters or args.shape:
        m, n = (int(x) for x in args.shape.lower().split("x")) if args.shape else (w.m, w.n)
        name = w.name if not args.shape else f"{w.name}_as_{m}x{n}"
        w = synth.Workload(name, m, n, w.r, w.k, w.p, w.q, args.iters or w.iters, w.sigma, w.w0_exp,
                           w.h0_zero_frac, w.seed)
    if args.impl == "reference":
        return run_reference(args, w)

    import torch
    import paper_1711_02037_gb300 as pkg

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = local if ws > 1 else 0
    torch.cuda.set_device(dev)
    peaks, peak_kind = measured_peaks()

    # ---- input: generated on the host (same bytes the oracle sees), pinned, copied once
    t0 = time.perf_counter()
    A_host = torch.empty((w.m, w.n), dtype=torch.float32, pin_memory=True)
    synth.lowrank_into(A_host.numpy(), w)
    log(f"[bench] generated A {w.m}x{w.n} in {time.perf_counter() - t0:.1f}s")
    A = A_host.to(f"cuda:{dev}", non_blocking=False)
    ctx = pkg.Context(dev)
    form = FORMS[args.form]
    sweep_tc = {"fp32": 0, "split3": 1}[args.sweep_products]

    def fopts(prec):
        """Options of a form: the tensor-core forms take the H half's product choice."""
        return dict(args.extra, sweep_products=sweep_tc) if prec != 0 and sweep_tc else args.extra

    # ---- calibration (untimed): the target is 1.001 x the FP32 form's error after the
    # workload's sweep count; the measured form may run up to 3x that many sweeps to
    # reach it (the NMF is far from converged there and trajectories that start from
    # slightly different bases diverge by a few percent in either direction).  Runs are
    # deterministic, so the first checkpoint at or under the target fixes the sweep
    # count of every timed step.
    _, _, st32 = ctx.rnmf(A, w.k, w.p, w.q, w.iters, w.seed, precision=0, track_every=CHECK_EVERY, **args.extra)
    target = 1.001 * st32.rel_err_hist[-1]
    t32 = first_reach(st32.rel_err_hist, target)
    cap = 3 * w.iters
    if form == 0:
        stf = st32
    else:
        _, _, stf = ctx.rnmf(A, w.k, w.p, w.q, cap, w.seed, precision=form, track_every=CHECK_EVERY, **fopts(form))
    tstar = first_reach(stf.rel_err_hist, target)
    # the FP32-accurate tensor-core form (every QB product in 3-term split BF16) to the same target
    st3, t3 = None, None
    if form == 2:
        st3, t3 = stf, tstar
    elif not args.no_fp32_leg:
        _, _, st3 = ctx.rnmf(A, w.k, w.p, w.q, cap, w.seed, precision=2, track_every=CHECK_EVERY, **fopts(2))
        t3 = first_reach(st3.rel_err_hist, target)
    reached = tstar is not None
    iters = tstar if reached else cap
    err_at_iters = stf.rel_err_hist[min(w.iters, len(stf.rel_err_hist) * CHECK_EVERY) // CHECK_EVERY - 1]
    log(f"[bench] target {target:.6g} (fp32 error after {w.iters} sweeps {st32.rel_err_hist[-1]:.6g}); form "
        f"{args.form} reaches it at sweep {tstar} (its error after {w.iters} sweeps {err_at_iters:.6g})")

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    W = torch.empty((w.m, w.k), dtype=torch.float32, device=f"cuda:{dev}")
    H = torch.empty((w.k, w.n), dtype=torch.float32, device=f"cuda:{dev}")

    def step():
        ctx.rnmf(A, w.k, w.p, w.q, iters, w.seed, precision=form, W=W, H=H, **fopts(form))

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(dev)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    n0 = ctx.launches()
    total_ms, times = timed_steps(step, args.steps, flush, stream)
    torch.cuda.synchronize()
    launches = ctx.launches() - n0
    if ws > 1:
        torch.distributed.barrier()
    # the same steps again with per-launch events (kernel shares and the roofline)
    ctx.profile(True)
    prof_total, _ = timed_steps(step, args.steps, flush, stream)
    prof = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    total_ms = max_over_ranks(total_ms, ws, dev)
    ms_step = total_ms / args.steps
    final_err = ctx.rel_err(A, W, H)

    # ---- the FP32 forms to the same target (comparison legs, same timing method): the
    # CUDA-core form and the 3-term split BF16 tensor-core form
    def time_form(prec, sweeps):
        ctx.rnmf(A, w.k, w.p, w.q, sweeps, w.seed, precision=prec, W=W, H=H, **fopts(prec))
        tt = []
        for _ in range(max(1, min(args.steps, 2))):
            flush.fill_(1.0)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            ctx.rnmf(A, w.k, w.p, w.q, sweeps, w.seed, precision=prec, W=W, H=H, **fopts(prec))
            ev1.record(stream)
            ev1.synchronize()
            tt.append(ev0.elapsed_time(ev1))
        return statistics.mean(tt)

    fp32_ms = split3_ms = None
    if form != 0 and not args.no_fp32_leg:
        fp32_ms = time_form(0, t32)
    if form == 2:
        split3_ms = ms_step
    elif st3 is not None and t3 is not None:
        split3_ms = time_form(2, t3)

    # ---- error against the float64 oracle (its stored trajectory on this workload)
    vs_oracle = None
    g = oracle_golden(w) if not args.extra and not args.shape and not args.iters else None
    if g:
        ore = g["rhals"]["rel_err_every_10"]
        o_fin = ore[w.iters // CHECK_EVERY - 1]

        def dev_of(st):
            h = st.rel_err_hist[: len(ore)]
            return {"rel_err": h[w.iters // CHECK_EVERY - 1],
                    "rel_dev": abs(h[w.iters // CHECK_EVERY - 1] - o_fin) / o_fin,
                    "max_rel_dev_every_10": max(abs(a - b) / b for a, b in zip(h, ore))}
        vs_oracle = {"oracle_rel_err": o_fin, "sweeps": w.iters, "fp32": dev_of(st32),
                     "split3": dev_of(st3) if st3 is not None else None, args.form: dev_of(stf),
                     "oracle_host": g.get("host"), "source": f"tests/golden/oracle_{w.name}.json"}

    # ---- e2e: the host-buffer C-ABI call, H2D of A and D2H of W, H inside the timed region
    e2e = None
    if not args.no_e2e:
        Wh = torch.empty((w.m, w.k), dtype=torch.float32, pin_memory=True)
        Hh = torch.empty((w.k, w.n), dtype=torch.float32, pin_memory=True)
        ctx.rnmf_host(A_host, w.k, w.p, w.q, iters, w.seed, precision=form, W_host=Wh, H_host=Hh, **fopts(form))
        et = []
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.rnmf_host(A_host, w.k, w.p, w.q, iters, w.seed, precision=form, W_host=Wh, H_host=Hh, **fopts(form))
            et.append(time.perf_counter() - t0)
        e2e = {"value": statistics.mean(et), "unit": "s", "h2d_bytes_per_step": w.m * w.n * 4,
               "d2h_bytes_per_step": (w.m * w.k + w.k * w.n) * 4}
        del Wh, Hh

    if rank != 0:
        return
    rf = roofline(prof, peaks, peak_kind, w.name)
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        v, info = cpu_baseline(w, order=args.extra.get("order", 0), init=args.extra.get("init", 0))
        cpu = dict(info, value=v, unit="s")
    out = {
        "metric": METRIC, "value": ms_step / 1e3, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if form == 1 else "f32", "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "n": w.n, "k": w.k, "p": w.p, "q": w.q, "max_sweeps": w.iters,
                   "form": args.form, "sweep_products": args.sweep_products if form != 0 else "fp32",
                   "target_rel_err": target, "sweeps_to_target": tstar,
                   "target_reached": reached, "max_sweeps_allowed": cap, "fp32_form_sweeps_to_target": t32,
                   "fp32_form_time_to_target_s": fp32_ms / 1e3 if fp32_ms else None,
                   "speedup_vs_fp32_form": (fp32_ms / ms_step) if fp32_ms else None,
                   "split3_form_sweeps_to_target": t3,
                   "split3_form_time_to_target_s": split3_ms / 1e3 if split3_ms else None,
                   "speedup_vs_split3_form": (split3_ms / ms_step) if split3_ms else None,
                   "rel_err_vs_fp64_oracle": vs_oracle,
                   "final_rel_err": final_err, "parallelism": f"replicas{ws}",
                   "options": args.extra or None,
                   "l2": "inputs larger than L2 (A is 20 GB) and a 256 MB buffer written between steps"},
        "roofline": rf, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "gpu_launches_per_step": launches / args.steps, "clocks": clk,
        "profiled_ms_per_step": prof_total / args.steps,
        "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 4)} for k, v in
                    sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
        "step_ms": [round(t, 3) for t in times],
    }
    print(json.dumps(out), flush=True)


def subspace_report(args, w):
    """Where the BF16 form's extra sweeps come from.  For each form's QB (FP32 CUDA
    cores, BF16 power passes, 3-term split BF16 everywhere), in float64 from the
    library's Q: the range finder's residual ||A - Q Q^T A||_F / ||A||_F (Section
    2.3's approximation error) and the error of the library's B against Q^T A
    (relative Frobenius, and the relative bias of ||B||_F^2).  Then the sweeps' own
    sensitivity: the same FP32 QB in two other orthonormal bases (Q U, B^T U with
    U a seeded random orthogonal l x l matrix) - the same computation in exact
    arithmetic (the result depends on Q only through its range) - and two FP32
    ranges from other Gaussian test matrices (same initial factors), run for the
    workload's sweep count and 10 % more.  Analysis products use torch float64
    on the GPU, in row blocks of A."""
    import torch
    import paper_1711_02037_gb300 as pkg

    ws_, rank, dev = gpu_setup()
    A_host = torch.empty((w.m, w.n), dtype=torch.float32, pin_memory=True)
    synth.lowrank_into(A_host.numpy(), w)
    A = A_host.to(f"cuda:{dev}")
    ctx = pkg.Context(dev)
    rb = 8192
    a2 = sum(float((A[r:r + rb].double() ** 2).sum()) for r in range(0, w.m, rb))
    qbs = {}
    for name, prec in (("fp32", 0), ("bf16", 1), ("split3", 2)):
        Q, Bt = ctx.qb(A, w.l, w.q, w.seed, precision=prec)
        qbs[name] = (Q, Bt)
    # ranges of the same quality from other test matrices (Omega seeds), FP32 form
    for sd in (1, 2):
        qbs[f"fp32_omega_seed{sd}"] = ctx.qb(A, w.l, w.q, w.seed + 1000 * sd, precision=0)
    out = {"workload": w.name, "range_residual": {}, "B_rel_err": {}, "B_norm2_rel_bias": {}, "final_rel_err": {}}
    for name, (Q, Bt) in qbs.items():
        Qd = Q.double()
        QtA = torch.zeros((w.l, w.n), dtype=torch.float64, device=A.device)
        for r in range(0, w.m, rb):
            QtA += Qd[r:r + rb].T @ A[r:r + rb].double()
        res2 = 0.0
        for r in range(0, w.m, rb):
            res2 += float(((A[r:r + rb].double() - Qd[r:r + rb] @ QtA) ** 2).sum())
        out["range_residual"][name] = float(np.sqrt(res2 / a2))
        Bd = Bt.double().T
        out["B_rel_err"][name] = float(torch.linalg.norm(Bd - QtA) / torch.linalg.norm(QtA))
        out["B_norm2_rel_bias"][name] = float((Bd ** 2).sum() / (QtA ** 2).sum() - 1.0)
        del QtA
    W0, H0 = ctx.init_factors(w.m, w.n, w.k, w.seed)
    iters = [w.iters, w.iters + w.iters // 10]
    rng = np.random.default_rng(12345)

    def run(Q, Bt, label):
        W, H = W0.clone(), H0.clone()
        _, _, st = ctx.sweeps(Q, Bt, W, H, iters[1], A=A, track_every=CHECK_EVERY)
        out["final_rel_err"][label] = {str(t): st.rel_err_hist[t // CHECK_EVERY - 1] for t in iters}

    for name, (Q, Bt) in qbs.items():
        run(Q, Bt, name)
    Q32, Bt32 = qbs["fp32"]
    for r in range(2):
        U, _ = np.linalg.qr(rng.standard_normal((w.l, w.l)))
        Ud = torch.from_numpy(U).to(f"cuda:{dev}")
        run((Q32.double() @ Ud).float().contiguous(), (Bt32.double() @ Ud).float().contiguous(),
            f"fp32_rotated_{r}")
    e = out["final_rel_err"]
    base = e["fp32"][str(w.iters)]
    out["rel_spread_at_iters"] = {k: (v[str(w.iters)] - base) / base for k, v in e.items()}
    g = oracle_golden(w)
    if g:
        o = g["rhals"]["rel_err_every_10"][w.iters // CHECK_EVERY - 1]
        out["oracle_rel_err_at_iters"] = o
        out["rel_dev_from_oracle_at_iters"] = {k: (v[str(w.iters)] - o) / o for k, v in e.items()}
    print(json.dumps(out), flush=True)


def main_scale(args, w):
    """The paper's comparison at scale (Section 4.4): randomized HALS (FP32 form)
    and deterministic HALS (Section 3.1, two passes over A per sweep) for the same
    sweep count from the same initial factors.  One timed step = one rnmf solve;
    the deterministic HALS solve is timed the same way beside it."""
    import torch
    import paper_1711_02037_gb300 as pkg

    ws_, rank, dev = gpu_setup()
    peaks, peak_kind = measured_peaks()
    t0 = time.perf_counter()
    A_host = torch.empty((w.m, w.n), dtype=torch.float32, pin_memory=True)
    synth.lowrank_into(A_host.numpy(), w)
    log(f"[bench] generated A {w.m}x{w.n} in {time.perf_counter() - t0:.1f}s")
    A = A_host.to(f"cuda:{dev}")
    ctx = pkg.Context(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    W = torch.empty((w.m, w.k), device=f"cuda:{dev}")
    H = torch.empty((w.k, w.n), device=f"cuda:{dev}")
    stream = torch.cuda.current_stream()
    # untimed: error trajectories (every 10 sweeps) of both methods
    _, _, st_r = ctx.rnmf(A, w.k, w.p, w.q, w.iters, w.seed, track_every=CHECK_EVERY)
    _, _, st_h = ctx.hals(A, w.k, w.iters, w.seed, track_every=CHECK_EVERY)

    def step_r():
        ctx.rnmf(A, w.k, w.p, w.q, w.iters, w.seed, W=W, H=H)

    def step_h():
        ctx.hals(A, w.k, w.iters, w.seed, W=W, H=H)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step_r()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    n0 = ctx.launches()
    total_ms, times = timed_steps(step_r, args.steps, flush, stream)
    launches = ctx.launches() - n0
    ctx.profile(True)
    prof_total, _ = timed_steps(step_r, args.steps, flush, stream)
    prof = ctx.profile_read()
    ctx.profile(False)
    step_h()
    hs = max(1, min(args.steps, 2))
    h_ms, _ = timed_steps(step_h, hs, flush, stream)
    ctx.profile(True)
    timed_steps(step_h, 1, flush, stream)
    prof_h = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    total_ms = max_over_ranks(total_ms, ws_, dev)
    ms_step = total_ms / args.steps
    h_ms /= hs
    e2e = None
    if not args.no_e2e:
        Wh = torch.empty((w.m, w.k), pin_memory=True)
        Hh = torch.empty((w.k, w.n), pin_memory=True)
        ctx.rnmf_host(A_host, w.k, w.p, w.q, w.iters, w.seed, W_host=Wh, H_host=Hh)
        et = []
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.rnmf_host(A_host, w.k, w.p, w.q, w.iters, w.seed, W_host=Wh, H_host=Hh)
            et.append(time.perf_counter() - t0)
        e2e = {"value": statistics.mean(et), "unit": "s", "h2d_bytes_per_step": w.m * w.n * 4,
               "d2h_bytes_per_step": (w.m * w.k + w.k * w.n) * 4}
    if rank != 0:
        return
    vs_oracle = None
    g = oracle_golden(w)
    if g:
        def dev_of(hist, ore):
            return {"rel_err": hist[-1], "oracle_rel_err": ore[-1], "rel_dev": abs(hist[-1] - ore[-1]) / ore[-1],
                    "max_rel_dev_every_10": max(abs(a - b) / b for a, b in zip(hist, ore))}
        vs_oracle = {"rhals": dev_of(st_r.rel_err_hist, g["rhals"]["rel_err_every_10"]),
                     "hals": dev_of(st_h.rel_err_hist, g["hals"]["rel_err_every_10"]),
                     "oracle_host": g.get("host"), "source": f"tests/golden/oracle_{w.name}.json"}
    cpu = None
    if not args.no_cpu_baseline and ws_ == 1:
        v, info = cpu_baseline(w)
        cpu = dict(info, value=v, unit="s")
    out = {"metric": METRIC_SCALE, "value": ms_step / 1e3, "unit": "s", "n_gpus": ws_, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name, "m": w.m, "n": w.n, "k": w.k, "p": w.p, "q": w.q, "iters": w.iters,
                      "rhals_final_rel_err": st_r.rel_err_hist[-1], "hals_final_rel_err": st_h.rel_err_hist[-1],
                      "hals_time_s": h_ms / 1e3, "speedup_vs_hals": h_ms / ms_step,
                      "rel_err_vs_fp64_oracle": vs_oracle, "parallelism": f"replicas{ws_}",
                      "l2": "inputs larger than L2 (A is 4 GB) and a 256 MB buffer written between steps"},
           "roofline": roofline(prof, peaks, peak_kind, w.name),
           "roofline_hals": roofline(prof_h, peaks, peak_kind, w.name + "_hals"),
           "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
           "gpu_launches_per_step": launches / args.steps, "clocks": clk,
           "profiled_ms_per_step": prof_total / args.steps,
           "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 4)} for k, v in
                       sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
           "kernels_hals": {k: {"launches": v["launches"], "ms": round(v["ms"], 4)} for k, v in
                            sorted(prof_h.items(), key=lambda kv: -kv[1]["ms"])},
           "step_ms": [round(t, 3) for t in times]}
    print(json.dumps(out), flush=True)


def timed_steps(step, steps, flush, stream):
    """K steps, each bracketed by CUDA events on the launching stream, with the
    L2 flush buffer written before each (outside the events)."""
    import torch
    total, times = 0.0, []
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select these launches
    for _ in range(steps):
        flush.fill_(1.0)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        total += times[-1]
    torch.cuda.nvtx.range_pop()
    return total, times


def gpu_setup():
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = local if ws > 1 else 0
    torch.cuda.set_device(dev)
    return ws, rank, dev


def max_over_ranks(total_ms, ws, dev):
    """The job's time: the slowest rank's timed region (each rank times its own
    replica between barriers).  dev is the rank's GPU (NCCL), or None for a
    CPU process group (gloo)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], device=f"cuda:{dev}" if dev is not None else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return total_ms


def main_adjoint(args):
    """Forward + backward of T unrolled compressed sweeps (the differentiation
    workload): one step = rnmf_sweeps_fwd with checkpoints, the caller's loss
    gradient G H^T, W^T G, rnmf_sweeps_bwd and dA = Q dB, all through the C ABI."""
    import torch
    import paper_1711_02037_gb300 as pkg
    from oracle import philox
    from oracle import rhals as R

    w = synth.ADJOINT
    ws, rank, dev = gpu_setup()
    peaks, peak_kind = measured_peaks()
    A64 = synth.lowrank(w).astype(np.float64)
    Q64, _ = R.rqb(A64, philox.omega(w.n, w.l, w.seed), w.q)
    W0h, H0h = philox.init_factors(w.m, w.n, w.k, w.seed)
    Gh = synth.cotangent(w.m, w.n)
    cuda = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(f"cuda:{dev}")
    A, Q, W0, H0, G = cuda(A64), cuda(Q64), cuda(W0h), cuda(H0h), cuda(Gh)
    ctx = pkg.Context(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    W = torch.empty_like(W0)
    H = torch.empty_like(H0)
    ck = torch.empty(int(pkg.lib().rnmf_ckpt_floats(w.m, w.n, w.l, w.k, w.iters)), device=f"cuda:{dev}")

    def step():
        Bt = ctx.sketch(A, Q, transpose=True)
        W.copy_(W0)
        H.copy_(H0)
        lib = pkg.lib()
        o = pkg.default_opts()
        ctx._check(lib.rnmf_sweeps_fwd(ctx.h, Q.data_ptr(), Bt.data_ptr(), w.m, w.n, w.l, w.k, w.iters,
                                       pkg.ctypes.byref(o), W.data_ptr(), H.data_ptr(), ck.data_ptr()), ctx.h)
        dW = G @ H.T
        dH = W.T @ G
        dBt, dW0, dH0 = ctx.sweeps_bwd(Q, Bt, ck, dW, dH, w.iters)
        return ctx.dA(Q, dBt)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    n0 = ctx.launches()
    total_ms, times = timed_steps(step, args.steps, flush, stream)
    launches = ctx.launches() - n0
    ctx.profile(True)
    prof_total, _ = timed_steps(step, args.steps, flush, stream)
    prof = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    total_ms = max_over_ranks(total_ms, ws, dev)
    ms_step = total_ms / args.steps
    # e2e: host inputs (A, G, W0, H0) copied in, dA, dW0, dH0 copied out, every step
    e2e = None
    if not args.no_e2e:
        hA = torch.from_numpy(A64.astype(np.float32)).pin_memory()
        hG = torch.from_numpy(Gh).pin_memory()
        hW0 = torch.from_numpy(W0h.astype(np.float32)).pin_memory()
        hH0 = torch.from_numpy(H0h.astype(np.float32)).pin_memory()
        out_dA = torch.empty((w.m, w.n), pin_memory=True)
        et = []
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            A.copy_(hA, non_blocking=True)
            G.copy_(hG, non_blocking=True)
            W0.copy_(hW0, non_blocking=True)
            H0.copy_(hH0, non_blocking=True)
            dA = step()
            out_dA.copy_(dA)
            torch.cuda.synchronize()
            et.append(time.perf_counter() - t0)
        e2e = {"value": statistics.mean(et), "unit": "s",
               "h2d_bytes_per_step": (2 * w.m * w.n + w.m * w.k + w.k * w.n) * 4,
               "d2h_bytes_per_step": w.m * w.n * 4}
    if rank != 0:
        return
    rf = roofline(prof, peaks, peak_kind, w.name)
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        v, info = cpu_baseline_adjoint(w)
        cpu = dict(info, value=v, unit="s")
    out = {"metric": METRIC_ADJOINT, "value": ms_step / 1e3, "unit": "s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": w.name, "m": w.m, "n": w.n, "k": w.k, "l": w.l, "T": w.iters,
                      "parallelism": f"replicas{ws}",
                      "l2": "256 MB buffer written between steps (inputs 32 MB each)"},
           "roofline": rf, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
           "gpu_launches_per_step": launches / args.steps, "clocks": clk,
           "profiled_ms_per_step": prof_total / args.steps,
           "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 4)} for k, v in
                       sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
           "step_ms": [round(t, 3) for t in times]}
    print(json.dumps(out), flush=True)


def main_streamed(args, w):
    """A (the precision recipe, 20 GB) in pinned host memory; QB over column blocks
    (Algorithm 2, q + 2 passes of host->device copies overlapped with the products),
    then the sweeps on the GPU.  One step = one rnmf_streamed call."""
    import torch
    import paper_1711_02037_gb300 as pkg

    ws_, rank, dev = gpu_setup()
    t0 = time.perf_counter()
    A_host = torch.empty((w.m, w.n), dtype=torch.float32, pin_memory=True)
    synth.lowrank_into(A_host.numpy(), w)
    log(f"[bench] generated A {w.m}x{w.n} in host memory in {time.perf_counter() - t0:.1f}s")
    ctx = pkg.Context(dev)
    Wd = torch.empty((w.m, w.k), device=f"cuda:{dev}")
    Hd = torch.empty((w.k, w.n), device=f"cuda:{dev}")
    bc = 4096
    stats = []

    form = FORMS[args.form]
    # the tensor-core forms take the sweeps' product choice, as in the in-memory benchmark
    sweep_tc = 1 if form != 0 and args.sweep_products == "split3" else 0

    def step():
        stats.append(ctx.rnmf_streamed(A_host, w.k, w.p, w.q, w.iters, w.seed, block_cols=bc, W=Wd, H=Hd,
                                       precision=form, sweep_products=sweep_tc)[2])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    n0 = ctx.launches()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    stats.clear()
    total_ms, times = timed_steps(step, args.steps, flush, torch.cuda.current_stream())
    launches = ctx.launches() - n0
    clk = clocks.stop()
    total_ms = max_over_ranks(total_ms, ws_, dev)
    ms_step = total_ms / args.steps
    qb_ms = statistics.mean(s.ms_qb for s in stats)
    moved = (w.q + 2) * 4.0 * w.m * w.n
    if rank != 0:
        return
    peaks, peak_kind = measured_peaks()
    out = {"metric": METRIC_STREAMED, "value": ms_step / 1e3, "unit": "s", "n_gpus": ws_, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16" if form == 1 else "f32", "data": "synthetic",
           "config": {"workload": w.name + "_host_resident", "m": w.m, "n": w.n, "k": w.k, "p": w.p, "q": w.q,
                      "iters": w.iters, "block_cols": bc, "passes_over_A": w.q + 2, "form": args.form,
                      "sweep_products": "split3" if sweep_tc else "fp32",
                      "qb_ms": qb_ms, "host_to_device_GBps_during_QB": moved / (qb_ms / 1e3) / 1e9,
                      "parallelism": f"replicas{ws_}", "l2": "A streamed from host memory every pass"},
           "roofline": {"kernel": "column-blocked QB passes (copy-bound)", "bound": "hbm",
                        "achieved": moved / (qb_ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": moved / (qb_ms / 1e3) / 1e9 / peaks["hbm_gbs"], "traffic": None,
                        "peak_source": f"{peak_kind} hbm_gbs (the host link is the binding limit)"},
           "cpu_baseline": None, "e2e": {"value": ms_step / 1e3, "unit": "s",
                                         "h2d_bytes_per_step": int(moved), "d2h_bytes_per_step": 0},
           "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps, "clocks": clk,
           "step_ms": [round(t, 3) for t in times]}
    print(json.dumps(out), flush=True)


def batch_bytes(ws):
    """Algorithmic HBM bytes of one batch: (2q + 2) float32 passes over every A
    (sketch, q power iterations of two passes, projection) plus, per sweep, B^T and
    H read and H written (the Q re-reads of the W half come from L2 / L1)."""
    b = 0
    for w in ws:
        b += (2 * w.q + 2) * 4 * w.m * w.n
        b += w.iters * 4 * (w.n * w.l + 2 * w.k * w.n + 2 * w.k * w.m)
    return b


def main_batch(args):
    """512 ragged problems through rnmf_batched (one graph replay per step)."""
    import torch
    import paper_1711_02037_gb300 as pkg

    ws_, rank, dev = gpu_setup()
    peaks, peak_kind = measured_peaks()
    bws = synth.batch_workloads()[: args.problems]
    t0 = time.perf_counter()
    hosts, items = [], []
    for w in bws:
        Ah = torch.from_numpy(synth.lowrank(w)).pin_memory()
        hosts.append(Ah)
        items.append(dict(A=Ah.to(f"cuda:{dev}"), k=w.k, p=w.p, q=w.q, iters=w.iters, seed=w.seed,
                          instance=w.instance, W=torch.empty(w.m, w.k, device=f"cuda:{dev}"),
                          H=torch.empty(w.k, w.n, device=f"cuda:{dev}")))
    log(f"[bench] generated {len(bws)} problems ({sum(w.m * w.n for w in bws) * 4 / 1e9:.1f} GB) "
        f"in {time.perf_counter() - t0:.1f}s")
    ctx = pkg.Context(dev)
    _, st0 = ctx.batched(items)  # builds the plan: autotuning + capture (untimed)
    for _ in range(args.warmup):
        ctx.batched(items)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(dev)
    n0 = ctx.launches()
    clocks.start()
    time.sleep(0.3)
    total_ms, times = 0.0, []
    for _ in range(args.steps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        _, st = ctx.batched(items)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        total_ms += times[-1]
    clk = clocks.stop()
    launches = ctx.launches() - n0
    total_ms = max_over_ranks(total_ms, ws_, dev)
    ms_step = total_ms / args.steps
    errs = ctx.batched_rel_err(items)
    # e2e: every A copied from pinned host memory, every W, H copied back, per step
    e2e = None
    if not args.no_e2e:
        Wh = [torch.empty(it["W"].shape, pin_memory=True) for it in items]
        Hh = [torch.empty(it["H"].shape, pin_memory=True) for it in items]
        et = []
        for _ in range(max(1, min(args.steps, 3))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for it, Ah in zip(items, hosts):
                it["A"].copy_(Ah, non_blocking=True)
            ctx.batched(items)
            for it, a, b in zip(items, Wh, Hh):
                a.copy_(it["W"], non_blocking=True)
                b.copy_(it["H"], non_blocking=True)
            torch.cuda.synchronize()
            et.append(time.perf_counter() - t0)
        e2e = {"value": len(bws) / statistics.mean(et), "unit": "problems/s",
               "h2d_bytes_per_step": sum(w.m * w.n for w in bws) * 4,
               "d2h_bytes_per_step": sum(w.m * w.k + w.k * w.n for w in bws) * 4}
    if rank != 0:
        return
    nbytes = batch_bytes(bws)
    ach = nbytes / (ms_step / 1e3) / 1e9
    rf = {"kernel": "whole batch graph (QB tile kernels + cluster sweeps)", "bound": "hbm", "achieved": ach,
          "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "traffic": None,
          "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch": nbytes}
    cpu = None
    if not args.no_cpu_baseline and ws_ == 1 and len(bws) >= 16:
        v, info = cpu_baseline_batch(bws)
        cpu = dict(info, value=len(bws) / v, unit="problems/s")
    out = {"metric": METRIC_BATCH, "value": len(bws) * ws_ / (ms_step / 1e3), "unit": "problems/s", "n_gpus": ws_,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batch_512_ragged" if len(bws) == 512 else f"batch_first_{len(bws)}_of_512",
                      "problems": len(bws), "m": "U{256..8192}",
                      "n": "U{128..4096}", "k": "U{4..32}", "p": 10, "q": 2, "iters": 100,
                      "parallelism": f"replicas{ws_}", "graph_kernels": st0["graph_kernels"],
                      "cluster_count": st0["cluster_count"], "threads_small": st0["threads_small"],
                      "autotune_ms": st0["tune_ms"], "rel_err_median": float(np.median(errs)),
                      "rel_err_max": float(np.max(errs)),
                      "l2": "inputs larger than L2 (18.7 GB of A per step)"},
           "roofline": rf, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
           "gpu_launches_per_step": launches / args.steps, "clocks": clk,
           "step_ms": [round(t, 3) for t in times]}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
