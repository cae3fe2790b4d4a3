"""Serving measurement: a stream of completion jobs through the serving runtime.

    python -m paper_0810_3286_gb300.serve_bench [--jobs 100] [--slots 8] [--loads 0.5,0.8,0.95] [--single 8]
                                                [--batch 16]

Jobs follow the serving workload: m, n uniform in [500, 8000], rank uniform in 5..20,
|Omega| = c r (m + n - r) with c uniform in [4, 6], N(0,1) planted factors, eps = 1e-4,
tau = 5 sqrt(m n), delta = 1.2 m n / |Omega|.  Three measurements on the same jobs:
  * saturated: all jobs submitted at once; mu = completed jobs per second;
  * Poisson: arrivals at load x mu (exponential gaps) for every load of --loads, time to eps of
    every job measured from its arrival, p50 / p99 by nearest rank;
  * one job at a time (slots = 1) in float32 and in float64 on the first `--single` jobs: mean time
    to eps per job, the plain single-job baseline;
  * batched (svt_batch_solve) on the first `--batch` jobs (at most 32), float32 and float64, with the
    fixed tile rule and with the tuner: all jobs in one lockstep batch, time to eps of each job
    from the batch's start, makespan, and the same jobs one at a time for comparison.
Every job is capped at K_MAX = 500 SVT iterations; jobs that end without meeting the stopping rule
(iteration cap, more than 64 singular values above tau, Lanczos stagnation) are counted as failed
and left out of the latency percentiles.  Prints one JSON line.  Problem generation happens before
any timing.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


K_MAX = 500


def _submit(srv, p, precision):
    return srv.submit(p.n1, p.n2, p.rows, p.cols, p.vals, p.tau_default(), p.delta_default(), 1e-4, 64,
                      precision=precision, k_max=K_MAX)


def _closed_loop(jobs, slots, precision):
    from paper_0810_3286_gb300.serve import Server
    with Server(slots=slots) as srv:
        ids = [_submit(srv, p, precision) for p in jobs]
        srv.drain()
        st = srv.stats()
        res = [srv.wait(i) for i in ids]
    return st, res


def _poisson(jobs, slots, rate, seed):
    from paper_0810_3286_gb300.serve import Server
    rng = np.random.default_rng(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=len(jobs))
    with Server(slots=slots) as srv:
        ids = []
        t_next = time.perf_counter()
        for p, g in zip(jobs, gaps):
            t_next += g
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ids.append(_submit(srv, p, "fp32"))
        srv.drain()
        st = srv.stats()
        for i in ids:
            srv.wait(i)
    return st


def _batched(jobs, precision, autotune, concurrent=True):
    import torch
    from paper_0810_3286_gb300 import Solver, batch_solve
    solvers = [Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision=precision, k_max=K_MAX) for p in jobs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res, st = batch_solve(solvers, [p.tau_default() for p in jobs], [p.delta_default() for p in jobs], 1e-4, 64,
                          autotune=autotune, concurrent=concurrent)
    wall = time.perf_counter() - t0
    for s in solvers:
        s.close()
    ok = [r for r, c in zip(res, st) if c == 0]
    ms = sorted(r["ms"] for r in ok)
    return {"jobs": len(jobs), "converged": len(ok), "makespan_ms": 1000.0 * wall,
            "mean_time_to_eps_ms": float(np.mean(ms)) if ms else None,
            "p50_ms": ms[(len(ms) - 1) // 2] if ms else None, "max_ms": ms[-1] if ms else None,
            "solves_per_s": len(ok) / wall, "iterations": [int(r["iterations"]) for r in res]}


def _one_at_a_time(jobs, precision):
    import torch
    from paper_0810_3286_gb300 import Solver, SVTError
    out = []
    t0 = time.perf_counter()
    for p in jobs:
        with Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision=precision, k_max=K_MAX) as s:
            try:
                r = s.solve(p.tau_default(), p.delta_default(), 1e-4, 64, raise_on_nonconvergence=False)
            except SVTError:   # rank limit or Lanczos stagnation: a failed job, as in the batch
                r = {"converged": 0, "ms": 0.0, "iterations": -1}
            out.append(r)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ok = [r for r in out if r["converged"]]
    return {"jobs": len(jobs), "converged": len(ok), "makespan_ms": 1000.0 * wall,
            "mean_solve_ms": float(np.mean([r["ms"] for r in ok])) if ok else None,
            "solves_per_s": len(ok) / wall, "iterations": [int(r["iterations"]) for r in out]}


def run_batch(jobs):
    """Batched vs one at a time vs served on the same jobs."""
    out = {"one_at_a_time": {}, "batched": {}, "batched_autotune": {}, "batched_in_order": {}}
    for prec in ("fp32", "fp64"):
        out["one_at_a_time"][prec] = _one_at_a_time(jobs, prec)
        out["batched"][prec] = _batched(jobs, prec, False)
        out["batched_autotune"][prec] = _batched(jobs, prec, True)
        out["batched_in_order"][prec] = _batched(jobs, prec, False, concurrent=False)
    st, res = _closed_loop(jobs, 8, "fp32")
    ok = [r for r in res if r["status"] == 0]
    out["served_8_slots_fp32"] = {"converged": len(ok), "solves_per_s": st["solves_per_s"], "p50_ms": st["p50_ms"],
                                  "p99_ms": st["p99_ms"]}
    return out


def run(n_jobs=100, slots=8, loads=(0.5, 0.8, 0.95), n_single=8, seed=0, n_batch=0):
    from svt_inputs import serving_job
    jobs = [serving_job(seed * 1_000_003 + i) for i in range(n_jobs)]
    nnz_mean = float(np.mean([p.nnz for p in jobs]))
    # warm-up: library load, first contexts
    _closed_loop(jobs[:2], 2, "fp32")
    sat, res = _closed_loop(jobs, slots, "fp32")
    mu = sat["solves_per_s"]
    failed = sum(1 for r in res if r["status"] != 0)
    poisson = []
    for load in loads:
        poi = _poisson(jobs, slots, load * mu, seed + 17)
        poisson.append({"load": load, "arrival_rate_per_s": load * mu, "solves_per_s": poi["solves_per_s"],
                        "p50_ms": poi["p50_ms"], "p99_ms": poi["p99_ms"], "mean_ms": poi["mean_ms"],
                        "completed": poi["completed"], "failed": poi["failed"]})
    single = {}
    for prec in (("fp32", "fp64") if n_single > 0 else ()):
        st, r = _closed_loop(jobs[:n_single], 1, prec)
        ok = [x for x in r if x["status"] == 0]
        single[prec] = {"jobs": n_single, "converged": len(ok),
                        "mean_time_to_eps_ms": float(np.mean([x["t_end_ms"] - x["t_start_ms"] for x in ok])) if ok else None,
                        "solves_per_s": st["solves_per_s"]}
    batch = run_batch(jobs[:min(n_batch, 32)]) if n_batch > 0 else None
    return {
        "workload": "%d jobs: m, n ~ U[500, 8000], rank ~ U{5..20}, |Omega| = c r (m + n - r), c ~ U[4, 6], "
                    "mean |Omega| %.0f, eps 1e-4, at most %d iterations, float32" % (n_jobs, nnz_mean, K_MAX),
        "batch": batch,
        "slots": slots,
        "saturated": {"solves_per_s": mu, "p50_ms": sat["p50_ms"], "p99_ms": sat["p99_ms"],
                      "peak_jobs_in_flight": sat["peak_running"], "peak_device_bytes": sat["peak_bytes"],
                      "failed": failed},
        "poisson": poisson,
        "one_job_at_a_time": single,
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--jobs", type=int, default=100)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--loads", default="0.5,0.8,0.95", help="Poisson loads as fractions of the saturated rate")
    ap.add_argument("--single", type=int, default=8)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--batch", type=int, default=0, help="jobs of the batched comparison (at most 32)")
    args = ap.parse_args()
    from paper_0810_3286_gb300 import build
    build.build()
    loads = tuple(float(x) for x in args.loads.split(",") if x)
    print(json.dumps(run(args.jobs, args.slots, loads, args.single, args.seed, args.batch)))


if __name__ == "__main__":
    main()
