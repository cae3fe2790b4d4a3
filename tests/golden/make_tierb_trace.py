"""Writes the float64 sparse-tier oracle's per-iterate trace of one Table 1 workload instance.

Usage:  python tests/golden/make_tierb_trace.py <workload> <seed> [k_max]
        (workload names as in svt_inputs.CONFIGS, e.g. single_10000 4)
        python tests/golden/make_tierb_trace.py --thin <trace file>
        (keeps the sampled values of every 10th iterate and of the last one only)

Runs Algorithm 1 (Sec. 5.1.5) with the oracle's sparse shrink (oracle/svt_sparse.py: block
subspace iteration with Rayleigh-Ritz through the oracle's Jacobi SVD, Ritz residuals <= 1e-12
sigma_1) on the planted instance of svt_inputs, with tau = 5n, delta = 1.2/p, eps = 1e-4 (Sec.
5.2.1), until the stopping rule eq. (5.5) holds or k_max iterations (default 400) have run.  Only
oracle/ and the input generator are called.  The output file

    tests/golden/tierb_trace_<workload>_seed<seed>.txt

holds a header (sizes, parameters, k0 of eq. (5.3), ||P_Omega M||_2, and 64 positions of Omega in
row-major order, drawn by a fixed PCG64 stream) and one line per iterate:

    k  r_k  s_k  passes  residual  [x_1 .. x_64]

with x_i = X^k at the i-th sampled position (every iterate as written; --thin keeps them on every
10th iterate and the last one).  Lines are flushed as they are produced, so a run that is stopped
early leaves a valid prefix.
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import svt_sparse  # noqa: E402
from svt_inputs import config_problem  # noqa: E402

N_SAMPLE = 64
SAMPLE_SEED = 20081001


def sample_positions(nnz: int) -> np.ndarray:
    rng = np.random.default_rng(np.random.PCG64(SAMPLE_SEED))
    return np.sort(rng.choice(nnz, size=min(N_SAMPLE, nnz), replace=False)).astype(np.int64)


def trace_path(workload: str, seed: int) -> str:
    return os.path.join(HERE, "tierb_trace_%s_seed%d.txt" % (workload, seed))


def thin(path: str, every: int = 10) -> None:
    """Rewrites a trace keeping the sampled X values of every `every`-th iterate and of the last."""
    with open(path) as f:
        lines = f.readlines()
    data = [i for i, ln in enumerate(lines) if ln.strip() and not ln.startswith("#")]
    last = data[-1] if data else -1
    out = []
    for i, ln in enumerate(lines):
        if i in data and i != last and int(ln.split()[0]) % every != 0:
            ln = " ".join(ln.split()[:5]) + "\n"
        out.append(ln)
    with open(path + ".tmp", "w") as f:
        f.writelines(out)
    os.replace(path + ".tmp", path)


def main(argv) -> int:
    if argv[1] == "--thin":
        thin(argv[2])
        return 0
    workload, seed = argv[1], int(argv[2])
    k_max = int(argv[3]) if len(argv) > 3 else 400
    p = config_problem(workload, seed)
    tau, delta, eps = p.tau_default(), p.delta_default(), 1e-4
    pos = sample_positions(p.nnz)
    out = trace_path(workload, seed)
    tmp = out + ".partial"
    t0 = time.time()
    with open(tmp, "w") as f:
        f.write("# float64 sparse-tier oracle trace (oracle/svt_sparse.py), written by tests/golden/make_tierb_trace.py\n")
        f.write("# workload %s seed %d n1 %d n2 %d r %d nnz %d\n" % (workload, seed, p.n1, p.n2, p.r, p.nnz))
        f.write("# tau %.17g delta %.17g eps %.17g tol 1e-12 k_max %d\n" % (tau, delta, eps, k_max))
        f.write("# positions %s\n" % " ".join(str(int(i)) for i in pos))
        f.flush()

        def on_iter(rec):
            f.write("%d %d %d %d %.17g %s\n" % (rec.k, rec.r_k, rec.s_k, rec.passes, rec.res,
                                                 " ".join("%.17g" % v for v in rec.x_omega[pos])))
            f.flush()
            print("k %d r %d res %.6e  (%.0f s)" % (rec.k, rec.r_k, rec.res, time.time() - t0), flush=True)

        res = svt_sparse.svt(p.n1, p.n2, p.rows, p.cols, p.vals, tau, delta, eps=eps, k_max=k_max,
                             keep_trace=False, on_iter=on_iter)
        f.write("# k0 %d norm2 %.17g converged %d iterations %d\n" % (res.k0, res.norm2, int(res.converged),
                                                                       res.iters))
    os.replace(tmp, out)
    print("wrote %s (%d iterations, converged %s, %.0f s)" % (out, res.iters, res.converged, time.time() - t0))
    return 0


def read_trace(path: str):
    """(header dict, positions, rows) with rows = list of (k, r_k, s_k, passes, res, x_sample or None)."""
    head, pos, rows = {}, None, []
    with open(path) as f:
        for line in f:
            if line.startswith("# positions"):
                pos = np.array([int(t) for t in line.split()[2:]], dtype=np.int64)
            elif line.startswith("#"):
                tok = line[1:].split()
                for i in range(len(tok) - 1):
                    if tok[i] in ("workload", "seed", "n1", "n2", "r", "nnz", "tau", "delta", "eps", "k0", "norm2",
                                  "converged", "iterations", "k_max"):
                        head[tok[i]] = tok[i + 1]
            elif line.strip():
                t = line.split()
                rows.append((int(t[0]), int(t[1]), int(t[2]), int(t[3]), float(t[4]),
                             np.array([float(v) for v in t[5:]]) if len(t) > 5 else None))
    return head, pos, rows


if __name__ == "__main__":
    sys.exit(main(sys.argv))
