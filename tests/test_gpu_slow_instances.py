"""Slow instances of Table 1's rank-10 shapes, checked against the float64 sparse-tier oracle's
committed trace.

Sec. 5.2.1 reports every run below 200 SVT iterations (Table 1 averages five random instances per
shape).  Some instances drawn here need more: at 10000 x 10000 the instance of seed 4 takes 270
iterations in the oracle (oracle/svt_sparse.py, written from the paper and pinned against the
dense tier).  Its trace (tests/golden/, written by make_tierb_trace.py, which calls only the
oracle) shows why: from k = 95 on, an eleventh singular value of the dual iterate crosses tau
every few dozen iterations, the rank goes to 11 for one iterate and the residual of eq. (5.5)
jumps ten-fold before it decays again.  The iterate at which each crossing happens depends on
perturbations far below any float64 tolerance: the float64 GPU path run with Ritz tolerances of
1e-8, 1e-10 and 1e-11 sigma_1 follows the oracle to 1e-6 and better up to k = 121, then leaves
its sequence of crossings at different excursions and converges after 270, 265 and 225
iterations respectively.  So the float64 GPU path (same k0 as the oracle) must:

* up to the oracle's first excursion of the rank above the planted rank: have the same rank r_k
  every iterate, the relative residual within 1e-3 relative (1e-8 absolute), and X on the
  trace's 64 sampled entries within 1e-5 (the float64 per-iterate bound, the error denominator
  guarded at 1e-2 ||M||);
* after it: be a slow instance as well (residual above eps at 1.15 times the paper's count for
  the shape), keep its rank at r or r + 1, and, where the oracle converged, converge by 1.15 times
  the oracle's count with relative error ||X - M||_F / ||M||_F below the 2e-4 of Table 1.
"""
import os
import sys

import numpy as np
import pytest

from svt_inputs import config_problem

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
from make_tierb_trace import read_trace  # noqa: E402

TRACES = sorted(f for f in os.listdir(GOLDEN) if f.startswith("tierb_trace_") and f.endswith(".txt"))
PAPER_ITERS = {10000: 123, 20000: 124, 30000: 125}   # Table 1, rank 10, m / d_r = 6


def _relerr(U, d, V, A, B):
    nx2 = float(np.sum(d * d))
    nm2 = float(np.trace((A.T @ A) @ (B.T @ B)))
    xm = float(np.trace(np.diag(d) @ (U.T @ A) @ (B.T @ V)))
    return np.sqrt(max(nx2 - 2 * xm + nm2, 0.0) / nm2)


@pytest.mark.parametrize("fname", TRACES)
def test_fp64_path_against_oracle_trace(cuda, fname):
    torch = cuda
    from paper_0810_3286_gb300 import Solver
    head, pos, rows = read_trace(os.path.join(GOLDEN, fname))
    p = config_problem(head["workload"], int(head["seed"]))
    assert p.nnz == int(head["nnz"])
    tau, delta = p.tau_default(), p.delta_default()
    assert tau == pytest.approx(float(head["tau"]), rel=1e-15) and delta == pytest.approx(float(head["delta"]),
                                                                                           rel=1e-15)
    pr, pc = p.rows[pos].astype(np.int64), p.cols[pos].astype(np.int64)
    mnorm = np.linalg.norm(p.vals[pos])
    k_sync = next((k for k, r_k, *_ in rows if r_k > p.r), len(rows) + 1)
    oracle_converged = head["converged"] == "1"
    slow_at = int(1.15 * PAPER_ITERS[p.n1])
    k_end = int(1.15 * len(rows)) if oracle_converged else len(rows)
    with Solver(p.n1, p.n2, torch.from_numpy(p.rows).cuda(), torch.from_numpy(p.cols).cuda(),
                torch.from_numpy(p.vals).cuda(), precision="fp64", k_max=k_end + 5) as s:
        s.configure(tau, delta, 1e-4, 27, int(head["k0"]))
        worst, stopped_at = 0.0, None
        for k in range(1, k_end + 1):
            info = s.step()
            assert info["k"] == k
            if k < k_sync:
                _, r_k, _, _, res, xs = rows[k - 1]
                assert info["r"] == r_k, (k, info["r"], r_k)
                assert info["residual"] == pytest.approx(res, rel=1e-3, abs=1e-8), (k, info["residual"], res)
                if xs is not None:
                    U, d, V = s.factors()
                    x = np.einsum("pj,j,pj->p", U[pr], d, V[pc])
                    err = np.linalg.norm(x - xs) / max(np.linalg.norm(xs), 1e-2 * mnorm)
                    worst = max(worst, err)
                    assert err <= 1e-5, (k, err)
            else:
                assert p.r <= info["r"] <= p.r + 1, (k, info["r"])
            if info["stopped"]:
                stopped_at = k
                break
        assert stopped_at is None or stopped_at > slow_at, (stopped_at, slow_at)
        if oracle_converged:
            assert stopped_at is not None, k_end
            U, d, V = s.factors()
            assert _relerr(U, d, V, p.A, p.B) < 2e-4
        else:
            assert stopped_at is None
    print("%s: parity through k = %d (worst sampled error %.2e), stopped at %s (oracle: %d, converged %s)"
          % (fname, k_sync - 1, worst, stopped_at, len(rows), oracle_converged))
