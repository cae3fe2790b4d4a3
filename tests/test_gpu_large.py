"""Full-size rank-10 workloads of Table 1 (Sec. 5.2.1) on the float32 path, checked by properties
that hold at any size (no oracle run inside the test).

Table 1 averages five random instances per row; here five seeds per shape are solved with
tau = 5n, delta = 1.2/p, eps = 1e-4 (eq. (5.5)), and:

* the mean iteration count over the instances is within +-15% of the paper's value for that row
  (123 at 10000 x 10000, 124 at 20000 x 20000, 125 at 30000 x 30000).  An instance is left out of
  the mean only when a committed trace of the float64 sparse-tier oracle (tests/golden/, written
  by make_tierb_trace.py from the oracle alone) shows that the iteration itself needs more than
  1.15 times the paper's count on it (seed 4 at 10000 x 10000, seeds 0 and 2 at 30000 x 30000: an
  (r+1)-th singular value of the dual iterate hovers at tau and the rank briefly rises to r + 1);
  such instances are followed iterate by iterate against their trace in
  test_gpu_slow_instances.py;
* every instance that converges within the paper's count (+15%) ends at the planted rank (the
  slow ones at r or r + 1), and every instance that meets the stopping rule has relative error
  ||X - M||_F / ||M||_F (eq. (5.8), closed form from the factors) below the 2e-4 the paper reports
  for all of Table 1;
* on one converged instance the final shrink satisfies the certificate of Theorem 2.1: with
  X = D_tau(Y) = U diag(sigma - tau) V^T, (Y - X) V = tau U on the kept singular vectors, where
  Y V comes from the library's own sparse product.
"""
import os
import sys

import numpy as np
import pytest

from svt_inputs import planted_problem, sample_count

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, GOLDEN)
from make_tierb_trace import read_trace  # noqa: E402

WORKLOAD = {10000: "single_10000", 30000: "large_30000"}


def _oracle_slow(n, seed, paper_iters):
    """True when the committed oracle trace of this instance needs more than 1.15x the paper's count
    (it did not stop by then); False when there is no such trace."""
    if n not in WORKLOAD:
        return False
    path = os.path.join(GOLDEN, "tierb_trace_%s_seed%d.txt" % (WORKLOAD[n], seed))
    if not os.path.exists(path):
        return False
    head, _, rows = read_trace(path)
    limit = int(1.15 * paper_iters)
    return len(rows) > limit and all(res > float(head["eps"]) for k, _, _, _, res, _ in rows if k <= limit)

pytestmark = pytest.mark.gpu

SEEDS = range(5)


def _relerr(U, d, V, A, B):
    nx2 = float(np.sum(d * d))
    nm2 = float(np.trace((A.T @ A) @ (B.T @ B)))
    xm = float(np.trace(np.diag(d) @ (U.T @ A) @ (B.T @ V)))
    return np.sqrt(max(nx2 - 2 * xm + nm2, 0.0) / nm2)


def _certificate(torch, s, U, d, V, tau):
    r = U.shape[1]
    Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    W = torch.empty((U.shape[0], r), dtype=torch.float64, device="cuda")
    s.apply_Y(Vd, W)
    torch.cuda.synchronize()
    lhs = W.cpu().numpy() - U * d   # (Y - X) V, with X V = U diag(d) for orthonormal V
    return np.linalg.norm(lhs - tau * U) / (tau * np.sqrt(r))


@pytest.mark.parametrize("n,paper_iters", [(10000, 123), (20000, 124), (30000, 125)])
def test_table1_rank10_rows(cuda, n, paper_iters):
    torch = cuda
    from paper_0810_3286_gb300 import Solver
    r = 10
    m = sample_count(n, n, r, 6.0)
    iters, checked = [], False
    for seed in SEEDS:
        p = planted_problem(n, n, r, m, seed)
        with Solver(n, n, torch.from_numpy(p.rows).cuda(), torch.from_numpy(p.cols).cuda(),
                    torch.from_numpy(p.vals).cuda(), precision="fp32", k_max=1500) as s:
            res = s.solve(p.tau_default(), p.delta_default(), 1e-4, 27, raise_on_nonconvergence=False)
            iters.append(res["iterations"])
            # an instance that converges in the paper's count has the planted rank; on the slow
            # instances the stop can fall inside an excursion to rank r + 1
            if res["converged"] and res["iterations"] <= 1.15 * paper_iters:
                assert res["rank"] == r, (seed, res)
            else:
                assert r <= res["rank"] <= r + 1, (seed, res)
            if res["converged"]:
                assert res["residual"] <= 1e-4
                U, d, V = s.factors()
                err = _relerr(U, d, V, p.A, p.B)
                assert err < 2e-4, (seed, err)
                if not checked:
                    # the factors are those of the last shrink, of the Y before its final update;
                    # that update moves Y V by at most delta * eps * ||P_Omega M||_F
                    assert _certificate(torch, s, U, d, V, p.tau_default()) < 1e-3, seed
                    checked = True
    kept = [it for sd, it in zip(SEEDS, iters) if not _oracle_slow(n, sd, paper_iters)]
    assert len(kept) >= 3, iters
    mean = float(np.mean(kept))
    print("n = %d: iterations %s, mean over the instances kept %.1f" % (n, iters, mean))
    assert 0.85 * paper_iters <= mean <= 1.15 * paper_iters, iters
    assert checked, iters


@pytest.mark.parametrize("n,r,ratio,paper_iters", [(1000, 50, 4.0, 114)])
def test_table1_rank50_row(cuda, n, r, ratio, paper_iters):
    """Table 1's 1000 x 1000 rank-50 row (m / d_r = 4, 39% of the entries sampled; 114 iterations,
    relative error 1.59e-4): a shrink of more than 28 wanted triplets, so the thick restarts keep
    two blocks of Ritz pairs.  Five instances: mean iteration count within +-15%, the planted rank,
    relative error below 2e-4."""
    torch = cuda
    from paper_0810_3286_gb300 import Solver
    m = sample_count(n, n, r, ratio)
    iters = []
    for seed in SEEDS:
        p = planted_problem(n, n, r, m, seed)
        with Solver(n, n, torch.from_numpy(p.rows).cuda(), torch.from_numpy(p.cols).cuda(),
                    torch.from_numpy(p.vals).cuda(), precision="fp32") as s:
            res = s.solve(p.tau_default(), p.delta_default(), 1e-4, 64)
            assert res["converged"] and res["rank"] == r, (seed, res)
            U, d, V = s.factors()
            err = _relerr(U, d, V, p.A, p.B)
            assert err < 2e-4, (seed, err)
            iters.append(res["iterations"])
    mean = float(np.mean(iters))
    print("n = %d, r = %d: iterations %s, mean %.1f" % (n, r, iters, mean))
    assert 0.85 * paper_iters <= mean <= 1.15 * paper_iters, iters
