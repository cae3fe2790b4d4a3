"""Noisy completion (Sec. 5.2.1, noisy model eq. (5.9), early stop eq. (5.10)) on the GPU.

* Parity of the float64 path with the oracle on the 200 x 200 rank-5 workload with noise ratio
  0.1: X^k on Omega within 1e-5 every iterate, same ranks, same stopping iteration.
* Table 2, rank-10 rows (1000 x 1000, m / d_r = 6, five seeds as the paper averages five runs),
  float32 path, eps of eq. (5.10) = 0 (the paper leaves it unspecified; this reading reproduces
  its Table 2): mean iteration count within +-15 % of 51 and 19 (noise ratio 1e-2, 1e-1) and within
  one iteration of 3 (noise ratio 1); mean relative error ||X - M||_F / ||M||_F within +-15 % of
  0.78e-2, 0.72e-1 and 0.52.
"""
import math

import numpy as np
import pytest

from oracle import svt as osvt
from oracle.sparse import sample_X
from svt_inputs import config_problem

pytestmark = pytest.mark.gpu


def _noisy(name, seed, ratio):
    p0 = config_problem(name, seed)
    sigma = ratio * np.linalg.norm(p0.vals) / math.sqrt(p0.nnz)
    return config_problem(name, seed, noise_sigma=sigma), sigma


def _relerr(U, d, V, A, B):
    nx2 = float(np.sum(d * d))
    nm2 = float(np.trace((A.T @ A) @ (B.T @ B)))
    xm = float(np.trace(np.diag(d) @ (U.T @ A) @ (B.T @ V)))
    return math.sqrt(max(nx2 - 2 * xm + nm2, 0.0) / nm2)


def test_noisy_parity_fp64_200(cuda):
    from paper_0810_3286_gb300 import Solver
    p, sigma = _noisy("plain_fp64_200", 0, 0.1)
    tau, delta = p.tau_default(), p.delta_default()
    ref = osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, tau, delta, noise_sigma=sigma, noise_eps=0.0)
    assert ref.converged
    s = Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64")
    s.set_noise_stop(sigma, 0.0)
    s.configure(tau, delta, 1e-4, 27, ref.k0)
    stopped_at = None
    for rec in ref.trace:
        info = s.step()
        U, d, V = s.factors()
        x = sample_X(p.rows, p.cols, U * d, V)
        err = np.linalg.norm(x - rec.x_omega) / max(np.linalg.norm(rec.x_omega), 1e-2 * np.linalg.norm(p.vals))
        assert err <= 1e-5, (info["k"], err)
        assert info["r"] == rec.r_k
        if info["stopped"]:
            stopped_at = info["k"]
            break
    assert stopped_at == ref.iters
    s.close()


@pytest.mark.parametrize("ratio,paper_iters,paper_err", [(1e-2, 51, 0.78e-2), (1e-1, 19, 0.72e-1), (1.0, 3, 0.52)])
def test_table2_rank10_rows(cuda, ratio, paper_iters, paper_err):
    torch = cuda
    from paper_0810_3286_gb300 import Solver
    iters, errs = [], []
    for seed in range(5):
        p, sigma = _noisy("single_1000", seed, ratio)
        with Solver(p.n1, p.n2, torch.from_numpy(p.rows).cuda(), torch.from_numpy(p.cols).cuda(),
                    torch.from_numpy(p.vals).cuda(), precision="fp32") as s:
            s.set_noise_stop(sigma, 0.0)
            res = s.solve(p.tau_default(), p.delta_default(), 1e-4, 27)
            assert res["converged"] == 1
            U, d, V = s.factors()
            iters.append(res["iterations"])
            errs.append(_relerr(U, d, V, p.A, p.B))
    mi, me = float(np.mean(iters)), float(np.mean(errs))
    if paper_iters >= 10:
        assert 0.85 * paper_iters <= mi <= 1.15 * paper_iters, iters
    else:
        assert abs(mi - paper_iters) <= 1.0, iters
    assert 0.85 * paper_err <= me <= 1.15 * paper_err, errs
