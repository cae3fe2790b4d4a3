"""Pins of the sparse oracle tier (oracle/svt_sparse.py) against the dense tier and LAPACK.

* partial_svd: the leading singular values of random sparse matrices with a planted decaying
  spectrum agree with numpy.linalg.svd (LAPACK) to 1e-11 relative, the singular subspaces to
  1e-9, and every returned triplet has Ritz residual <= 1e-12 sigma_1.
* svt: Algorithm 1 with the sparse shrink reproduces the dense tier on the 200 x 200 rank-5
  workload iterate by iterate (X^k on Omega within 1e-9, identical ranks and s_k, the same k0 and
  the same iteration count) and on a ragged rectangular problem.
"""
import numpy as np
import pytest

from oracle import svt as osvt
from oracle import svt_sparse as ssvt
from svt_inputs import planted_problem, random_sparse_pattern


@pytest.mark.parametrize("n1,n2,m,k,seed", [(300, 250, 6000, 6, 0), (180, 400, 9000, 12, 1)])
def test_partial_svd_matches_lapack(n1, n2, m, k, seed):
    rows, cols, vals = random_sparse_pattern(n1, n2, m, seed)
    p = planted_problem(n1, n2, 8, m, seed)
    # iterate-like values: a low-rank part on the pattern plus noise
    vals = 40.0 * p.vals[: rows.size] if p.vals.size >= rows.size else vals
    Y = ssvt.sparse_iterate(n1, n2, rows, cols, vals[: rows.size])
    ps = ssvt.partial_svd(Y, k, tol=1e-12)
    s_ref = np.linalg.svd(Y.toarray(), compute_uv=False)
    assert np.abs(ps.s - s_ref[:k]).max() <= 1e-11 * s_ref[0]
    assert np.all(ps.res <= 1e-12 * ps.s[0] * 1.0000001)
    Ud, sd, Vdt = np.linalg.svd(Y.toarray(), full_matrices=False)
    # subspace of the leading triplets with a clear gap after them
    gap_ok = [i for i in range(1, k) if s_ref[i - 1] - s_ref[i] > 1e-3 * s_ref[0]]
    j = gap_ok[-1] if gap_ok else k
    P1 = ps.V[:, :j] @ ps.V[:, :j].T
    P2 = Vdt[:j].T @ Vdt[:j]
    assert np.abs(P1 - P2).max() <= 1e-9


def _compare(p, dense, sparse_res):
    assert sparse_res.k0 == dense.k0
    assert sparse_res.iters == dense.iters
    assert sparse_res.converged == dense.converged
    for a, b in zip(sparse_res.trace, dense.trace):
        assert a.r_k == b.r_k and a.s_k == b.s_k and a.passes == b.passes
        den = max(np.linalg.norm(b.x_omega), 1e-2 * np.linalg.norm(p.vals))
        assert np.linalg.norm(a.x_omega - b.x_omega) <= 1e-9 * den, a.k
        assert a.res == pytest.approx(b.res, rel=1e-9, abs=1e-13)


def test_sparse_tier_matches_dense_tier_200(oracle_c1_run):
    p, dense = oracle_c1_run
    res = ssvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, p.tau_default(), p.delta_default())
    _compare(p, dense, res)


def test_sparse_tier_matches_dense_tier_rectangular():
    p = planted_problem(140, 95, 4, 4300, 9)
    tau, delta = p.tau_default(), p.delta_default()
    dense = osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, tau, delta)
    res = ssvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, tau, delta)
    _compare(p, dense, res)
