"""Pins of the oracle's alternative shrink engines (Sec. 6), each against a result the mathematics
fixes independently of the code under test.

* The test block's random columns are the published SplitMix64 outputs (tests/golden, Steele, Lea &
  Flood 2014) mapped to [-1, 1): checked value by value.
* With as many test columns as min(n1, n2), the range finder spans the whole column space, so the
  randomized shrink must equal the exact one (D_tau by the full SVD, eq. (2.2)); on an exactly
  rank-q iterate, any l >= q columns must give the exact shrink too (Q Q^T Y = Y).
* With a single tau the continuation is Algorithm 1 itself (same iterates as oracle.svt).
* With a schedule tau_0 < tau_1, the continuation's final X solves the same problem as the direct
  run at tau_1: both stop at eq. (5.5) with eps and agree to the accuracy the stopping rule leaves.
* A planted mistake (the warm columns dropped and replaced by zeros, so Omega loses rank) is caught
  by the exact-shrink comparison.
"""
import os

import numpy as np
import pytest

from oracle import alt_shrink, svt as osvt
from oracle.svt_sparse import sparse_iterate
from svt_inputs import planted_problem

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64_vectors.txt")


def _golden_outputs():
    """{seed: [output 1, output 2, ...]} from the published reference outputs."""
    seeds = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        seed, idx, out = (int(t) for t in line.split())
        seeds.setdefault(seed, {})[idx] = out
    return {sd: [d[i] for i in sorted(d)] for sd, d in seeds.items()}


def test_test_block_is_splitmix64_mapped_to_pm1():
    for seed, outs in _golden_outputs().items():
        k = min(len(outs), 6)
        blk = alt_shrink.test_block(1, k, 0, seed)
        want = np.array([(z >> 11) * (2.0 / 9007199254740992.0) - 1.0 for z in outs[:k]])
        assert np.array_equal(blk[0], want)
        assert np.all(blk >= -1.0) and np.all(blk < 1.0)


def _exact(Y, tau):
    U, d, V, _ = osvt.shrink(Y.toarray(), tau)
    return (U * d) @ V.T


def test_full_range_randomized_shrink_is_exact():
    p = planted_problem(40, 32, 3, 600, seed=5)
    Y = sparse_iterate(p.n1, p.n2, p.rows, p.cols, 3.0 * p.vals)
    tau = 0.5 * np.linalg.norm(Y.toarray(), 2)
    # l = 32 = min(n1, n2) test columns: the range finder spans the whole column space
    sh = alt_shrink.randomized_shrink(Y, tau, 0, None, ell=5, oversample=24, power=0, seed_of_pass=lambda ps: 7 + ps)
    X = (sh.U * sh.d) @ sh.V.T
    assert np.abs(X - _exact(Y, tau)).max() <= 1e-10 * np.abs(X).max()


def test_low_rank_iterate_randomized_shrink_is_exact():
    rng = np.random.default_rng(3)
    A, B = rng.standard_normal((40, 4)), rng.standard_normal((35, 4))
    import scipy.sparse as sp
    Y = sp.csr_matrix(A @ B.T)   # full support: a rank-4 iterate
    tau = 0.2 * np.linalg.norm(A @ B.T, 2)
    sh = alt_shrink.randomized_shrink(Y, tau, 0, None, ell=5, oversample=4, power=0, seed_of_pass=lambda ps: ps)
    X = (sh.U * sh.d) @ sh.V.T
    assert np.abs(X - _exact(Y, tau)).max() <= 1e-9 * np.abs(X).max()


def test_planted_mistake_zero_warm_columns_is_caught():
    p = planted_problem(40, 32, 3, 600, seed=5)
    Y = sparse_iterate(p.n1, p.n2, p.rows, p.cols, 3.0 * p.vals)
    tau = 0.2 * np.linalg.norm(Y.toarray(), 2)
    # a warm start of 28 zero columns: Omega has rank 4 only, the range misses directions
    bad = alt_shrink.randomized_shrink(Y, tau, 27, np.zeros((32, 28)), ell=5, oversample=4, power=0,
                                       seed_of_pass=lambda ps: 7 + ps)
    Xb = (bad.U * bad.d) @ bad.V.T
    assert np.abs(Xb - _exact(Y, tau)).max() > 1e-6 * np.abs(Xb).max()


def _small():
    # 60 x 50, rank 3, |Omega| = 6 r (n1 + n2 - r): the paper's oversampling on a small instance
    return planted_problem(60, 50, 3, 6 * 3 * (60 + 50 - 3), seed=11)


def test_continuation_with_one_tau_is_algorithm_1():
    p = _small()
    tau, delta = p.tau_default(), p.delta_default()
    ref = osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, tau, delta, k_max=300)
    cont = alt_shrink.svt_continuation(p.n1, p.n2, p.rows, p.cols, p.vals, [tau], delta, k_max=300)
    assert cont.iters == ref.iters and cont.k0 == ref.k0 and cont.converged == ref.converged
    for a, b in zip(cont.trace, ref.trace):
        assert a.r_k == b.r_k
        assert np.abs(a.x_omega - b.x_omega).max() <= 1e-10 * max(1.0, np.abs(b.x_omega).max())


def test_continuation_reaches_the_direct_solution():
    p = _small()
    tau, delta = p.tau_default(), p.delta_default()
    ref = osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, tau, delta, eps=1e-6, k_max=1000)
    cont = alt_shrink.svt_continuation(p.n1, p.n2, p.rows, p.cols, p.vals, [tau / 4, tau / 2, tau], delta,
                                       eps=1e-6, k_max=1000)
    assert ref.converged and cont.converged and len(cont.stage_iters) == 3
    Xr = (ref.U * ref.d) @ ref.V.T
    Xc = (cont.U * cont.d) @ cont.V.T
    assert np.linalg.norm(Xc - Xr) <= 1e-3 * np.linalg.norm(Xr)
