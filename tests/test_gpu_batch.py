"""Batched engine (svt_batch_solve): Algorithm 1 for several completion problems at once, with the
sparse products and the fused updates of all jobs as single persistent launches over the ragged
job list.

* Against each job solved alone with the shrink decided on the host (svt_solve with device_loop =
  0, the decisions the batch takes), in the batch's in-order mode (concurrent = 0: solo launch
  shapes) with the fixed tile rule: the same stopping iteration, rank and k0, and the final X on
  Omega to 1e-13 in float64 and float32 (every sparse product and update entry is computed exactly
  as in the solo run; only the residual sums are grouped differently).
* The concurrent mode (default: jobs' own kernels on their own streams with smaller cooperative
  grids) against the oracle, with and without the tuner.
* Against the float64 oracle (oracle/svt.py, Algorithm 1 with exact SVDs): the same stopping
  iteration and X on Omega within 1e-5 for every job of a ragged batch (square and rectangular,
  ranks 2-5).
* The tuner (autotune = 1) changes only the grouping of the sparse products' sums: the oracle's
  stopping iteration and X within 1e-5 of it.
* A job that stops early (its own k_max reached) leaves the batch with its own status; the others
  match their solo runs.  Bad batches are rejected with SVT_ERR_ARG.
"""
import numpy as np
import pytest

from oracle import svt as osvt
from oracle.sparse import sample_X
from svt_inputs import planted_problem

pytestmark = pytest.mark.gpu


def _x(s, p):
    U, d, V = s.factors()
    return sample_X(p.rows, p.cols, U * d, V)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problems():
    # several tiles of rows per job, ragged last tiles, square and rectangular, ranks 2-5, m / d_r = 6;
    # the float64 oracle stops them after 130, 163, 169 and 150 iterations
    shapes = [(160, 260, 5, 23), (120, 90, 2, 24), (256, 64, 3, 25), (200, 200, 5, 0)]
    return [planted_problem(n1, n2, r, 6 * r * (n1 + n2 - r), seed=sd) for n1, n2, r, sd in shapes]


def _solo(p, prec, **kw):
    from paper_0810_3286_gb300 import Solver
    s = Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision=prec, device_loop=False, **kw)
    res = s.solve(p.tau_default(), p.delta_default(), 1e-4, 27, raise_on_nonconvergence=False)
    x = _x(s, p)
    s.close()
    return res, x


def _oracle_x(p, ref):
    return sample_X(p.rows, p.cols, ref.U * ref.d, ref.V)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_each_job_alone(cuda, prec):
    from paper_0810_3286_gb300 import Solver, batch_solve
    probs = _problems()
    solo = [_solo(p, prec) for p in probs]
    solvers = [Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision=prec) for p in probs]
    res, st = batch_solve(solvers, [p.tau_default() for p in probs], [p.delta_default() for p in probs], 1e-4, 27,
                          concurrent=False)
    assert st == [0] * len(probs), st
    for p, s, r, (r1, x1) in zip(probs, solvers, res, solo):
        x = _x(s, p)
        assert r["converged"] == 1 and r1["converged"] == 1
        assert r["k0"] == r1["k0"] and r["rank"] == r1["rank"]
        assert r["iterations"] == r1["iterations"], (r["iterations"], r1["iterations"])
        assert _rel(x, x1) <= 1e-13, _rel(x, x1)
        assert r["ms"] > 0
        s.close()


@pytest.fixture(scope="module")
def oracle_refs():
    return [osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, p.tau_default(), p.delta_default(), eps=1e-4, k_max=400,
                     keep_trace=False) for p in _problems()]


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_against_oracle_fp64(cuda, oracle_refs, autotune):
    from paper_0810_3286_gb300 import Solver, batch_solve
    probs = _problems()
    solvers = [Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64") for p in probs]
    res, st = batch_solve(solvers, [p.tau_default() for p in probs], [p.delta_default() for p in probs], 1e-4, 27,
                          autotune=autotune)
    assert st == [0] * len(probs)
    for p, s, r, ref in zip(probs, solvers, res, oracle_refs):
        assert ref.converged
        assert r["k0"] == ref.k0 and r["rank"] == ref.rank
        assert r["iterations"] == ref.iters, (r["iterations"], ref.iters)
        xr = _oracle_x(p, ref)
        err = np.linalg.norm(_x(s, p) - xr) / max(np.linalg.norm(xr), 1e-2 * np.linalg.norm(p.vals))
        assert err <= 1e-5, err
        s.close()


def test_failed_job_leaves_the_others_untouched(cuda):
    from paper_0810_3286_gb300 import Solver, batch_solve
    from paper_0810_3286_gb300._abi import SVT_ERR_NOT_CONVERGED
    probs = _problems()[:3]
    solo = [_solo(p, "fp64") for p in probs]
    # the first job may run 5 iterations only: it leaves the batch after iteration 5
    solvers = [Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64", k_max=5 if i == 0 else 1000)
               for i, p in enumerate(probs)]
    res, st = batch_solve(solvers, [p.tau_default() for p in probs], [p.delta_default() for p in probs], 1e-4, 27,
                          concurrent=False)
    assert st[0] == SVT_ERR_NOT_CONVERGED and res[0]["iterations"] == 5 and res[0]["converged"] == 0
    for i in (1, 2):
        assert st[i] == 0 and res[i]["iterations"] == solo[i][0]["iterations"]
        assert _rel(_x(solvers[i], probs[i]), solo[i][1]) <= 1e-13
    for s in solvers:
        s.close()


def test_bad_batches_are_rejected(cuda):
    from paper_0810_3286_gb300 import Solver, SVTError, batch_solve
    p = _problems()[0]
    a = Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64")
    b = Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp32")
    with pytest.raises(SVTError):
        batch_solve([a, b])        # two precisions
    with pytest.raises(SVTError):
        batch_solve([a, a])        # the same context twice
    a.close()
    b.close()
