"""Serving runtime on the GPU: jobs admitted by slots and memory, overlapping on the device.

* Every job's result in a mix of concurrent jobs is the one it gives alone (same status,
  iterations, rank, residual and factors, bit for bit: the same kernels, launch shapes and
  fixed-order reductions run in both cases), in float32 and float64.  "Alone" is a context with
  the cooperative-grid cap the server gives its jobs (max(16, 2 SMs / slots)).
* With a budget of 2.5 times the largest job's footprint, the footprints in flight never exceed
  it, several jobs are in flight at once, and the jobs finish.
"""
import numpy as np
import pytest

from svt_inputs import serving_job

pytestmark = pytest.mark.gpu


def _small_jobs(k, seed0):
    # the better-conditioned end of the serving distribution (oversampling 5.5 - 6): SVT with
    # tau = 5 sqrt(m n) and delta = 1.2 / p converges on these within k_max
    return [serving_job(seed0 + i, n_range=(500, 1200), rank_range=(8, 12), c_range=(5.5, 6.0)) for i in range(k)]


def _server_orth_grid(slots):
    import torch
    return max(16, 2 * torch.cuda.get_device_properties(0).multi_processor_count // slots)


def _alone(p, precision, orth_grid=0):
    from paper_0810_3286_gb300 import Solver
    from paper_0810_3286_gb300._abi import SVTError
    with Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision=precision, orth_grid=orth_grid) as s:
        try:
            res = s.solve(p.tau_default(), p.delta_default(), 1e-4, 27, raise_on_nonconvergence=False)
            return (0 if res["converged"] else 6), res, s.factors()
        except SVTError as ex:
            return ex.status, None, None


@pytest.mark.parametrize("precision,k", [("fp32", 8), ("fp64", 3)])
def test_results_same_alone_and_in_mix(cuda, precision, k):
    from paper_0810_3286_gb300.serve import Server
    jobs = _small_jobs(k, 500)
    if precision == "fp64":
        jobs = [serving_job(900 + i, n_range=(150, 300), rank_range=(3, 6), c_range=(5.5, 6.0)) for i in range(k)]
    alone = [_alone(p, precision, _server_orth_grid(4)) for p in jobs]
    with Server(slots=4, keep_factors=True) as srv:
        ids = [srv.submit(p.n1, p.n2, p.rows, p.cols, p.vals, p.tau_default(), p.delta_default(), 1e-4, 27,
                          precision=precision) for p in jobs]
        mixed = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["completed"] + st["failed"] == k
    assert sum(1 for a in alone if a[0] == 0) >= k - 1       # the jobs are meant to converge
    for (status, res, fac), m in zip(alone, mixed):
        assert m["status"] == status
        if res is None:
            continue
        U, d, V = fac
        assert m["iterations"] == res["iterations"] and m["rank"] == res["rank"]
        assert m["residual"] == res["residual"]
        assert np.array_equal(m["d"], d) and np.array_equal(m["U"], U) and np.array_equal(m["V"], V)


def test_memory_budget_and_overlap(cuda):
    import ctypes
    from paper_0810_3286_gb300 import library, _abi
    from paper_0810_3286_gb300.serve import Server
    L = library()
    jobs = _small_jobs(12, 700)
    o = _abi.svt_options()
    L.svt_default_options(ctypes.byref(o))
    o.precision = _abi.SVT_FP32
    biggest = max(L.svt_estimate_device_bytes(p.n1, p.n2, p.nnz, ctypes.byref(o)) for p in jobs)
    budget = int(2.5 * biggest)
    with Server(slots=8, device_budget=budget) as srv:
        ids = [srv.submit(p.n1, p.n2, p.rows, p.cols, p.vals) for p in jobs]
        srv.drain()
        st = srv.stats()
        res = [srv.wait(i) for i in ids]
    assert st["completed"] + st["failed"] == 12 and st["completed"] >= 11
    assert st["peak_bytes"] <= budget
    assert st["peak_running"] >= 2
    assert all(r["residual"] <= 1e-4 for r in res if r["status"] == 0)


def test_orth_grid_cap_same_solution(cuda):
    # a capped cooperative grid changes only the row chunks of the Gram sums (rounding order)
    from paper_0810_3286_gb300 import Solver
    from svt_inputs import config_problem
    p = config_problem("single_1000", 0)
    out = []
    for g in (0, 16):
        with Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp32", orth_grid=g) as s:
            res = s.solve(p.tau_default(), p.delta_default(), 1e-4, 27)
            U, d, V = s.factors()
            out.append((res, (U * d) @ V.T))
    (r0, X0), (r1, X1) = out
    assert r0["converged"] and r1["converged"] and r0["rank"] == r1["rank"] == 10
    assert abs(r0["iterations"] - r1["iterations"]) <= 1
    assert np.linalg.norm(X1 - X0) <= 1e-3 * np.linalg.norm(X0)


_ORACLE_RUNS = []   # the oracle's solves of the three jobs, shared by both precisions


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-5), ("fp32", 1e-3)])
def test_mix_against_oracle_rectangular(cuda, precision, bound):
    """Rectangular jobs of the serving distribution (m != n, rank 5 - 12, |Omega| = c r (m + n - r)
    with c in [5.5, 6]) run as a mix of concurrent jobs in the server, each compared with the float64
    sparse-tier oracle run alone on the same job: the same stopping iteration (float64), X on Omega
    within the per-iterate bound of the path (1e-5 float64, 1e-3 float32) at the final iterate, and
    ||X - X_oracle||_F / ||X_oracle||_F (closed form from the factors) within 1e-3."""
    from oracle import svt_sparse
    from oracle.sparse import sample_X
    from paper_0810_3286_gb300.serve import Server
    jobs = [serving_job(1300 + i, n_range=(500, 700), rank_range=(5, 12), c_range=(5.5, 6.0)) for i in range(3)]
    assert any(p.n1 != p.n2 for p in jobs)
    if not _ORACLE_RUNS:
        _ORACLE_RUNS.extend(svt_sparse.svt(p.n1, p.n2, p.rows, p.cols, p.vals, p.tau_default(), p.delta_default(),
                                           k_max=600, keep_trace=False) for p in jobs)
    refs = _ORACLE_RUNS
    assert all(r.converged for r in refs)
    with Server(slots=3, keep_factors=True) as srv:
        ids = [srv.submit(p.n1, p.n2, p.rows, p.cols, p.vals, p.tau_default(), p.delta_default(), 1e-4, 64,
                          precision=precision, k_max=600) for p in jobs]
        out = [srv.wait(i) for i in ids]
    for p, ref, o in zip(jobs, refs, out):
        assert o["status"] == 0, (p.n1, p.n2, p.r, o)
        if precision == "fp64":
            assert o["iterations"] == ref.iters, (o["iterations"], ref.iters)
        else:
            assert abs(o["iterations"] - ref.iters) <= 2, (o["iterations"], ref.iters)
        assert o["rank"] == ref.d.shape[0] == p.r
        x = sample_X(p.rows, p.cols, o["U"] * o["d"], o["V"])
        x_ref = sample_X(p.rows, p.cols, ref.U * ref.d, ref.V)
        assert np.linalg.norm(x - x_ref) <= bound * np.linalg.norm(x_ref)
        # ||X - X_ref||_F from the factors: ||X||^2 + ||X_ref||^2 - 2 <X, X_ref>
        G = (o["U"].T @ ref.U) * np.outer(o["d"], ref.d) * (o["V"].T @ ref.V)
        nx, nr = float(np.sum(o["d"] ** 2)), float(np.sum(ref.d ** 2))
        assert np.sqrt(max(nx + nr - 2 * G.sum(), 0.0) / nr) <= 1e-3
