"""Failure statuses of the C-ABI, each made to happen on purpose without faulting the GPU.

* SVT_ERR_TIMEOUT: the grid-barrier waits of the cooperative orthonormalisation are bounded; the
  test lowers the bound to one poll (svt_set_barrier_spins), so that early CTAs give up, the
  kernel returns and the host reads the error word.  The same context then solves again at the
  normal bound and must follow the float64 oracle iterate by iterate (the barrier word was reset).
* SVT_ERR_OOM: every device allocation of a context goes through the caller's allocator hook;
  a hook that refuses its k-th request makes svt_create fail cleanly (no leak: a second context
  of the same size fits and solves), for several k.
* SVT_ERR_NUMERIC: a NaN placed in the dual iterate (svt_set_Y) reaches the basis Grams and the
  step reports it; a NaN in the sampled values is rejected by svt_create (SVT_ERR_ARG).
* SVT_ERR_RANK_LIMIT: a max_rank below the planted rank.
* SVT_ERR_NOT_CONVERGED: a k_max below the iteration count; the factors of the last iterate stay.
"""
import ctypes

import numpy as np
import pytest

from svt_inputs import config_problem, planted_problem

pytestmark = pytest.mark.gpu


def _status_of(fn):
    from paper_0810_3286_gb300 import SVTError
    try:
        fn()
    except SVTError as e:
        return e.status
    return 0


def test_barrier_timeout_then_context_recovers(cuda, oracle_c1_run):
    torch = cuda
    from oracle.sparse import sample_X
    from paper_0810_3286_gb300 import Solver, library
    L = library()
    p, ref = oracle_c1_run
    tau, delta = p.tau_default(), p.delta_default()
    s = Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64")
    assert L.svt_set_barrier_spins(s._ctx, 1) == 0
    st = _status_of(lambda: s.configure(tau, delta, 1e-4, 27, ref.k0))
    assert st == 8, st   # SVT_ERR_TIMEOUT
    assert b"grid barrier" in L.svt_last_error(s._ctx)
    # normal bound again: the same context must now reproduce the oracle's iterates
    assert L.svt_set_barrier_spins(s._ctx, 0) == 0
    s.configure(tau, delta, 1e-4, 27, ref.k0)
    worst = 0.0
    for rec in ref.trace:
        info = s.step()
        U, d, V = s.factors()
        x = sample_X(p.rows, p.cols, U * d, V)
        denom = max(np.linalg.norm(rec.x_omega), 1e-2 * np.linalg.norm(p.vals))
        worst = max(worst, float(np.linalg.norm(x - rec.x_omega) / denom))
        assert info["r"] == rec.r_k, rec.k
    assert info["stopped"]
    assert worst <= 1e-5, worst
    s.close()


def test_allocation_failure_through_allocator_hook(cuda):
    torch = cuda
    from paper_0810_3286_gb300 import Solver, SVTError
    p = config_problem("plain_fp64_200", 1)
    live = {}

    def make_hook(fail_at):
        count = [0]

        def alloc(nbytes):
            count[0] += 1
            if count[0] == fail_at:
                return 0
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes))
            live[ptr] = nbytes
            return ptr

        def free(ptr):
            live.pop(ptr)
            torch.cuda.caching_allocator_delete(ptr)
        return alloc, free, count

    # count the allocations of one context
    alloc, free, count = make_hook(0)
    with Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64", allocator=(alloc, free)) as s:
        res = s.solve(p.tau_default(), p.delta_default(), 1e-4, 27)
        assert res["converged"]
        n_alloc = count[0]
    assert n_alloc > 10 and not live
    for fail_at in sorted({1, 2, n_alloc // 2, n_alloc - 1, n_alloc}):
        alloc, free, _ = make_hook(fail_at)
        with pytest.raises(SVTError) as ei:
            Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64", allocator=(alloc, free))
        assert ei.value.status == 3, (fail_at, ei.value)   # SVT_ERR_OOM
        assert not live, fail_at   # everything the failed create held was handed back
    # the device is still usable: a full solve through the hook
    alloc, free, _ = make_hook(0)
    with Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64", allocator=(alloc, free)) as s:
        assert s.solve(p.tau_default(), p.delta_default(), 1e-4, 27)["converged"]
    assert not live


def test_nan_in_iterate_is_numeric_error_and_nan_input_rejected(cuda):
    torch = cuda
    from paper_0810_3286_gb300 import Solver, SVTError
    p = config_problem("plain_fp64_200", 2)
    s = Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64")
    s.configure(p.tau_default(), p.delta_default(), 1e-4, 27)
    s.step()
    y = s.get_Y()
    y[17] = np.nan
    s.set_Y(y)
    assert _status_of(s.step) == 7   # SVT_ERR_NUMERIC
    s.close()
    bad = p.vals.copy()
    bad[5] = np.inf
    with pytest.raises(SVTError) as ei:
        Solver(p.n1, p.n2, p.rows, p.cols, bad, precision="fp64")
    assert ei.value.status == 1   # SVT_ERR_ARG


def test_rank_limit(cuda):
    torch = cuda
    from paper_0810_3286_gb300 import Solver
    p = config_problem("plain_fp64_200", 0)   # planted rank 5
    with Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64") as s:
        st = _status_of(lambda: s.solve(p.tau_default(), p.delta_default(), 1e-4, 3))
        assert st == 5, st   # SVT_ERR_RANK_LIMIT


def test_not_converged_keeps_last_factors(cuda):
    torch = cuda
    from paper_0810_3286_gb300 import Solver
    p = config_problem("plain_fp64_200", 0)
    with Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64", k_max=7) as s:
        res = s.solve(p.tau_default(), p.delta_default(), 1e-4, 27, raise_on_nonconvergence=False)
        assert not res["converged"] and res["iterations"] == 7
        st = _status_of(lambda: s.solve(p.tau_default(), p.delta_default(), 1e-4, 27))
        assert st == 6, st   # SVT_ERR_NOT_CONVERGED
        U, d, V = s.factors()
        assert U.shape[1] == s.rank() > 0 and np.all(d > 0)
