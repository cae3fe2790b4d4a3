"""The alternative ways of running the SVT iteration proposed in Sec. 6, on the GPU through the
C-ABI, against the float64 oracle (oracle/alt_shrink.py) iterate by iterate.

* Randomized shrink engine (svt_options.shrink_engine = SVT_SHRINK_RANDOMIZED): the same test
  columns on both sides (the previous shrink's right vectors, then SplitMix64 columns defined by
  the seed rule in include/svt.h), so both compute D_tau(Q Q^T Y) for the same range; float64: X on
  Omega within 1e-5 per iterate and identical ranks and stopping iteration; float32 values: within
  1e-3 per iterate.
* Continuation (svt_solve_continuation, svt_set_tau): tau_0 = tau / 2 < tau_1 = tau with the kick at
  tau_0, each stage from the previous stage's dual iterate, against the oracle's continuation:
  the same iterations per stage, X on Omega within 1e-5 every iterate (float64).
"""
import numpy as np
import pytest

from oracle import alt_shrink
from oracle.sparse import sample_X
from svt_inputs import config_problem

pytestmark = pytest.mark.gpu


def _err(x, ref, vals):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-2 * np.linalg.norm(vals)))


@pytest.mark.parametrize("prec,bound", [("fp64", 1e-5), ("fp32", 1e-3)])
def test_randomized_engine_per_iterate(cuda, prec, bound):
    from paper_0810_3286_gb300 import Solver
    p = config_problem("plain_fp64_200", 0)
    tau, delta = p.tau_default(), p.delta_default()
    ref = alt_shrink.svt_randomized(p.n1, p.n2, p.rows, p.cols, p.vals, tau, delta, k_max=400, oversample=8,
                                    power=1, base_seed=12345)
    assert ref.converged
    with Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision=prec, shrink_engine="randomized",
                rsvd_oversample=8, rsvd_power=1, rsvd_seed=12345) as s:
        s.configure(tau, delta, 1e-4, 27, ref.k0)
        worst = 0.0
        for rec in ref.trace:
            info = s.step()
            U, d, V = s.factors()
            worst = max(worst, _err(sample_X(p.rows, p.cols, U * d, V), rec.x_omega, p.vals))
            assert info["r"] == rec.r_k, (rec.k, info["r"], rec.r_k)
            if prec == "fp64":
                assert info["s"] == rec.s_k and info["passes"] == rec.passes, rec.k
        if prec == "fp64":
            assert info["stopped"]
    print("randomized engine %s: %d iterations, worst per-iterate error %.2e" % (prec, len(ref.trace), worst))
    assert worst <= bound, worst


def test_continuation_per_iterate_fp64(cuda):
    from paper_0810_3286_gb300 import Solver
    p = config_problem("plain_fp64_200", 1)
    tau, delta = p.tau_default(), p.delta_default()
    taus = [tau / 2, tau]
    ref = alt_shrink.svt_continuation(p.n1, p.n2, p.rows, p.cols, p.vals, taus, delta, k_max=400)
    assert ref.converged
    with Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64") as s:
        # stage by stage through svt_configure / svt_step / svt_set_tau
        s.configure(taus[0], delta, 1e-4, 27, ref.k0)
        worst, k, stages = 0.0, 0, []
        for i, t in enumerate(taus):
            if i > 0:
                s.set_tau(t)
            n = 0
            while True:
                info = s.step()
                rec = ref.trace[k]
                k += 1
                n += 1
                U, d, V = s.factors()
                worst = max(worst, _err(sample_X(p.rows, p.cols, U * d, V), rec.x_omega, p.vals))
                assert info["r"] == rec.r_k, (k, info["r"], rec.r_k)
                if info["stopped"]:
                    break
            stages.append(n)
        assert stages == ref.stage_iters, (stages, ref.stage_iters)
        assert worst <= 1e-5, worst
        # the native loop gives the same stages
        res, st = s.solve_continuation(taus, delta, 1e-4, 27)
        assert st == ref.stage_iters and res["converged"] == 1 and res["iterations"] == sum(st)
    print("continuation: stages %s, worst per-iterate error %.2e" % (stages, worst))
