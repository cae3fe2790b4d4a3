"""GPU parity of the shrink and of Algorithm 1 against the float64 oracle.

* svt_shrink vs D_tau of eq. (2.2): singular values above tau and X on Omega.
* Per-iterate parity (Algorithm 1, Sec. 5.1.5) of the float64 path on the 200 x 200 rank-5
  workload and on a ragged rectangular case: r_k identical, X^k on Omega within 1e-5 relative
  Frobenius error, same k0, same iteration count.
* The float32 (mixed) path: per-iterate error <= 1e-3 and the same stopping iteration +- 2.
* Recovery ||X - M||_F / ||M||_F agrees with the oracle to within 1e-3.
* Checkpoint / resume reproduces later iterates bit for bit.
"""
import numpy as np
import pytest

from oracle import svt as osvt
from oracle.sparse import sample_X
from svt_inputs import config_problem, planted_problem

pytestmark = pytest.mark.gpu


def _per_iterate_error(x, x_ref, m_vals):
    """||x - x_ref|| / max(||x_ref||, 1e-2 ||P_Omega M||) (the guarded relative error on Omega)."""
    return float(np.linalg.norm(x - x_ref) / max(np.linalg.norm(x_ref), 1e-2 * np.linalg.norm(m_vals)))


def _x_on_omega(s, p):
    U, d, V = s.factors()
    return sample_X(p.rows, p.cols, U * d, V)


@pytest.mark.parametrize("precision,lanczos_tol,tol,xtol", [("fp64", 0.0, 1e-9, 1e-5), ("fp64", 1e-9, 1e-9, 1e-8),
                                                           ("fp32", 0.0, 1e-4, 1e-3)])
def test_shrink_matches_definition(cuda, precision, lanczos_tol, tol, xtol):
    """svt_shrink against D_tau of eq. (2.2) computed from a full SVD: the singular values above tau
    to `tol` sigma_1 (Ritz values converge to second order in the residual) and X on Omega to xtol,
    the Ritz-vector accuracy the Lanczos tolerance allows (float64 default 1e-6: X within the
    per-iterate bound 1e-5; with lanczos_tol = 1e-9: within 1e-8; float32 default 1e-4: within
    the mixed path's 1e-3)."""
    from paper_0810_3286_gb300 import Solver
    p = planted_problem(150, 110, 4, 4000, seed=2)
    tau = p.tau_default()
    # a dual iterate with its leading singular value at 1.6 tau: Y = c P_Omega(M)
    norm2 = osvt.spectral_norm(p.n1, p.n2, p.rows, p.cols, p.vals)
    y = 1.6 * tau / norm2 * p.vals
    s = Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision=precision, lanczos_tol=lanczos_tol)
    s.set_Y(y)
    r, sig = s.shrink(tau)
    U0, d0, V0, s_all = osvt.shrink(osvt.dense_from_omega(p.n1, p.n2, p.rows, p.cols, y), tau)
    assert r == d0.size and r >= 1
    assert np.abs(sig - (d0 + tau)).max() <= tol * s_all[0]
    x = _x_on_omega(s, p)
    x_ref = sample_X(p.rows, p.cols, U0 * d0, V0)
    err = _per_iterate_error(x, x_ref, p.vals)
    print("shrink %s lanczos_tol %g: X error %.2e" % (precision, lanczos_tol, err))
    assert err <= xtol, err
    s.close()


def _run_parity(p, precision, k0, trace, tau, delta, **solver_kw):
    from paper_0810_3286_gb300 import Solver
    s = Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision=precision, **solver_kw)
    s.configure(tau, delta, 1e-4, 27, k0)
    errs, ranks, stopped_at = [], [], None
    for rec in trace:
        info = s.step()
        x = _x_on_omega(s, p)
        errs.append(_per_iterate_error(x, rec.x_omega, p.vals))
        ranks.append((info["r"], rec.r_k))
        if info["stopped"]:
            stopped_at = info["k"]
            break
    # the GPU run may need a couple more iterations than the oracle in the mixed path
    extra = 0
    while stopped_at is None and extra < 10:
        info = s.step()
        extra += 1
        if info["stopped"]:
            stopped_at = info["k"]
    return s, errs, ranks, stopped_at


def test_parity_fp64_plain_200(cuda, oracle_c1_run):
    p, ref = oracle_c1_run
    tau, delta = p.tau_default(), p.delta_default()
    s, errs, ranks, stopped_at = _run_parity(p, "fp64", ref.k0, ref.trace, tau, delta)
    assert max(errs) <= 1e-5, (np.argmax(errs), max(errs))
    assert all(a == b for a, b in ranks)
    assert stopped_at == ref.iters
    U, d, V = s.factors()
    err_gpu = osvt.relative_error(U, d, V, p.A, p.B)
    err_ref = osvt.relative_error(ref.U, ref.d, ref.V, p.A, p.B)
    assert abs(err_gpu - err_ref) <= 1e-3
    # ||X_gpu - X_oracle||_F / ||X_oracle||_F from the factors
    Xg = (U * d) @ V.T
    assert np.linalg.norm(Xg - ref.X()) / np.linalg.norm(ref.X()) <= 1e-3
    s.close()


def test_parity_fp64_ragged_rectangular(cuda):
    p = planted_problem(173, 131, 3, 3 * 5 * (173 + 131 - 3), seed=12)
    tau, delta = p.tau_default(), p.delta_default()
    ref = osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, tau, delta, k_max=40, eps=1e-4)
    s, errs, ranks, _ = _run_parity(p, "fp64", ref.k0, ref.trace, tau, delta)
    assert max(errs) <= 1e-5
    assert all(a == b for a, b in ranks)
    s.close()


@pytest.mark.parametrize("variant", [{"fused_orth": False}, {"use_graphs": False}, {"orth_grid": 8},
                                     {"device_loop": False}, {"orth_tf32": True}, {"jacobi_cluster": 1}])
def test_parity_fp64_other_launch_paths(cuda, variant):
    """The eight-kernel orthonormalisation (fused_orth = 0, the path taken without cooperative
    launches), kernel-by-kernel launches without CUDA graphs, a small cooperative grid, the shrink
    decided on the host after every Lanczos cycle (device_loop = 0), the first Gram-Schmidt pass
    on the tensor cores (orth_tf32, off by default in float64), and the projected SVD in one CTA
    (jacobi_cluster = 1, the form taken where a cluster launch is not possible) give the same
    iterates as the oracle."""
    p = planted_problem(173, 131, 3, 3 * 5 * (173 + 131 - 3), seed=12)
    tau, delta = p.tau_default(), p.delta_default()
    ref = osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, tau, delta, k_max=25, eps=1e-4)
    s, errs, ranks, _ = _run_parity(p, "fp64", ref.k0, ref.trace, tau, delta, **variant)
    assert max(errs) <= 1e-5, (variant, max(errs))
    assert all(a == b for a, b in ranks)
    s.close()


def test_parity_fp32_plain_200(cuda, oracle_c1_run):
    p, ref = oracle_c1_run
    tau, delta = p.tau_default(), p.delta_default()
    s, errs, ranks, stopped_at = _run_parity(p, "fp32", ref.k0, ref.trace, tau, delta)
    assert max(errs) <= 1e-3, max(errs)
    assert stopped_at is not None and abs(stopped_at - ref.iters) <= 2
    U, d, V = s.factors()
    assert abs(osvt.relative_error(U, d, V, p.A, p.B) - osvt.relative_error(ref.U, ref.d, ref.V, p.A, p.B)) <= 1e-3
    s.close()


def test_solve_kick_matches_oracle(cuda, oracle_c1_run):
    """svt_solve computes ||P_Omega M||_2 and k0 itself (eq. (5.3)); both match the oracle."""
    from paper_0810_3286_gb300 import Solver
    p, ref = oracle_c1_run
    s = Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64")
    res = s.solve(p.tau_default(), p.delta_default(), 1e-4, 27)
    assert res["k0"] == ref.k0
    assert abs(res["norm2_M"] - ref.norm2) <= 1e-10 * ref.norm2
    assert res["converged"] == 1 and res["iterations"] == ref.iters and res["rank"] == p.r
    s.close()


def test_checkpoint_resume_bit_identical(cuda):
    from paper_0810_3286_gb300 import Solver
    p = planted_problem(120, 100, 3, 3000, seed=21)
    a = Solver(p.n1, p.n2, p.rows, p.cols, p.vals)
    a.configure(p.tau_default(), p.delta_default(), 1e-4, 27)
    for _ in range(6):
        a.step()
    blob = a.save_state()
    cont = [a.step()["residual"] for _ in range(5)]
    Ua, da, Va = a.factors()
    b = Solver(p.n1, p.n2, p.rows, p.cols, p.vals)
    b.load_state(blob)
    resumed = [b.step()["residual"] for _ in range(5)]
    Ub, db, Vb = b.factors()
    assert cont == resumed
    assert np.array_equal(da, db) and np.array_equal(Ua, Ub) and np.array_equal(Va, Vb)
    a.close()
    b.close()


def test_recovery_single_1000_fp32(cuda):
    """1000 x 1000, rank 10, |Omega| = 6 d_r (Table 1, first row): the stopping rule is met and the
    relative error is below the 2e-4 the paper reports for all its Table 1 runs; the iteration
    count is within the range of Table 1's rank-10 rows (117-125, +-15%)."""
    from paper_0810_3286_gb300 import Solver
    p = config_problem("single_1000", 0)
    s = Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp32")
    res = s.solve(p.tau_default(), p.delta_default(), 1e-4, 27)
    assert res["converged"] == 1 and res["rank"] == 10
    U, d, V = s.factors()
    # closed form of ||X - M||_F with X = U diag(d) V^T and M = A B^T
    A, B = p.A, p.B
    nx2 = float(np.sum(d * d))
    nm2 = float(np.trace((A.T @ A) @ (B.T @ B)))
    xm = float(np.trace(np.diag(d) @ (U.T @ A) @ (B.T @ V)))
    relerr = np.sqrt(max(nx2 - 2 * xm + nm2, 0.0) / nm2)
    assert relerr < 2e-4
    assert 0.85 * 117 <= res["iterations"] <= 1.15 * 125
    s.close()


def test_iterations_run_as_device_controlled_graphs(cuda, oracle_c1_run):
    """With svt_options.device_loop (the default) every SVT iteration is one graph launch: the
    Lanczos cycles repeat under a conditional `while` node whose condition the device sets from
    the convergence test, the rank r_k is read on the device, and the host synchronises once per
    iteration.  The counter of such iterations equals the iteration count (no iteration fell back
    to the host loop here), and the solve reproduces the oracle's iteration count, k0 and rank."""
    from paper_0810_3286_gb300 import Solver
    p, ref = oracle_c1_run
    with Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp64") as s:
        res = s.solve(p.tau_default(), p.delta_default(), 1e-4, 27)
        cnt = s.counters()
        assert res["converged"] and res["iterations"] == ref.iters and res["k0"] == ref.k0
        assert res["rank"] == ref.d.shape[0]
        assert cnt["device_loop_iterations"] >= ref.iters - 2, cnt
