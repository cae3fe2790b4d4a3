"""Pins of the oracle's SVT iteration (Algorithm 1, Sec. 5.1.5) against what the paper fixes.

* Full Omega (P_Omega = I, p = 1): every iterate is U diag(y) V^T with the scalar recurrence
  y_i <- y_i + delta (sigma_i - (y_i - tau)_+) from y = k0 delta sigma (eq. (2.7) with eq. (2.2));
  this fixes X^k, r_k and the residual of every iterate and the iteration count.
* Kicking device (Sec. 5.1.3): from Y^0 = 0, X^k = 0 and Y^k = k delta P_Omega M for k <= k0, and
  the un-kicked run continues exactly as the kicked one.
* k0 definition, eq. (5.3), including the integer boundary.
* Rank policy of Sec. 5.1.1 on known spectra.
* Theorem 4.2: ||P_Omega(Y^k - Y*)||_F is nonincreasing for 0 < delta < 2, and the limit satisfies
  the KKT system (5.4) and minimises tau||X||_* + 1/2||X||_F^2 on the feasible set (eq. (2.8)).
* Sparsity (Sec. 2.2): Y^k is supported on Omega.
"""
import math

import numpy as np
import pytest

from oracle import svt as osvt
from oracle.sparse import sample_X


def _full_omega_problem(n1, n2, sigma, seed):
    rng = np.random.default_rng(seed)
    Qu, _ = np.linalg.qr(rng.standard_normal((n1, len(sigma))))
    Qv, _ = np.linalg.qr(rng.standard_normal((n2, len(sigma))))
    M = (Qu * sigma) @ Qv.T
    rows, cols = np.divmod(np.arange(n1 * n2), n2)
    return Qu, Qv, M, rows.astype(np.int32), cols.astype(np.int32), M.ravel().copy()


@pytest.mark.parametrize("n1,n2,sigma,tau,seed", [
    (8, 8, [9.0, 6.0, 4.0], 5.0, 0),
    (9, 7, [20.0, 3.1, 1.3, 0.7], 12.5, 1),
    (6, 10, [7.0, 6.5], 40.0, 2),
])
def test_full_omega_closed_form(n1, n2, sigma, tau, seed):
    sigma = np.array(sigma)
    Qu, Qv, M, rows, cols, vals = _full_omega_problem(n1, n2, sigma, seed)
    delta = 1.2 * n1 * n2 / (n1 * n2)          # eq. (5.1) with p = 1
    eps = 1e-4
    res = osvt.svt(n1, n2, rows, cols, vals, tau, delta, eps=eps, k_max=500)
    # Scalar recurrence.
    k0 = math.ceil(tau / (delta * sigma.max()))
    assert res.k0 == k0
    y = k0 * delta * sigma
    normM = np.linalg.norm(sigma)
    expected = []
    for k in range(1, 501):
        xs = np.maximum(y - tau, 0.0)
        assert np.all(np.abs(y - tau) > 1e-8 * tau)   # no tie sigma_i(Y) = tau on this path
        rk = int(np.count_nonzero(y > tau))
        r = np.linalg.norm(xs - sigma) / normM
        expected.append((rk, r, xs.copy()))
        if r <= eps:
            break
        y = y + delta * (sigma - xs)
    assert res.iters == len(expected)
    assert res.converged
    for rec, (rk, r, xs) in zip(res.trace, expected):
        assert rec.r_k == rk
        assert rec.res == pytest.approx(r, rel=1e-9, abs=1e-12)
        X_expected = (Qu * xs) @ Qv.T
        assert np.abs(rec.x_omega - X_expected.ravel()).max() <= 1e-11 * sigma.max()


def test_full_omega_planted_sign_error_is_caught():
    """Planting a sign error in the dual update (Y - delta(M - X)) breaks the closed form."""
    sigma = np.array([9.0, 6.0, 4.0])
    Qu, Qv, M, rows, cols, vals = _full_omega_problem(8, 8, sigma, 0)
    good = osvt.svt(8, 8, rows, cols, vals, 5.0, 1.2, k_max=30, eps=0.0)
    bad = osvt.svt(8, 8, rows, cols, -vals, 5.0, 1.2, k_max=30, eps=0.0)
    # with the sign flipped the iterates cannot follow the recurrence driven by +M
    assert np.abs(good.trace[-1].x_omega - bad.trace[-1].x_omega).max() > 1.0


@pytest.mark.parametrize("tau,delta,norm2,k0", [(10.0, 1.0, 3.0, 4), (9.0, 1.0, 3.0, 3), (1.0, 2.0, 5.0, 1),
                                                 (5000.0, 10.05, 80.0, 7)])
def test_k0_definition(tau, delta, norm2, k0):
    got = osvt.kick_k0(tau, delta, norm2)
    assert got == k0
    ratio = tau / (delta * norm2)
    assert got - 1 < ratio <= got


def test_kick_identity():
    from svt_inputs import planted_problem
    p = planted_problem(30, 24, 2, 400, seed=3)
    tau, delta = p.tau_default(), p.delta_default()
    kicked = osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, tau, delta, k_max=25, eps=0.0)
    plain = osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, tau, delta, k_max=25 + kicked.k0, eps=0.0, kick=False)
    k0 = kicked.k0
    assert k0 >= 2
    for k in range(1, k0 + 1):
        rec = plain.trace[k - 1]
        assert rec.r_k == 0 and np.all(rec.x_omega == 0.0)
        # Y^{k-1} = (k-1) delta P_Omega M
        assert np.abs(rec.y_omega - (k - 1) * delta * p.vals).max() <= 1e-12 * np.abs(p.vals).max() * k
    for j in range(len(kicked.trace)):
        a, b = kicked.trace[j], plain.trace[k0 + j]
        assert a.r_k == b.r_k
        assert np.abs(a.x_omega - b.x_omega).max() <= 1e-9 * np.abs(p.vals).max()


def test_rank_policy_known_spectra():
    s = np.array([10.0, 9.0, 8.0, 7.0, 6.0, 5.0, 4.0, 3.0, 2.0, 1.0, 0.5, 0.1])
    # s_1 = 10 > tau: s becomes 6, s_6 = 5 <= tau=5.5: two passes, 6 triplets
    assert osvt.rank_policy(s, 0, 5.5, 5) == (6, 2)
    # r_prev = 5: s = 6, s_6 = 5 <= 5.5: one pass
    assert osvt.rank_policy(s, 5, 5.5, 5) == (6, 1)
    # tau below everything: 1, 6, 11 (s_11 = 0.5 > 0.05), 16 -> capped at 12 (all computed)
    assert osvt.rank_policy(s, 0, 0.05, 5) == (12, 4)
    # tau above everything
    assert osvt.rank_policy(s, 3, 100.0, 5) == (4, 1)


def test_theorem_4_2_monotone_and_kkt():
    from svt_inputs import planted_problem
    p = planted_problem(7, 6, 1, 26, seed=11)
    tau = 2.0 * p.tau_default()
    delta = 1.5                                   # 0 < delta < 2 (Theorem 4.2)
    res = osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, tau, delta, eps=1e-13, k_max=20000)
    assert res.converged
    y_star = res.trace[-1].y_omega
    dist = [np.linalg.norm(rec.y_omega - y_star) for rec in res.trace]
    assert all(dist[i + 1] <= dist[i] * (1 + 1e-9) + 1e-12 for i in range(len(dist) - 1))
    # KKT (5.4): X = D_tau(Y) with Y supported on Omega, and P_Omega(X - M) = 0.
    Y = osvt.dense_from_omega(p.n1, p.n2, p.rows, p.cols, res.trace[-1].y_omega)
    X = res.X()
    assert np.abs(X - osvt.shrink_dense(Y, tau)).max() <= 1e-10 * np.abs(Y).max()
    x_omega = X[p.rows, p.cols]
    assert np.linalg.norm(x_omega - p.vals) <= 1e-12 * np.linalg.norm(p.vals)
    # eq. (2.8): X minimises f(X) = tau||X||_* + 1/2||X||_F^2 among matrices equal to M on Omega.
    f = lambda Z: tau * np.linalg.svd(Z, compute_uv=False).sum() + 0.5 * np.sum(Z * Z)
    rng = np.random.default_rng(0)
    mask = np.zeros((p.n1, p.n2), bool)
    mask[p.rows, p.cols] = True
    base = f(X)
    for _ in range(50):
        Z = rng.standard_normal(X.shape) * ~mask
        for t in (1e-4, 1e-2, 1.0):
            assert f(X + t * Z) >= base - 1e-9 * abs(base)


def test_sparsity_of_iterates():
    from svt_inputs import planted_problem
    p = planted_problem(20, 15, 2, 150, seed=4)
    res = osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, p.tau_default(), p.delta_default(), k_max=10, eps=0.0)
    mask = np.zeros((p.n1, p.n2), bool)
    mask[p.rows, p.cols] = True
    for rec in res.trace:
        Y = osvt.dense_from_omega(p.n1, p.n2, p.rows, p.cols, rec.y_omega)
        assert np.all(Y[~mask] == 0.0)
    # X on Omega from the factors equals the dense product sampled on Omega
    X = res.X()
    assert np.abs(sample_X(p.rows, p.cols, res.U * res.d, res.V) - X[p.rows, p.cols]).max() <= 1e-10


def test_recovery_plain_fp64_200(oracle_c1_run):
    """200 x 200, rank 5, |Omega| = 6 d_r: converges to the stopping rule (eq. (5.5)) with a
    relative error of the order of the residual.  No paper number exists for this size, so
    only the qualitative statement of Sec. 5.2.1 (error ~ 1e-4, fewer than 200 iterations) is
    checked here."""
    p, res = oracle_c1_run
    assert res.converged and res.trace[-1].res <= 1e-4
    assert res.rank == p.r
    assert res.iters < 200
    assert osvt.relative_error(res.U, res.d, res.V, p.A, p.B) < 1e-3
    ranks = [rec.r_k for rec in res.trace]
    assert max(ranks) == p.r and ranks[-1] == p.r


@pytest.mark.parametrize("eps_noise", [0.0, 0.1])
def test_noisy_stop_full_omega_closed_form(eps_noise):
    """Noisy data, eq. (5.9)-(5.10), with Omega = all entries: B = M + Z has the SVD
    U_B diag(sigma_B) V_B^T, every iterate is U_B diag(y) V_B^T with the scalar recurrence on all
    singular values of B, ||X^k - B||_F^2 = sum_i (sigma_B,i - (y_i - tau)_+)^2, and the loop stops
    at the first k with that below (1 + eps) m sigma^2."""
    n1, n2, noise = 9, 8, 0.4
    sigma = np.array([14.0, 9.0, 6.0])
    Qu, Qv, M, rows, cols, _ = _full_omega_problem(n1, n2, sigma, 3)
    rng = np.random.default_rng(11)
    B = M + noise * rng.standard_normal(M.shape)
    UB, sB, VBt = np.linalg.svd(B, full_matrices=False)
    tau, delta = 5.0, 1.2
    res = osvt.svt(n1, n2, rows, cols, B.ravel().copy(), tau, delta, k_max=500, noise_sigma=noise,
                   noise_eps=eps_noise)
    y = math.ceil(tau / (delta * sB[0])) * delta * sB
    thr = (1.0 + eps_noise) * n1 * n2 * noise ** 2
    for k in range(1, 501):
        xs = np.maximum(y - tau, 0.0)
        assert np.all(np.abs(y - tau) > 1e-8 * tau)
        if float(np.sum((sB - xs) ** 2)) <= thr:
            break
        y = y + delta * (sB - xs)
    assert res.converged and res.iters == k
    X_expected = (UB * xs) @ VBt
    assert np.abs(res.trace[-1].x_omega - X_expected.ravel()).max() <= 1e-10 * sB[0]
    # the previous iterate was not yet consistent with the data
    assert np.sum((res.trace[-2].x_omega - B.ravel()) ** 2) > thr


@pytest.mark.parametrize("ratio", [1e-2, 1e-1])
def test_noisy_recovery_error_about_noise_ratio(ratio):
    """Sec. 5.2.1 (Table 2 and the heuristic after it): with the early stop eq. (5.10), the relative
    reconstruction error is about the noise ratio ||P_Omega Z||_F / ||P_Omega M||_F (Table 2:
    0.72 - 0.78 times it for rank 10)."""
    from svt_inputs import config_problem
    p0 = config_problem("plain_fp64_200", 0)
    sig = ratio * np.linalg.norm(p0.vals) / math.sqrt(p0.nnz)
    p = config_problem("plain_fp64_200", 0, noise_sigma=sig)
    res = osvt.svt(p.n1, p.n2, p.rows, p.cols, p.vals, p.tau_default(), p.delta_default(), noise_sigma=sig,
                   keep_trace=False)
    assert res.converged
    err = osvt.relative_error(res.U, res.d, res.V, p.A, p.B)
    nr = np.linalg.norm(p.vals - p0.vals) / np.linalg.norm(p0.vals)
    assert 0.4 * nr <= err <= 1.2 * nr, (err, nr)


def _ds_problem(n1, n2, r, m, seed, noise):
    from svt_inputs import planted_problem
    return planted_problem(n1, n2, r, m, seed, noise_sigma=noise)


def test_dantzig_kick_identity():
    """Un-kicked Dantzig iteration from Y_+ = Y_- = 0: X^k = 0 and Y_+ - Y_- = k delta soft_E(B) for
    k <= k0, after which it continues exactly as the kicked run."""
    p = _ds_problem(20, 16, 2, 180, 4, 0.3)
    E = 0.2
    tau, delta = p.tau_default(), p.delta_default()
    kicked = osvt.svt_dantzig(p.n1, p.n2, p.rows, p.cols, p.vals, E, tau, delta, eps=1e-3, k_max=60)
    k0 = kicked.k0
    assert k0 >= 2
    plain = osvt.svt_dantzig(p.n1, p.n2, p.rows, p.cols, p.vals, E, tau, delta, eps=1e-3, k_max=60 + k0, kick=False)
    soft = osvt.soft_values(p.vals, E)
    for k in range(k0 - 1):     # iterates 1 .. k0-1 see Y = k delta soft(B) with ||.||_2 <= tau
        rec = plain.trace[k]
        assert rec.r_k == 0
        assert np.allclose(rec.y_omega, k * delta * soft, rtol=0, atol=1e-12 * np.abs(soft).max() * k0 * delta)
    for a, b in zip(kicked.trace, plain.trace[k0:]):
        assert a.r_k == b.r_k
        assert np.abs(a.x_omega - b.x_omega).max() <= 1e-9 * max(1.0, np.abs(a.x_omega).max())


def test_dantzig_limit_satisfies_kkt():
    """The limit of the Dantzig iteration solves min tau||X||_* + 1/2||X||_F^2 s.t. |B - X| <= E on
    Omega: feasibility, multipliers Y_+, Y_- >= 0 with complementary slackness (Y_+ > 0 only where
    B - X = E, Y_- > 0 only where X - B = E) and stationarity X = D_tau(Y_+ - Y_-)."""
    p = _ds_problem(8, 7, 2, 40, 7, 0.5)
    E = 0.3
    tau = 2.0
    res = osvt.svt_dantzig(p.n1, p.n2, p.rows, p.cols, p.vals, E, tau, 0.9, eps=1e-11, k_max=20000,
                           keep_trace=True)
    assert res.converged
    x = res.trace[-1].x_omega
    b = p.vals
    scale = np.abs(b).max()
    assert np.all(np.abs(b - x) <= E + 1e-9 * scale)
    assert np.all(res.yp >= 0) and np.all(res.ym >= 0)
    ymax = max(res.yp.max(), res.ym.max(), 1.0)
    act_p = res.yp > 1e-6 * ymax
    act_m = res.ym > 1e-6 * ymax
    assert np.all(np.abs((b - x)[act_p] - E) <= 1e-6 * scale)
    assert np.all(np.abs((x - b)[act_m] - E) <= 1e-6 * scale)
    # stationarity: X = D_tau(Y_+ - Y_-) (the multipliers of the last step)
    U, d, V, _ = osvt.shrink(osvt.dense_from_omega(p.n1, p.n2, p.rows, p.cols, res.yp - res.ym), tau)
    x_st = sample_X(p.rows, p.cols, U * d, V)
    assert np.abs(x_st - x).max() <= 1e-6 * scale
