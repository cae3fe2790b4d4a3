"""Float64 CPU oracle of the SVT iteration (dense tier).  TEST INFRASTRUCTURE ONLY.

Only tests/, the package smoke check and bench.py's CPU-baseline leg use this module.  It shares
no code with the CUDA path.

Everything follows the paper (Cai, Candes, Shen 2008) step by step in float64:

  shrink          D_tau(Y) = U diag((sigma_i - tau)_+) V^T          Sec. 2.1, eq. (2.2)
                  (full SVD by the oracle's own one-sided Jacobi, then the definition)
  kick_k0         k0 with tau / (delta ||P_Omega M||_2) in (k0 - 1, k0]      Sec. 5.1.3, eq. (5.3)
  svt_dantzig     the matrix Dantzig selector iteration (iterDS2) of Sec. 3.3 with two clamped
                  multipliers Y_+, Y_- (linear inequality constraints |B - X| <= E on Omega)
  svt             Algorithm 1 of Sec. 5.1.5: Y^0 = k0 delta P_Omega(M), r_0 = 0, then for
                  k = 1..k_max: the s_k rank policy (Sec. 5.1.1), r_k = #{sigma_j > tau},
                  X^k = sum_{j <= r_k} (sigma_j - tau) u_j v_j^T, stop when
                  ||P_Omega(X^k - M)||_F / ||P_Omega M||_F <= eps (eq. (5.5)), else
                  Y^k = Y^{k-1} + delta P_Omega(M - X^k) (eq. (2.7)).

The dense Y is n1 x n2 with exact zeros off Omega: the iterate is held densely only so that
the SVD can be taken by the definition.  Cost per iteration is one dense Jacobi SVD, so this
tier is meant for n up to a few hundred (seconds) and for bounded timing samples beyond that.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

from ._clib import jacobi_svd


def svd(Y: np.ndarray):
    """Full thin SVD of a dense matrix (one-sided Jacobi), singular values decreasing."""
    return jacobi_svd(Y)


def shrink(Y: np.ndarray, tau: float):
    """D_tau(Y) in factored form (Sec. 2.1, eq. (2.2)).

    Returns (U_r, d, V_r, sigma): U_r n1 x r, d = sigma_1..r - tau > 0, V_r n2 x r, and the full
    list of singular values of Y.  r = #{sigma_i > tau}; D_tau(Y) = U_r diag(d) V_r^T.
    """
    U, s, V = svd(Y)
    r = int(np.count_nonzero(s > tau))
    return U[:, :r], s[:r] - tau, V[:, :r], s


def shrink_dense(Y: np.ndarray, tau: float) -> np.ndarray:
    U, d, V, _ = shrink(Y, tau)
    return (U * d) @ V.T


def dense_from_omega(n1: int, n2: int, rows, cols, vals) -> np.ndarray:
    """P_Omega(Z) as a dense n1 x n2 array: vals at (rows, cols), zero elsewhere."""
    Z = np.zeros((n1, n2))
    Z[np.asarray(rows), np.asarray(cols)] = vals
    return Z


def spectral_norm(n1: int, n2: int, rows, cols, vals) -> float:
    """||P_Omega(M)||_2, the largest singular value of the sampled matrix (Sec. 5.1.3)."""
    _, s, _ = svd(dense_from_omega(n1, n2, rows, cols, vals))
    return float(s[0]) if s.size else 0.0


def kick_k0(tau: float, delta: float, norm2: float) -> int:
    """The integer k0 with tau / (delta * norm2) in (k0 - 1, k0]  (Sec. 5.1.3, eq. (5.3))."""
    return int(math.ceil(tau / (delta * norm2)))


@dataclasses.dataclass
class IterRecord:
    k: int                # iteration index of Algorithm 1 (after the kick)
    s_k: int              # singular triplets computed in the last pass of the rank policy
    passes: int           # passes of the repeat-until loop
    r_k: int              # rank of X^k
    res: float            # ||P_Omega(X^k - M)||_F / ||P_Omega M||_F
    x_omega: np.ndarray   # X^k on Omega (sampled order)
    y_omega: np.ndarray   # Y^{k-1} on Omega (the matrix that was shrunk)
    sigma: np.ndarray     # singular values of Y^{k-1} (first r_k + ell)


@dataclasses.dataclass
class SVTResult:
    iters: int                    # k at exit
    k0: int
    norm2: float
    converged: bool
    U: np.ndarray                 # n1 x r
    d: np.ndarray                 # sigma - tau, length r
    V: np.ndarray                 # n2 x r
    y_omega: np.ndarray           # final Y on Omega (Y^{k-1} if the loop broke at k)
    trace: List[IterRecord]

    @property
    def rank(self) -> int:
        return int(self.d.shape[0])

    def X(self) -> np.ndarray:
        return (self.U * self.d) @ self.V.T


def rank_policy(sigma: np.ndarray, r_prev: int, tau: float, ell: int):
    """The repeat-until loop of Algorithm 1 on a known spectrum (Sec. 5.1.1).

    s_k = r_{k-1} + 1; repeat: compute the first s_k triplets, s_k += ell, until
    sigma_{s_k - ell} <= tau.  When s_k exceeds the number of singular values, every one
    has been computed and the loop ends (the last value counts as <= tau).
    Returns (number of triplets computed in the final pass, number of passes).
    """
    kmax = sigma.shape[0]
    s = r_prev + 1
    passes = 0
    while True:
        passes += 1
        s_eff = min(s, kmax)
        s += ell
        last = sigma[s_eff - 1] if s_eff >= 1 else 0.0
        if s_eff >= kmax or last <= tau:
            return s_eff, passes


@dataclasses.dataclass
class StepResult:
    """One pass of Algorithm 1's loop body (Sec. 5.1.5) from the dual iterate y."""
    s_k: int
    passes: int
    r_k: int
    U: np.ndarray
    d: np.ndarray
    V: np.ndarray
    sigma: np.ndarray       # all singular values of Y, decreasing
    x: np.ndarray           # X^k on Omega
    e: np.ndarray           # M - X^k on Omega
    res: float              # ||P_Omega(X^k - M)||_F / ||P_Omega M||_F  (eq. (5.5))


def svt_step(n1: int, n2: int, rows, cols, m_vals, y, tau: float, r_prev: int, ell: int,
             norm_m: float) -> StepResult:
    """The loop body of Algorithm 1 for the dual iterate y on Omega: the shrink X^k = D_tau(Y^{k-1})
    by the full SVD (eq. (2.2)) with the s_k path of the rank policy (Sec. 5.1.1), X^k on Omega and
    the relative residual of eq. (5.5).  The dual step Y^k = Y^{k-1} + delta P_Omega(M - X^k)
    (eq. (2.7)) is left to the caller, which takes it only when the stopping rule fails."""
    Y = dense_from_omega(n1, n2, rows, cols, y)
    Uf, s, Vf = svd(Y)
    s_k, passes = rank_policy(s, r_prev, tau, ell)
    r_k = int(np.count_nonzero(s > tau))
    U, d, V = Uf[:, :r_k], s[:r_k] - tau, Vf[:, :r_k]
    # X^k on Omega: x_p = sum_j d_j U[i_p, j] V[j_p, j]
    x = np.einsum("pj,j,pj->p", U[rows], d, V[cols]) if r_k > 0 else np.zeros_like(y)
    e = m_vals - x
    res = math.sqrt(float(np.sum(e * e))) / norm_m
    return StepResult(s_k=s_k, passes=passes, r_k=r_k, U=U, d=d, V=V, sigma=s, x=x, e=e, res=res)


def svt(n1: int, n2: int, rows, cols, m_vals, tau: float, delta: float, eps: float = 1e-4,
        ell: int = 5, k_max: int = 1000, k0: Optional[int] = None, kick: bool = True,
        keep_trace: bool = True, max_iters: Optional[int] = None, noise_sigma: float = 0.0,
        noise_eps: float = 0.0) -> SVTResult:
    """Algorithm 1 (Sec. 5.1.5) in float64 on a dense copy of the iterate.

    kick=False starts from Y^0 = 0 (eq. (2.7) without the kicking device); kick=True uses
    Y^0 = k0 delta P_Omega(M) with k0 from eq. (5.3) unless k0 is given.
    max_iters stops early (a bounded sample for timing); the result is then not converged.
    noise_sigma > 0: the values are noisy observations B (eq. (5.9)) and the loop stops at the
    first X^k with ||P_Omega(X^k - B)||_F^2 <= (1 + noise_eps) m sigma^2 (eq. (5.10), m = |Omega|)
    instead of the relative-residual rule eq. (5.5).
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    m_vals = np.asarray(m_vals, dtype=np.float64)
    norm_m = math.sqrt(float(np.sum(m_vals * m_vals)))
    norm2 = spectral_norm(n1, n2, rows, cols, m_vals)
    if kick:
        if k0 is None:
            k0 = kick_k0(tau, delta, norm2)
        y = k0 * delta * m_vals
    else:
        k0 = 0
        y = np.zeros_like(m_vals)
    r_prev = 0
    trace: List[IterRecord] = []
    converged = False
    U = np.zeros((n1, 0)); d = np.zeros(0); V = np.zeros((n2, 0))
    k = 0
    limit = k_max if max_iters is None else min(k_max, max_iters)
    for k in range(1, limit + 1):
        st = svt_step(n1, n2, rows, cols, m_vals, y, tau, r_prev, ell, norm_m)
        U, d, V = st.U, st.d, st.V
        if keep_trace:
            trace.append(IterRecord(k=k, s_k=st.s_k, passes=st.passes, r_k=st.r_k, res=st.res,
                                    x_omega=st.x.copy(), y_omega=y.copy(), sigma=st.sigma[:st.r_k + ell].copy()))
        r_prev = st.r_k
        if noise_sigma > 0.0:
            stop = float(np.sum(st.e * st.e)) <= (1.0 + noise_eps) * len(m_vals) * noise_sigma ** 2
        else:
            stop = st.res <= eps
        if stop:
            converged = True
            break
        y = y + delta * st.e
    return SVTResult(iters=k, k0=k0, norm2=norm2, converged=converged, U=U, d=d, V=V, y_omega=y, trace=trace)


def soft_values(vals, E: float):
    """Entrywise soft threshold sign(b) (|b| - E)_+ of the sampled values."""
    vals = np.asarray(vals, dtype=np.float64)
    return np.sign(vals) * np.maximum(np.abs(vals) - E, 0.0)


@dataclasses.dataclass
class DSResult:
    iters: int
    k0: int
    converged: bool
    U: np.ndarray
    d: np.ndarray
    V: np.ndarray
    yp: np.ndarray
    ym: np.ndarray
    trace: List[IterRecord]


def svt_dantzig(n1: int, n2: int, rows, cols, b_vals, E: float, tau: float, delta: float, eps: float = 1e-4,
                ell: int = 5, k_max: int = 1000, k0: Optional[int] = None, kick: bool = True,
                keep_trace: bool = True) -> DSResult:
    """SVT for the matrix Dantzig selector (Sec. 3.3, problem (DS)) in matrix completion form,
    iteration (iterDS2): with Y_+, Y_- >= 0 the multipliers of B - X <= E and X - B <= E on Omega,
        X^k = D_tau(Y_+^{k-1} - Y_-^{k-1}),
        Y_+^k = [Y_+^{k-1} + delta P_Omega( (B - X^k) - E)]_+,
        Y_-^k = [Y_-^{k-1} + delta P_Omega(-(B - X^k) - E)]_+,
    from Y_+^0 = Y_-^0 = 0, in float64 on dense copies (E constant over Omega).

    Kick (the device of Sec. 5.1.3 carried over): while X^k = 0 the updates give
    Y_+^k = k delta [B - E]_+ and Y_-^k = k delta [-B - E]_+ exactly, so Y_+ - Y_- = k delta soft_E(B);
    with kick=True the loop starts after k0 such steps, k0 from eq. (5.3) with ||P_Omega soft_E(B)||_2.
    Stop: the relative constraint violation ||[|B - X^k| - E]_+||_F / ||P_Omega B||_F <= eps (the
    analogue of eq. (5.5): zero exactly when X^k is feasible); the multipliers are then left at
    step k - 1 as in Algorithm 1.  IterRecord.res holds that violation.
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    b = np.asarray(b_vals, dtype=np.float64)
    norm_b = math.sqrt(float(np.sum(b * b)))
    soft = soft_values(b, E)
    if kick:
        if k0 is None:
            k0 = kick_k0(tau, delta, spectral_norm(n1, n2, rows, cols, soft))
        yp = k0 * delta * np.maximum(b - E, 0.0)
        ym = k0 * delta * np.maximum(-b - E, 0.0)
    else:
        k0 = 0
        yp = np.zeros_like(b)
        ym = np.zeros_like(b)
    r_prev = 0
    trace: List[IterRecord] = []
    converged = False
    U = np.zeros((n1, 0)); d = np.zeros(0); V = np.zeros((n2, 0))
    k = 0
    for k in range(1, k_max + 1):
        y = yp - ym
        Y = dense_from_omega(n1, n2, rows, cols, y)
        Uf, s, Vf = svd(Y)
        s_k, passes = rank_policy(s, r_prev, tau, ell)
        r_k = int(np.count_nonzero(s > tau))
        U, d, V = Uf[:, :r_k], s[:r_k] - tau, Vf[:, :r_k]
        x = np.einsum("pj,j,pj->p", U[rows], d, V[cols]) if r_k > 0 else np.zeros_like(b)
        e = b - x
        viol = np.maximum(np.abs(e) - E, 0.0)
        res = math.sqrt(float(np.sum(viol * viol))) / norm_b
        if keep_trace:
            trace.append(IterRecord(k=k, s_k=s_k, passes=passes, r_k=r_k, res=res, x_omega=x.copy(),
                                    y_omega=y.copy(), sigma=s[:r_k + ell].copy()))
        r_prev = r_k
        if res <= eps:
            converged = True
            break
        yp = np.maximum(yp + delta * (e - E), 0.0)
        ym = np.maximum(ym + delta * (-e - E), 0.0)
    return DSResult(iters=k, k0=k0, converged=converged, U=U, d=d, V=V, yp=yp, ym=ym, trace=trace)


def relative_error(U: np.ndarray, d: np.ndarray, V: np.ndarray, A: np.ndarray, B: np.ndarray) -> float:
    """||X - M||_F / ||M||_F with X = U diag(d) V^T, M = A B^T, formed densely (Sec. 5.2.1, eq. (5.8))."""
    X = (U * d) @ V.T
    M = A @ B.T
    return float(np.linalg.norm(X - M) / np.linalg.norm(M))
