"""Float64 CPU oracle of the SVT iteration, sparse tier (tier B).  TEST INFRASTRUCTURE ONLY.

Only tests/, the package smoke check and bench.py's CPU-baseline leg use this module.  It shares
no code with the CUDA path.

The dense tier (oracle/svt.py) takes a full SVD of the densified iterate, which is out of reach
beyond a few thousand rows.  This tier computes the same shrink from products with the sparse
iterate only (Sec. 2.2: Y^k vanishes off Omega, and the shrink needs only the singular triplets
above tau, Sec. 5.1.1):

  partial_svd      the leading singular triplets of Y by block subspace iteration (repeated
                   application of Y^T Y to an orthonormal block, re-orthonormalised by QR), with
                   Rayleigh-Ritz through the oracle's own one-sided Jacobi SVD after every step,
                   until every wanted Ritz triplet above tau has residual ||Y^T u - theta v|| <=
                   tol theta_1 (tol = 1e-12 by default) and every wanted one at or below tau is
                   resolved (residual <= 1e-3 theta_1) with theta + residual <= tau
  shrink           D_tau(Y) (eq. (2.2)) with the rank policy of Sec. 5.1.1 (s_k = r_{k-1} + 1, then
                   s_k += ell while sigma_{s_k} > tau), warm-started from the previous shrink
  svt              Algorithm 1 (Sec. 5.1.5) with that shrink: kick of eq. (5.3) (||P_Omega M||_2 by
                   the same partial SVD), stop eq. (5.5), dual step eq. (2.7)

The sparse products (scipy.sparse CSR) and QR (numpy) are library primitives; the small SVDs are
the oracle's Jacobi.  The dense tier pins this one (tests/test_oracle_sparse_tier.py).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np
import scipy.sparse as sp

from ._clib import jacobi_svd
from .svt import IterRecord, kick_k0


def sparse_iterate(n1: int, n2: int, rows, cols, vals) -> sp.csr_matrix:
    """Y with the values on Omega and exact zeros elsewhere, in CSR storage."""
    return sp.csr_matrix((np.asarray(vals, dtype=np.float64), (np.asarray(rows), np.asarray(cols))), shape=(n1, n2))


@dataclasses.dataclass
class PartialSVD:
    U: np.ndarray        # n1 x k
    s: np.ndarray        # k, decreasing
    V: np.ndarray        # n2 x k
    res: np.ndarray      # Ritz residuals ||Y^T u_i - s_i v_i||
    iters: int


def partial_svd(Y: sp.csr_matrix, k: int, V0: Optional[np.ndarray] = None, oversample: int = 20, tol: float = 1e-12,
                max_iter: int = 5000, seed: int = 0, tau: Optional[float] = None) -> PartialSVD:
    """Leading k singular triplets of Y (block subspace iteration + Rayleigh-Ritz).

    The Rayleigh-Ritz step factors Y V = Q R (QR) and takes the Jacobi SVD of the small p x p
    factor R = U_R diag(s) W^T, so Y (V W) = (Q U_R) diag(s).  Stops when every wanted triplet
    has residual <= tol s_1; with tau given, a wanted triplet that is resolved (res_i <= 1e-3 s_1,
    so the block has found the singular value it stands for) and has s_i + res_i <= tau needs no
    more: its value is only compared against tau.  (An unresolved Ritz value with a large residual
    bounds no particular singular value: from a random start the first Ritz value can lie far
    below sigma_1 with s_1 + res_1 <= tau.)"""
    n1, n2 = Y.shape
    kmin = min(n1, n2)
    k = min(k, kmin)
    p = min(kmin, k + oversample)
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((n2, p))
    if V0 is not None and V0.shape[1] > 0:
        c = min(p, V0.shape[1])
        V[:, :c] = V0[:, :c]
    V, _ = np.linalg.qr(V)
    YT = Y.T.tocsr()
    it = 0
    while True:
        it += 1
        # Rayleigh-Ritz on span(V): Y V = U_B diag(s) W^T  =>  Y (V W) = U_B diag(s)
        Q, R = np.linalg.qr(Y @ V)
        UR, s, W = jacobi_svd(R)
        UB = Q @ UR
        Vr = V @ W
        R = YT @ UB - Vr * s
        res = np.linalg.norm(R, axis=0)
        ok = res[:k] <= tol * max(s[0], 1e-300)
        if tau is not None:
            ok |= (res[:k] <= 1e-3 * max(s[0], 1e-300)) & (s[:k] + res[:k] <= tau)
        if np.all(ok) or it >= max_iter:
            return PartialSVD(U=UB[:, :k], s=s[:k], V=Vr[:, :k], res=res[:k], iters=it)
        # one step of subspace iteration on Y^T Y, started from the Ritz basis
        V, _ = np.linalg.qr(YT @ (Y @ Vr))


def shrink(Y: sp.csr_matrix, tau: float, r_prev: int, ell: int = 5, V0: Optional[np.ndarray] = None,
           tol: float = 1e-12):
    """D_tau(Y) in factored form with the rank policy of Sec. 5.1.1.

    Returns (U_r, d, V_r, sigma, s_k, passes, V_warm) with d = sigma_1..r - tau > 0, sigma the
    computed singular values (the first s_k) and V_warm the right vectors of the last pass."""
    kmin = min(Y.shape)
    s_k = min(r_prev + 1, kmin)
    passes = 0
    warm = V0
    while True:
        passes += 1
        ps = partial_svd(Y, s_k, V0=warm, tol=tol, tau=tau)
        warm = ps.V
        if s_k >= kmin or ps.s[s_k - 1] <= tau:
            break
        s_k = min(s_k + ell, kmin)
    r = int(np.count_nonzero(ps.s > tau))
    return ps.U[:, :r], ps.s[:r] - tau, ps.V[:, :r], ps.s, s_k, passes, ps.V


@dataclasses.dataclass
class SparseSVTResult:
    iters: int
    k0: int
    norm2: float
    converged: bool
    U: np.ndarray
    d: np.ndarray
    V: np.ndarray
    y_omega: np.ndarray
    trace: List[IterRecord]


def svt(n1: int, n2: int, rows, cols, m_vals, tau: float, delta: float, eps: float = 1e-4, ell: int = 5,
        k_max: int = 1000, k0: Optional[int] = None, keep_trace: bool = True, tol: float = 1e-12,
        on_iter: Optional[Callable[[IterRecord], None]] = None) -> SparseSVTResult:
    """Algorithm 1 (Sec. 5.1.5) with the sparse shrink; the same records as the dense tier.

    on_iter, when given, receives every iterate's record as it is produced (x_omega and y_omega
    included), so that long runs can be summarised without keeping the whole trace in memory."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    m_vals = np.asarray(m_vals, dtype=np.float64)
    norm_m = math.sqrt(float(np.sum(m_vals * m_vals)))
    norm2 = float(partial_svd(sparse_iterate(n1, n2, rows, cols, m_vals), 1, tol=tol).s[0])
    if k0 is None:
        k0 = kick_k0(tau, delta, norm2)
    y = k0 * delta * m_vals
    r_prev = 0
    warm = None
    trace: List[IterRecord] = []
    converged = False
    U = np.zeros((n1, 0)); d = np.zeros(0); V = np.zeros((n2, 0))
    k = 0
    for k in range(1, k_max + 1):
        Y = sparse_iterate(n1, n2, rows, cols, y)
        U, d, V, s, s_k, passes, warm = shrink(Y, tau, r_prev, ell, V0=warm, tol=tol)
        r_k = d.shape[0]
        x = np.einsum("pj,j,pj->p", U[rows], d, V[cols]) if r_k > 0 else np.zeros_like(y)
        e = m_vals - x
        res = math.sqrt(float(np.sum(e * e))) / norm_m
        if keep_trace or on_iter is not None:
            rec = IterRecord(k=k, s_k=s_k, passes=passes, r_k=r_k, res=res, x_omega=x.copy(),
                             y_omega=y.copy(), sigma=s[:r_k + ell].copy())
            if keep_trace:
                trace.append(rec)
            if on_iter is not None:
                on_iter(rec)
        r_prev = r_k
        if res <= eps:
            converged = True
            break
        y = y + delta * e
    return SparseSVTResult(iters=k, k0=k0, norm2=norm2, converged=converged, U=U, d=d, V=V, y_omega=y, trace=trace)
