"""Float64 CPU oracle of the two alternative ways of running the SVT iteration that Sec. 6 of the
paper proposes.  TEST INFRASTRUCTURE ONLY: only tests/, the package smoke check and bench.py's
CPU-baseline leg use this module; it shares no code with the CUDA path.

  randomized_shrink   D_tau(Y) evaluated through a randomized range finder (the first proposal of
                      Sec. 6: approximate Y by a low-rank matrix from randomized procedures and keep
                      the part of its SVD above tau).  With a test block Omega (n2 x l), the range
                      Q = orth(Y Omega) is refined by `power` steps Q <- orth(Y orth(Y^T Q)); then
                      Y ~ Q Q^T Y = Q B with B = Q^T Y, and D_tau(Q B) = Q U_B diag((s - tau)_+)
                      V_B^T from the SVD B = U_B diag(s) V_B^T.  The rank policy of Sec. 5.1.1 sets
                      the number of wanted values: s_k = r_{k-1} + 1, then s_k += ell while the
                      s_k-th computed value exceeds tau; l = min(32, s_k + oversample rounded up
                      to a multiple of 8) columns (min(n1, n2) >= l is required).  Omega holds
                      the previous shrink's right singular vectors (warm start) followed by
                      uniform(-1, 1) columns: element (i, c) of the n2 x l block is
                      (SplitMix64 output number i l + c + 1 at the seed) >> 11 times 2^-52, minus 1,
                      with seed = base_seed + 1000 k + pass (k the SVT iteration, pass the rank
                      policy's pass).
  svt_randomized      Algorithm 1 (Sec. 5.1.5) with that shrink.
  svt_continuation    the continuation strategy of Sec. 6: Algorithm 1 at tau_0 (with the kick of
                      Sec. 5.1.3), then at tau_1, tau_2, ... in turn, each started from the final
                      dual iterate Y of the previous value (warm start), each run to the stopping
                      rule eq. (5.5).

Library primitives: scipy sparse products, numpy QR (the orthonormal range bases; only their span
enters D_tau(Q Q^T Y)), the oracle's own Jacobi SVD for the l x n2 matrix B.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np
import scipy.sparse as sp

from ._clib import jacobi_svd, splitmix64
from .svt import IterRecord, kick_k0, spectral_norm


def test_block(n2: int, l: int, c0: int, seed: int) -> np.ndarray:
    """n2 x l block with columns c >= c0 uniform(-1, 1) from SplitMix64 (columns < c0 zero)."""
    out = np.zeros((n2, l))
    for i in range(n2):
        for c in range(c0, l):
            z = splitmix64(seed, i * l + c + 1)
            out[i, c] = (z >> 11) * (2.0 / 9007199254740992.0) - 1.0
    return out


def _orth(A: np.ndarray) -> np.ndarray:
    Q, _ = np.linalg.qr(A)
    return Q


@dataclasses.dataclass
class RandShrink:
    U: np.ndarray        # n1 x r
    d: np.ndarray        # sigma - tau > 0
    V: np.ndarray        # n2 x r
    sigma: np.ndarray    # the computed values (l of them), decreasing
    V_all: np.ndarray    # n2 x l right vectors (warm start of the next shrink)
    s_k: int
    passes: int


def randomized_shrink(Y: sp.csr_matrix, tau: float, r_prev: int, V_prev: Optional[np.ndarray], ell: int,
                      oversample: int, power: int, seed_of_pass) -> RandShrink:
    """D_tau(Y) through the randomized range finder with the rank policy (see the module header).
    seed_of_pass(pass) gives the SplitMix64 seed of the random columns of that pass (0-based)."""
    n1, n2 = Y.shape
    kmin = min(n1, n2)
    YT = Y.T.tocsr()
    s = min(r_prev + 1, kmin)
    warm = V_prev
    passes = 0
    while True:
        if s + oversample > 32 and s < kmin:
            raise ValueError("s_k + oversample exceeds 32 test columns")
        l = min(32, (s + oversample + 7) // 8 * 8)
        if l > kmin:
            raise ValueError("the test block needs min(n1, n2) >= %d" % l)
        c0 = 0 if warm is None else min(warm.shape[1], l)
        Om = test_block(n2, l, c0, seed_of_pass(passes))
        if c0 > 0:
            Om[:, :c0] = warm[:, :c0]
        passes += 1
        Q = _orth(Y @ Om)
        for _ in range(power):
            Q = _orth(Y @ _orth(YT @ Q))
        B = (YT @ Q).T                      # l x n2 = Q^T Y
        UB, sig, VB = jacobi_svd(B)
        U_all = Q @ UB
        s_eff = min(s, sig.shape[0])
        if s_eff < kmin and sig[s_eff - 1] > tau:
            s = min(s + ell, kmin)
            warm = VB
            continue
        r = int(np.count_nonzero(sig > tau))
        return RandShrink(U=U_all[:, :r], d=sig[:r] - tau, V=VB[:, :r], sigma=sig, V_all=VB, s_k=s_eff,
                          passes=passes)


@dataclasses.dataclass
class AltResult:
    iters: int
    k0: int
    converged: bool
    U: np.ndarray
    d: np.ndarray
    V: np.ndarray
    y_omega: np.ndarray
    trace: List[IterRecord]
    stage_iters: List[int] = dataclasses.field(default_factory=list)


def _csr(n1, n2, rows, cols, vals):
    return sp.csr_matrix((np.asarray(vals, dtype=np.float64), (np.asarray(rows), np.asarray(cols))), shape=(n1, n2))


def svt_randomized(n1: int, n2: int, rows, cols, m_vals, tau: float, delta: float, eps: float = 1e-4,
                   ell: int = 5, k_max: int = 1000, k0: Optional[int] = None, oversample: int = 8,
                   power: int = 1, base_seed: int = 0) -> AltResult:
    """Algorithm 1 (Sec. 5.1.5) with the randomized shrink; kick of eq. (5.3) as in Algorithm 1."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    m_vals = np.asarray(m_vals, dtype=np.float64)
    norm_m = math.sqrt(float(np.sum(m_vals * m_vals)))
    if k0 is None:
        k0 = kick_k0(tau, delta, spectral_norm(n1, n2, rows, cols, m_vals))
    y = k0 * delta * m_vals
    r_prev, warm = 0, None
    trace: List[IterRecord] = []
    converged = False
    U = np.zeros((n1, 0)); d = np.zeros(0); V = np.zeros((n2, 0))
    k = 0
    for k in range(1, k_max + 1):
        sh = randomized_shrink(_csr(n1, n2, rows, cols, y), tau, r_prev, warm, ell, oversample, power,
                               lambda ps, kk=k: base_seed + 1000 * kk + ps)
        U, d, V = sh.U, sh.d, sh.V
        x = np.einsum("pj,j,pj->p", U[rows], d, V[cols]) if d.size else np.zeros_like(y)
        e = m_vals - x
        res = math.sqrt(float(np.sum(e * e))) / norm_m
        trace.append(IterRecord(k=k, s_k=sh.s_k, passes=sh.passes, r_k=d.size, res=res, x_omega=x.copy(),
                                y_omega=y.copy(), sigma=sh.sigma[:d.size + ell].copy()))
        r_prev, warm = d.size, sh.V_all
        if res <= eps:
            converged = True
            break
        y = y + delta * e
    return AltResult(iters=k, k0=k0, converged=converged, U=U, d=d, V=V, y_omega=y, trace=trace)


def svt_continuation(n1: int, n2: int, rows, cols, m_vals, taus: Sequence[float], delta: float,
                     eps: float = 1e-4, ell: int = 5, k_max: int = 1000, k0: Optional[int] = None) -> AltResult:
    """The continuation strategy of Sec. 6: Algorithm 1 for tau_0 (kick of eq. (5.3) at tau_0), then for
    each later tau_i from the previous stage's final dual iterate, every stage to the stopping rule
    eq. (5.5).  The exact shrink is the dense tier's (full Jacobi SVD); the trace runs across stages
    (k counts every iteration) and stage_iters holds the iterations of each stage."""
    from .svt import svt_step
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    m_vals = np.asarray(m_vals, dtype=np.float64)
    norm_m = math.sqrt(float(np.sum(m_vals * m_vals)))
    if k0 is None:
        k0 = kick_k0(taus[0], delta, spectral_norm(n1, n2, rows, cols, m_vals))
    y = k0 * delta * m_vals
    r_prev = 0
    trace: List[IterRecord] = []
    stage_iters: List[int] = []
    converged = False
    U = np.zeros((n1, 0)); d = np.zeros(0); V = np.zeros((n2, 0))
    k = 0
    for tau in taus:
        converged = False
        it = 0
        while it < k_max:
            it += 1
            k += 1
            st = svt_step(n1, n2, rows, cols, m_vals, y, tau, r_prev, ell, norm_m)
            U, d, V = st.U, st.d, st.V
            trace.append(IterRecord(k=k, s_k=st.s_k, passes=st.passes, r_k=st.r_k, res=st.res, x_omega=st.x.copy(),
                                    y_omega=y.copy(), sigma=st.sigma[:st.r_k + ell].copy()))
            r_prev = st.r_k
            if st.res <= eps:
                converged = True
                break
            y = y + delta * st.e
        stage_iters.append(it)
    return AltResult(iters=k, k0=k0, converged=converged, U=U, d=d, V=V, y_omega=y, trace=trace,
                     stage_iters=stage_iters)
