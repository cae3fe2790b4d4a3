"""Planted low-rank completion problems (Sec. 5.2.1 workload) drawn from a seeded PCG64 stream.

Recipe (paper Sec. 5.2.1, Table 1):
  * M_L (n1 x r), M_R (n2 x r) with i.i.d. N(0, 1) entries, M = M_L M_R^T;
  * Omega: m distinct linear ids i*n2 + j drawn uniformly without replacement from [0, n1*n2),
    returned sorted (row-major order, i.e. sorted by (i, j));
  * m = c * d_r with d_r = r(n1 + n2 - r) degrees of freedom (c = m/d_r, the oversampling ratio;
    the square case gives the paper's d_r = r(2n - r));
  * values M_ij on Omega accumulated in float64 in the fixed order t = 0..r-1;
  * optional noise: B_ij = M_ij + sigma * z_ij with z_ij ~ N(0, 1) (Sec. 5.2.1, noisy model).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def dof(n1: int, n2: int, r: int) -> int:
    """Degrees of freedom of an n1 x n2 rank-r matrix, r(n1 + n2 - r) (footnote to Sec. 1.1)."""
    return r * (n1 + n2 - r)


def sample_count(n1: int, n2: int, r: int, ratio: float) -> int:
    """|Omega| = ratio * d_r, rounded to the nearest integer and capped at n1*n2."""
    return int(min(n1 * n2, round(ratio * dof(n1, n2, r))))


@dataclasses.dataclass
class PlantedProblem:
    n1: int
    n2: int
    r: int
    seed: int
    A: np.ndarray          # n1 x r, float64 (M_L)
    B: np.ndarray          # n2 x r, float64 (M_R)
    rows: np.ndarray       # nnz, int32, sorted row-major together with cols
    cols: np.ndarray       # nnz, int32
    vals: np.ndarray       # nnz, float64: M_ij (+ noise if sigma > 0) on Omega
    noise_sigma: float = 0.0

    @property
    def nnz(self) -> int:
        return int(self.rows.shape[0])

    @property
    def p(self) -> float:
        """Sampling ratio p = m / (n1 n2) (Sec. 5.1.2)."""
        return self.nnz / float(self.n1 * self.n2)

    def tau_default(self) -> float:
        """tau = 5 n (Sec. 5.2.1); for rectangular inputs 5 sqrt(n1 n2)."""
        return 5.0 * math.sqrt(self.n1 * self.n2)

    def delta_default(self) -> float:
        """delta = 1.2 n1 n2 / m (Sec. 5.1.2, step-size heuristic)."""
        return 1.2 * self.n1 * self.n2 / self.nnz

    def dense_M(self) -> np.ndarray:
        return self.A @ self.B.T


def _sample_omega(rng: np.random.Generator, n1: int, n2: int, m: int) -> np.ndarray:
    N = n1 * n2
    if m > N:
        raise ValueError("m exceeds n1*n2")
    if m == N:
        return np.arange(N, dtype=np.int64)
    ids = rng.choice(N, size=m, replace=False)
    ids = np.asarray(ids, dtype=np.int64)
    ids.sort()
    return ids


def planted_problem(n1: int, n2: int, r: int, m: int, seed: int, noise_sigma: float = 0.0) -> PlantedProblem:
    """Draw one planted problem. Draw order: M_L, M_R, Omega, noise (fixed, so results are stable)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    A = rng.standard_normal((n1, r))
    B = rng.standard_normal((n2, r))
    ids = _sample_omega(rng, n1, n2, m)
    rows = (ids // n2).astype(np.int32)
    cols = (ids % n2).astype(np.int32)
    vals = np.zeros(m, dtype=np.float64)
    for t in range(r):
        vals += A[rows, t] * B[cols, t]
    if noise_sigma > 0.0:
        vals = vals + noise_sigma * rng.standard_normal(m)
    return PlantedProblem(n1=n1, n2=n2, r=r, seed=seed, A=A, B=B, rows=rows, cols=cols, vals=vals,
                          noise_sigma=noise_sigma)


# The problem shapes of the workloads (paper Table 1 rows and smaller companions).
CONFIGS = {
    # 200 x 200, rank 5, |Omega| = 6 d_r = 11850 (no paper number: small FP64 parity case)
    "plain_fp64_200": dict(n1=200, n2=200, r=5, ratio=6.0),
    # 1000 x 1000, rank 10, |Omega| = 6 d_r = 119400 (Table 1, first row)
    "single_1000": dict(n1=1000, n2=1000, r=10, ratio=6.0),
    # 2000 x 2000, rank 10, |Omega| = 6 d_r = 239400 (companion of the 10000^2 case)
    "companion_2000": dict(n1=2000, n2=2000, r=10, ratio=6.0),
    # 10000 x 10000, rank 10, |Omega| = 6 d_r = 1199400 (Table 1)
    "single_10000": dict(n1=10000, n2=10000, r=10, ratio=6.0),
    # 30000 x 30000, rank 10, |Omega| = 6 d_r = 3599400 (Table 1, last row)
    "large_30000": dict(n1=30000, n2=30000, r=10, ratio=6.0),
}


def config_problem(name: str, seed: int = 0, noise_sigma: float = 0.0) -> PlantedProblem:
    c = CONFIGS[name]
    m = sample_count(c["n1"], c["n2"], c["r"], c["ratio"])
    return planted_problem(c["n1"], c["n2"], c["r"], m, seed, noise_sigma)


def random_dense(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """i.i.d. N(0,1) dense array (kernel-level parity inputs such as Lanczos blocks or factors)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    return rng.standard_normal(shape).astype(dtype)


def random_sparse_pattern(n1: int, n2: int, m: int, seed: int, empty_rows=(), empty_cols=(),
                          dense_rows=()):
    """A sorted sampled set with structure (empty rows/cols, dense rows) and N(0,1) values.

    Rows listed in empty_rows / columns in empty_cols get no samples; rows in dense_rows are
    fully sampled. The remaining budget is drawn uniformly without replacement.
    Returns (rows int32, cols int32, vals float64), sorted row-major.
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    mask = np.ones((n1, n2), dtype=bool)
    for i in empty_rows:
        mask[i, :] = False
    for j in empty_cols:
        mask[:, j] = False
    forced = np.zeros((n1, n2), dtype=bool)
    for i in dense_rows:
        forced[i, :] = mask[i, :]
    free = np.flatnonzero((mask & ~forced).ravel())
    need = max(0, m - int(forced.sum()))
    need = min(need, free.size)
    pick = rng.choice(free.size, size=need, replace=False) if need > 0 else np.zeros(0, dtype=np.int64)
    ids = np.concatenate([np.flatnonzero(forced.ravel()), free[pick]]).astype(np.int64)
    ids.sort()
    rows = (ids // n2).astype(np.int32)
    cols = (ids % n2).astype(np.int32)
    vals = rng.standard_normal(ids.size)
    return rows, cols, vals


def serving_job(seed: int, n_range=(500, 8000), rank_range=(5, 20), c_range=(4.0, 6.0),
                noise_sigma: float = 0.0) -> PlantedProblem:
    """One job of the serving workload: m, n uniform in n_range, rank uniform in rank_range,
    |Omega| = c r (m + n - r) with c uniform in c_range, N(0,1) planted factors, Omega uniform
    without replacement.  Omega is drawn as the distinct values of i.i.d. uniform ids, a uniform
    random subset of the right size of them kept (a procedure symmetric in the ids, hence uniform
    over m-subsets), which is much faster than choice without replacement for large n1 n2."""
    rng = np.random.default_rng(np.random.PCG64([seed, 0x5E4E]))
    n1 = int(rng.integers(n_range[0], n_range[1] + 1))
    n2 = int(rng.integers(n_range[0], n_range[1] + 1))
    r = int(rng.integers(rank_range[0], rank_range[1] + 1))
    c = float(rng.uniform(c_range[0], c_range[1]))
    m = min(int(round(c * r * (n1 + n2 - r))), n1 * n2)
    A = rng.standard_normal((n1, r))
    B = rng.standard_normal((n2, r))
    N = n1 * n2
    ids = np.zeros(0, dtype=np.int64)
    draw = m + m // 8 + 64
    while ids.size < m:
        ids = np.sort(np.concatenate([ids, rng.integers(0, N, size=draw, dtype=np.int64)]))
        ids = ids[np.concatenate(([True], ids[1:] != ids[:-1]))]
    if ids.size > m:
        ids = np.sort(rng.choice(ids, size=m, replace=False))
    rows = (ids // n2).astype(np.int32)
    cols = (ids % n2).astype(np.int32)
    vals = np.einsum("pt,pt->p", A[rows], B[cols])
    if noise_sigma > 0.0:
        vals = vals + noise_sigma * rng.standard_normal(m)
    return PlantedProblem(n1=n1, n2=n2, r=r, seed=seed, A=A, B=B, rows=rows, cols=cols, vals=vals,
                          noise_sigma=noise_sigma)
