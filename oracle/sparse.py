"""Float64 definitions of the sparse building blocks of the SVT path.  TEST INFRASTRUCTURE ONLY.

Only tests/, the package smoke check and bench.py's CPU-baseline leg use this module.  It shares
no code with the CUDA path.

  csr_structure / csc_structure  storage of the fixed sampled set Omega, sorted (Sec. 2.2, the
                                 sparsity remark: Y^k vanishes off Omega, so only Omega is stored)
  apply_Y / apply_Yt             W = Y V and Z = Y^T U for Y supported on Omega (the products the
                                 Lanczos partial SVD needs, Sec. 2.2 and Sec. 5.1.1)
  sample_X                       X^k on Omega from the factors, x_ij = sum_t U~_it V_jt
                                 (X^k = sum_j (sigma_j - tau) u_j v_j^T, Algorithm 1)
  dual_update                    Y^k_ij = Y^{k-1}_ij + delta (M_ij - X^k_ij) on Omega and the squared
                                 residual sum ||P_Omega(X^k - M)||_F^2 (Algorithm 1; eq. (5.5))
"""
from __future__ import annotations

import numpy as np


def csr_structure(n1: int, n2: int, rows, cols):
    """Row-major storage of Omega: (row_ptr[n1+1], col_idx[nnz], order) with `order` the
    permutation that sorts the input pairs by (row, col).  Duplicates raise ValueError."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    if rows.size and (rows.min() < 0 or rows.max() >= n1 or cols.min() < 0 or cols.max() >= n2):
        raise ValueError("index out of range")
    order = np.lexsort((cols, rows))
    r_s, c_s = rows[order], cols[order]
    if r_s.size > 1:
        dup = (r_s[1:] == r_s[:-1]) & (c_s[1:] == c_s[:-1])
        if dup.any():
            raise ValueError("duplicate index")
    row_ptr = np.zeros(n1 + 1, dtype=np.int64)
    np.add.at(row_ptr, r_s + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr.astype(np.int32), c_s.astype(np.int32), order


def csc_structure(n1: int, n2: int, csr_rows, csr_cols):
    """Column-major storage of Omega given the row-major sorted pairs: (col_ptr[n2+1],
    row_idx[nnz], csc_to_csr[nnz]) where csc_to_csr[q] is the row-major position of the q-th
    column-major entry."""
    csr_rows = np.asarray(csr_rows, dtype=np.int64)
    csr_cols = np.asarray(csr_cols, dtype=np.int64)
    order = np.lexsort((csr_rows, csr_cols))
    col_ptr = np.zeros(n2 + 1, dtype=np.int64)
    np.add.at(col_ptr, csr_cols[order] + 1, 1)
    col_ptr = np.cumsum(col_ptr)
    return col_ptr.astype(np.int32), csr_rows[order].astype(np.int32), order.astype(np.int32)


def apply_Y(n1: int, rows, cols, yvals, V: np.ndarray) -> np.ndarray:
    """W = Y V: W[i, :] = sum over samples p in row i of y_p V[col_p, :]."""
    W = np.zeros((n1, V.shape[1]))
    np.add.at(W, np.asarray(rows), np.asarray(yvals)[:, None] * V[np.asarray(cols)])
    return W


def apply_Yt(n2: int, rows, cols, yvals, U: np.ndarray) -> np.ndarray:
    """Z = Y^T U: Z[j, :] = sum over samples p in column j of y_p U[row_p, :]."""
    Z = np.zeros((n2, U.shape[1]))
    np.add.at(Z, np.asarray(cols), np.asarray(yvals)[:, None] * U[np.asarray(rows)])
    return Z


def sample_X(rows, cols, Ut: np.ndarray, V: np.ndarray) -> np.ndarray:
    """x_p = sum_t Ut[row_p, t] V[col_p, t] (X = Ut V^T evaluated on Omega only)."""
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    x = np.zeros(rows.shape[0])
    for t in range(Ut.shape[1]):
        x += Ut[rows, t] * V[cols, t]
    return x


def dual_update(yvals, mvals, xvals, delta: float):
    """(Y^k on Omega, ||P_Omega(M - X^k)||_F^2) for Y^k = Y^{k-1} + delta P_Omega(M - X^k)."""
    e = np.asarray(mvals) - np.asarray(xvals)
    return np.asarray(yvals) + delta * e, float(np.sum(e * e))
