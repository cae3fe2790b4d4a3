"""Pins of the oracle's sparse building blocks against dense definitions (Sec. 2.2: Y^k is
supported on Omega; the Lanczos partial SVD needs only products with Y and Y^T)."""
import numpy as np
import pytest

from oracle import sparse as osp
from oracle import svt as osvt
from svt_inputs import random_sparse_pattern


@pytest.mark.parametrize("n1,n2,m,seed", [(17, 23, 90, 0), (40, 7, 150, 1), (5, 60, 300, 2)])
def test_csr_csc_structure(n1, n2, m, seed):
    rows, cols, vals = random_sparse_pattern(n1, n2, m, seed, empty_rows=(0, 3), empty_cols=(1,))
    perm = np.random.default_rng(seed).permutation(rows.size)
    row_ptr, col_idx, order = osp.csr_structure(n1, n2, rows[perm], cols[perm])
    assert row_ptr[0] == 0 and row_ptr[-1] == rows.size
    for i in range(n1):
        seg = col_idx[row_ptr[i]:row_ptr[i + 1]]
        assert np.all(np.diff(seg) > 0)
        assert np.array_equal(np.sort(cols[rows == i]), seg)
    assert np.array_equal(rows[perm][order], rows) and np.array_equal(cols[perm][order], cols)
    col_ptr, row_idx, csc_to_csr = osp.csc_structure(n1, n2, rows, cols)
    for j in range(n2):
        seg = row_idx[col_ptr[j]:col_ptr[j + 1]]
        assert np.all(np.diff(seg) > 0)
        assert np.array_equal(np.sort(rows[cols == j]), seg)
    assert np.array_equal(rows[csc_to_csr], row_idx)


def test_duplicate_and_range_rejected():
    with pytest.raises(ValueError):
        osp.csr_structure(3, 3, [0, 1, 1], [2, 0, 0])
    with pytest.raises(ValueError):
        osp.csr_structure(3, 3, [0, 3], [0, 0])


def test_products_match_dense():
    n1, n2 = 31, 19
    rows, cols, y = random_sparse_pattern(n1, n2, 200, 5, empty_rows=(2,), dense_rows=(7,))
    Y = osvt.dense_from_omega(n1, n2, rows, cols, y)
    rng = np.random.default_rng(0)
    V = rng.standard_normal((n2, 6))
    U = rng.standard_normal((n1, 6))
    assert np.abs(osp.apply_Y(n1, rows, cols, y, V) - Y @ V).max() <= 1e-13
    assert np.abs(osp.apply_Yt(n2, rows, cols, y, U) - Y.T @ U).max() <= 1e-13
    Ut = rng.standard_normal((n1, 4))
    Vt = rng.standard_normal((n2, 4))
    assert np.abs(osp.sample_X(rows, cols, Ut, Vt) - (Ut @ Vt.T)[rows, cols]).max() <= 1e-13
    mvals = rng.standard_normal(rows.size)
    x = osp.sample_X(rows, cols, Ut, Vt)
    ynew, r2 = osp.dual_update(y, mvals, x, 2.5)
    assert np.abs(ynew - (y + 2.5 * (mvals - x))).max() == 0.0
    assert r2 == pytest.approx(float(np.sum((mvals - x) ** 2)))
