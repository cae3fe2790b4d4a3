"""GPU parity of the per-iteration kernels against the oracle's float64 definitions:
Y V and Y^T U (the products of the Lanczos partial SVD, Sec. 5.1.1) and the fused evaluation of
X on Omega + dual step + residual (Algorithm 1; eq. (5.5))."""
import numpy as np
import pytest

from oracle import sparse as osp
from svt_inputs import random_dense, random_sparse_pattern

pytestmark = pytest.mark.gpu

# float64 path: the only differences are summation orders (a few ulps times the row length).
# float32 path: float32 values and accumulation; relative error bound ~ row length * 2^-24.
TOL = {"fp64": 1e-12, "fp32": 2e-5}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("b", [2, 8, 16, 24, 32, 64])
def test_apply_Y_and_Yt(cuda, precision, b):
    torch = cuda
    from paper_0810_3286_gb300 import Solver
    n1, n2 = 517, 389   # several warps' worth of rows and a ragged tail
    rows, cols, y = random_sparse_pattern(n1, n2, 30000, 3, empty_rows=(0, 100), empty_cols=(5,), dense_rows=(7,))
    s = Solver(n1, n2, rows, cols, y, precision=precision)
    s.set_Y(y)
    V = random_dense((n2, b), 1)
    U = random_dense((n1, b), 2)
    Vd = torch.from_numpy(V).cuda()
    Ud = torch.from_numpy(U).cuda()
    W = torch.empty((n1, b), dtype=torch.float64, device="cuda")
    Z = torch.empty((n2, b), dtype=torch.float64, device="cuda")
    s.apply_Y(Vd, W)
    s.apply_Yt(Ud, Z)
    torch.cuda.synchronize()
    W_ref = osp.apply_Y(n1, rows, cols, y, V)
    Z_ref = osp.apply_Yt(n2, rows, cols, y, U)
    assert _rel(W.cpu().numpy(), W_ref) <= TOL[precision]
    assert _rel(Z.cpu().numpy(), Z_ref) <= TOL[precision]
    # empty rows/cols give exact zeros
    assert np.all(W.cpu().numpy()[[0, 100]] == 0.0)
    assert np.all(Z.cpu().numpy()[5] == 0.0)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("r", [0, 1, 5, 10, 33, 64])
def test_sddmm_update(cuda, precision, r):
    torch = cuda
    from paper_0810_3286_gb300 import Solver
    n1, n2 = 611, 301
    rows, cols, mvals = random_sparse_pattern(n1, n2, 25000, 4, empty_rows=(3,), dense_rows=(9,))
    s = Solver(n1, n2, rows, cols, mvals, precision=precision)
    y = random_dense(rows.size, 5)
    Ut = random_dense((n1, max(r, 1)), 6)[:, :r].copy()
    V = random_dense((n2, max(r, 1)), 7)[:, :r].copy()
    delta = 3.7
    y_in = torch.from_numpy(y).cuda()
    y_out = torch.empty_like(y_in)
    res2 = s.sddmm_update(torch.from_numpy(Ut).cuda() if r else None, torch.from_numpy(V).cuda() if r else None,
                          delta, y_in, y_out)
    x = osp.sample_X(rows, cols, Ut, V)
    y_ref, r2_ref = osp.dual_update(y, mvals, x, delta)
    tol = TOL[precision] * (10 if precision == "fp32" else 1)
    assert _rel(y_out.cpu().numpy(), y_ref) <= tol
    assert abs(res2 - r2_ref) <= tol * r2_ref
    s.close()


def test_sddmm_update_full_size_sampled(cuda):
    """1000 x 1000, |Omega| = 119400, rank 10 (the single-solve workload): sampled entries
    recomputed one by one by the oracle's definition."""
    torch = cuda
    from paper_0810_3286_gb300 import Solver
    from svt_inputs import config_problem
    p = config_problem("single_1000", 0)
    s = Solver(p.n1, p.n2, p.rows, p.cols, p.vals, precision="fp32")
    Ut = random_dense((p.n1, 10), 8)
    V = random_dense((p.n2, 10), 9)
    y = random_dense(p.nnz, 10)
    y_out = torch.empty(p.nnz, dtype=torch.float64, device="cuda")
    res2 = s.sddmm_update(torch.from_numpy(Ut).cuda(), torch.from_numpy(V).cuda(), 10.05,
                          torch.from_numpy(y).cuda(), y_out)
    yo = y_out.cpu().numpy()
    idx = np.random.default_rng(0).choice(p.nnz, 2000, replace=False)
    for q in idx:
        i, j = p.rows[q], p.cols[q]
        x = float(np.dot(Ut[i], V[j]))
        ref = y[q] + 10.05 * (p.vals[q] - x)
        assert abs(yo[q] - ref) <= 2e-5 * max(1.0, abs(ref))
    x_all = osp.sample_X(p.rows, p.cols, Ut, V)
    r2 = float(np.sum((p.vals - x_all) ** 2))
    assert abs(res2 - r2) <= 1e-5 * r2
    s.close()


def test_newton_helpers_against_cuda_division_and_rsqrt(cuda):
    """The library's float64 reciprocal / reciprocal square root (Newton's iteration from float32
    seeds; the Cholesky pivot's variant halves the exponent exactly first, so it covers every normal
    double) against CUDA's correctly rounded float64 division and square root.  The float32-seeded
    helpers serve values inside the float32 range (2^-100 .. 2^100 here); the pivot helper is tested
    over 2^-1000 .. 2^1000.  Relative errors: the square of the seed error (2^-23 for the
    reciprocal, ~2^-22 for rsqrtf) per single step, plus a few roundings."""
    torch = cuda
    from paper_0810_3286_gb300 import library
    L = library()
    g = torch.Generator().manual_seed(7)
    rel = lambda a, b: float(((a - b) / b).abs().max())
    for lo, hi, slots in ((-100, 100, (0, 1, 2, 3, 4)), (-1000, 1000, (4,))):
        e = torch.randint(lo, hi, (20000,), generator=g).double()
        m = 1.0 + torch.rand(20000, generator=g, dtype=torch.float64)
        x = (m * torch.pow(2.0, e)).cuda()
        out = torch.empty((20000, 5), dtype=torch.float64, device="cuda")
        assert L.svt_selftest_math(x.numel(), x.data_ptr(), out.data_ptr(), None) == 0
        rcp = 1.0 / x
        rs = 1.0 / torch.sqrt(x)
        bounds = {0: (rcp, 1e-15), 1: (rcp, 1e-14), 2: (rs, 1e-15), 3: (rs, 2e-13), 4: (rs, 2e-13)}
        for sl in slots:
            ref, b = bounds[sl]
            assert rel(out[:, sl], ref) <= b, (lo, hi, sl, rel(out[:, sl], ref))
