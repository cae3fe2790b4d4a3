"""svt_sddmm_update_noalloc, the allocation-free variant of the fused X-on-Omega + dual step for
callers that cannot call cudaMalloc (device memory owned by another pool, or a loop that cannot
afford the synchronisation of an allocation).  Its output must match svt_sddmm_update, the
entry point that works through a context, on two calls in a row (the second call reuses the
static scratch the first one left behind), and the float64 oracle's X-on-Omega and dual step
(oracle.sparse.sample_X, oracle.sparse.dual_update: Y^k = Y^{k-1} + delta P_Omega(M - X^k)).

This file is collected last so that a run that stops at the first failure has run every other
test before it; it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from oracle.sparse import dual_update, sample_X
from svt_inputs import random_dense, random_sparse_pattern

pytestmark = pytest.mark.gpu


def _noalloc(L, torch, n1, n2, rp, ci, mv, Ut, V, r, delta, y_in, y_out):
    res2 = ctypes.c_double()
    st = L.svt_sddmm_update_noalloc(n1, n2, int(ci.numel()), rp.data_ptr(), ci.data_ptr(), mv.data_ptr(),
                                    Ut.data_ptr() if r else None, V.data_ptr() if r else None, r, delta,
                                    y_in.data_ptr(), y_out.data_ptr(), ctypes.byref(res2), None)
    assert st == 0, L.svt_noalloc_last_error()
    return res2.value


def test_noalloc_matches_context_entry_point_twice(cuda):
    torch = cuda
    from paper_0810_3286_gb300 import Solver, library
    L = library()
    n1, n2 = 700, 433   # several CTAs of 64 rows and a ragged last one
    rows, cols, mvals = random_sparse_pattern(n1, n2, 30000, 31, empty_rows=(5,), dense_rows=(11,))
    s = Solver(n1, n2, rows, cols, mvals, precision="fp64")
    rp, ci, _, _, _ = s.structure()
    rp_d = torch.from_numpy(rp).cuda()
    ci_d = torch.from_numpy(ci).cuda()
    mv_d = torch.from_numpy(mvals).cuda()   # the pattern is generated in row-major order
    for call, (r, delta, seed) in enumerate([(10, 10.05, 1), (23, 3.5, 2)]):
        Ut = torch.from_numpy(random_dense((n1, r), seed)).cuda()
        V = torch.from_numpy(random_dense((n2, r), seed + 100)).cuda()
        y_in = torch.from_numpy(random_dense(rows.size, seed + 200)).cuda()
        y_ref = torch.empty_like(y_in)
        y_out = torch.full_like(y_in, float("nan"))
        res_ref = s.sddmm_update(Ut, V, delta, y_in, y_ref)
        res_na = _noalloc(L, torch, n1, n2, rp_d, ci_d, mv_d, Ut, V, r, delta, y_in, y_out)
        torch.cuda.synchronize()
        a, b = y_out.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), "call %d left entries unwritten" % call
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b), call
        assert abs(res_na - res_ref) <= 1e-12 * res_ref, (call, res_na, res_ref)
        # the oracle, on the same row-major entries: float64 sums of r <= 23 products reordered
        y_or, res_or = dual_update(y_in.cpu().numpy(), mvals,
                                   sample_X(rows, cols, Ut.cpu().numpy(), V.cpu().numpy()), delta)
        assert np.linalg.norm(a - y_or) <= 1e-12 * np.linalg.norm(y_or), call
        assert abs(res_na - res_or) <= 1e-12 * res_or, (call, res_na, res_or)
    s.close()


def test_noalloc_rejects_rows_beyond_scratch(cuda):
    torch = cuda
    from paper_0810_3286_gb300 import library
    L = library()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    idx = torch.zeros(8, dtype=torch.int32, device="cuda")
    res2 = ctypes.c_double()
    st = L.svt_sddmm_update_noalloc(262081, 10, 1, idx.data_ptr(), idx.data_ptr(), dummy.data_ptr(), None, None, 0,
                                    1.0, dummy.data_ptr(), dummy[4:].data_ptr(), ctypes.byref(res2), None)
    assert st == 1  # SVT_ERR_ARG
    assert b"262080" in L.svt_noalloc_last_error()
