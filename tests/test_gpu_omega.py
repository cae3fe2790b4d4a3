"""GPU parity of the Omega storage build and the random-keys sampler (bit-exact against the
oracle): Sec. 2.2 (the iterate lives on Omega only) and Sec. 5.2.1 (Omega uniform of size m)."""
import numpy as np
import pytest

from oracle import sample_omega as oracle_sample_omega
from oracle import sparse as osp
from svt_inputs import planted_problem, random_sparse_pattern

pytestmark = pytest.mark.gpu


def _check_structure(n1, n2, rows, cols, vals, precision="fp64"):
    from paper_0810_3286_gb300 import Solver
    perm = np.random.default_rng(n1 * 7 + n2).permutation(rows.size)
    r_in, c_in, v_in = rows[perm], cols[perm], vals[perm]
    s = Solver(n1, n2, r_in, c_in, v_in, precision=precision)
    rp, ci, cp, ri, c2r = s.structure()
    row_ptr, col_idx, order = osp.csr_structure(n1, n2, r_in, c_in)
    col_ptr, row_idx, csc_to_csr = osp.csc_structure(n1, n2, r_in[order], c_in[order])
    assert np.array_equal(rp, row_ptr)
    assert np.array_equal(ci, col_idx)
    assert np.array_equal(cp, col_ptr)
    assert np.array_equal(ri, row_idx)
    assert np.array_equal(c2r, csc_to_csr)
    s.close()


@pytest.mark.parametrize("n1,n2,m,seed", [(17, 23, 90, 0), (40, 7, 150, 1), (5, 60, 300, 2), (1, 1, 1, 3),
                                          (300, 257, 20000, 4)])
def test_structure_bit_exact(cuda, n1, n2, m, seed):
    rows, cols, vals = random_sparse_pattern(n1, n2, m, seed, empty_rows=(0,) if n1 > 2 else (),
                                             empty_cols=(n2 - 1,) if n2 > 2 else ())
    _check_structure(n1, n2, rows, cols, vals)


def test_structure_long_segments(cuda):
    # rows and columns longer than the shared-memory sort capacity take the global-memory path
    rows, cols, vals = random_sparse_pattern(6, 5000, 12000, 9, dense_rows=(2, 4))
    _check_structure(6, 5000, rows, cols, vals)
    rows, cols, vals = random_sparse_pattern(5000, 3, 9000, 10)
    _check_structure(5000, 3, rows, cols, vals, precision="fp32")


def test_structure_rejects_bad_input(cuda):
    from paper_0810_3286_gb300 import Solver, SVTError
    from paper_0810_3286_gb300._abi import SVT_ERR_ARG, SVT_ERR_DUP_INDEX
    rows = np.array([0, 1, 1, 2], np.int32)
    cols = np.array([0, 2, 2, 1], np.int32)
    with pytest.raises(SVTError) as e:
        Solver(3, 3, rows, cols, np.ones(4))
    assert e.value.status == SVT_ERR_DUP_INDEX
    with pytest.raises(SVTError) as e:
        Solver(3, 3, np.array([0, 3], np.int32), np.array([0, 0], np.int32), np.ones(2))
    assert e.value.status == SVT_ERR_ARG
    with pytest.raises(SVTError) as e:
        Solver(3, 3, np.array([0, 1], np.int32), np.array([-1, 0], np.int32), np.ones(2))
    assert e.value.status == SVT_ERR_ARG


def test_structure_from_device_inputs(cuda):
    torch = cuda
    from paper_0810_3286_gb300 import Solver
    p = planted_problem(120, 90, 3, 2000, seed=5)
    s = Solver(p.n1, p.n2, torch.from_numpy(p.rows).cuda(), torch.from_numpy(p.cols).cuda(),
               torch.from_numpy(p.vals).cuda())
    rp, ci, cp, ri, c2r = s.structure()
    row_ptr, col_idx, _ = osp.csr_structure(p.n1, p.n2, p.rows, p.cols)
    assert np.array_equal(rp, row_ptr) and np.array_equal(ci, col_idx)
    s.close()


@pytest.mark.parametrize("n1,n2,m,seed", [(7, 9, 20, 0), (13, 5, 65, 1), (40, 33, 500, 3), (200, 200, 11850, 0),
                                          (1000, 1000, 119400, 1), (3, 2, 6, 4), (2000, 3000, 1, 5)])
def test_sampler_bit_exact(cuda, n1, n2, m, seed):
    torch = cuda
    from paper_0810_3286_gb300 import sample_omega
    r = torch.empty(m, dtype=torch.int32, device="cuda")
    c = torch.empty(m, dtype=torch.int32, device="cuda")
    sample_omega(n1, n2, m, seed, r, c)
    ro, co = oracle_sample_omega(n1, n2, m, seed)
    assert np.array_equal(r.cpu().numpy(), ro)
    assert np.array_equal(c.cpu().numpy(), co)


def test_sampler_full_size_30000(cuda):
    """The 30000 x 30000 workload: |Omega| = 6 r (2n - r) = 3,599,400 of 9e8 ids, bit-exact."""
    torch = cuda
    from paper_0810_3286_gb300 import sample_omega
    n, m = 30000, 3599400
    r = torch.empty(m, dtype=torch.int32, device="cuda")
    c = torch.empty(m, dtype=torch.int32, device="cuda")
    sample_omega(n, n, m, 11, r, c)
    ro, co = oracle_sample_omega(n, n, m, 11)
    assert np.array_equal(r.cpu().numpy(), ro)
    assert np.array_equal(c.cpu().numpy(), co)
