"""Float64 CPU oracle of the SVT method.  TEST INFRASTRUCTURE, not part of the product.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this package.
It shares no code with the CUDA path (paper_0810_3286_gb300), and the CUDA path never imports
it.  Every function cites the passage of the paper it follows:

  oracle.svt      Algorithm 1 (Sec. 5.1.5), the shrink operator D_tau (Sec. 2.1, eq. (2.2)),
                  the kicking device (Sec. 5.1.3), the stopping rule (Sec. 5.1.4)
  oracle.sparse   Omega storage, Y V / Y^T U products, X on Omega, the dual update
  oracle._clib    one-sided Jacobi SVD, SplitMix64, the random-keys sampler of Omega (C)

Pins against values fixed by the paper and by mathematics live in tests/test_oracle_*.py.
"""
from . import sparse, svt
from ._clib import jacobi_svd, sample_omega, splitmix64

__all__ = ["sparse", "svt", "jacobi_svd", "sample_omega", "splitmix64"]
