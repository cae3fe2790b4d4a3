"""Seeded synthetic inputs for matrix completion (shared by the oracle, the tests and the bench).

This module holds no arithmetic of the SVT method itself: it only draws the planted problem
of the paper's experiments (Sec. 5.2.1): two i.i.d. N(0,1) factors M_L (n1 x r) and
M_R (n2 x r), M = M_L M_R^T, and a sampled set Omega of cardinality m drawn uniformly at
random among all subsets of that size, plus the sampled entries M_ij, (i,j) in Omega.
Optional additive Gaussian noise follows the noisy model of Sec. 5.2.1 (B = M + Z on Omega).

Everything is drawn from numpy's PCG64 generator seeded with the caller's seed, so the same
(n1, n2, r, m, seed) always yields bit-identical arrays on any host.
"""
from .planted import (PlantedProblem, planted_problem, config_problem, CONFIGS, dof, sample_count,
                      random_dense, random_sparse_pattern, serving_job)

__all__ = ["PlantedProblem", "planted_problem", "config_problem", "CONFIGS", "dof", "sample_count",
           "random_dense", "random_sparse_pattern", "serving_job"]
