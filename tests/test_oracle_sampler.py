"""Pins of the oracle's random-keys sampler of Omega and of SplitMix64.

* SplitMix64 against its published reference outputs (tests/golden/splitmix64_vectors.txt).
* The heap selection against brute force: all keys, sorted, first m.
* Structure: m distinct, sorted, in range; m = 0 and m = n1 n2.
* Uniformity over m-subsets (Sec. 5.2.1 samples Omega uniformly among all sets of cardinality m):
  chi-square of the subset frequencies over many seeds on a tiny grid.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import sample_omega, splitmix64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_vectors.txt")


def _golden():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            s, i, v = line.split()
            out.append((int(s), int(i), int(v)))
    return out


def test_splitmix64_reference_vectors():
    vecs = _golden()
    assert len(vecs) >= 8
    for seed, idx, val in vecs:
        assert splitmix64(seed, idx) == val


@pytest.mark.parametrize("n1,n2,m,seed", [(7, 9, 20, 0), (13, 5, 64, 1), (1, 50, 7, 2), (40, 33, 500, 3)])
def test_heap_selection_matches_brute_force(n1, n2, m, seed):
    N = n1 * n2
    keys = [(splitmix64(seed, i + 1), i) for i in range(N)]
    keys.sort()
    ids = sorted(i for _, i in keys[:m])
    rows, cols = sample_omega(n1, n2, m, seed)
    assert list(rows.astype(np.int64) * n2 + cols) == ids


def test_structure_and_edges():
    rows, cols = sample_omega(300, 200, 5000, 9)
    ids = rows.astype(np.int64) * 200 + cols
    assert ids.size == 5000 and np.all(np.diff(ids) > 0)
    assert rows.min() >= 0 and rows.max() < 300 and cols.min() >= 0 and cols.max() < 200
    r0, c0 = sample_omega(5, 5, 0, 1)
    assert r0.size == 0
    rows, cols = sample_omega(4, 6, 24, 1)
    assert np.array_equal(rows.astype(np.int64) * 6 + cols, np.arange(24))
    with pytest.raises(ValueError):
        sample_omega(4, 6, 25, 1)


def test_uniform_over_subsets():
    n1, n2, m = 2, 3, 2
    subsets = {s: 0 for s in itertools.combinations(range(n1 * n2), m)}
    trials = 6000
    for seed in range(trials):
        rows, cols = sample_omega(n1, n2, m, seed)
        subsets[tuple(int(v) for v in rows.astype(np.int64) * n2 + cols)] += 1
    counts = np.array(list(subsets.values()), dtype=float)
    expected = trials / len(subsets)
    chi2 = float(np.sum((counts - expected) ** 2 / expected))
    # 14 degrees of freedom: P(chi2 > 36.1) ~ 1e-3
    assert chi2 < 36.1
