"""Pins of the oracle's one-sided Jacobi SVD against closed forms, library routines and brute force.

The SVD is the building block of the shrink operator D_tau (Sec. 2.1, eq. (2.2)); these tests
pin it to values fixed by mathematics, not to itself.
"""
import math

import numpy as np
import pytest

from oracle import jacobi_svd


def _check_factorisation(A, U, s, V, tol=1e-13):
    scale = max(1.0, np.abs(A).max())
    assert np.abs((U * s) @ V.T - A).max() <= tol * scale * max(A.shape)
    k = s.shape[0]
    nz = s > 1e-12 * max(1.0, s[0] if k else 1.0)
    Un, Vn = U[:, nz], V[:, nz]
    assert np.abs(Un.T @ Un - np.eye(Un.shape[1])).max() <= 1e-13 * max(A.shape)
    assert np.abs(Vn.T @ Vn - np.eye(Vn.shape[1])).max() <= 1e-13 * max(A.shape)
    assert np.all(np.diff(s) <= 0)
    assert np.all(s >= 0)


@pytest.mark.parametrize("a,b,c,d", [(3.0, 1.0, -2.0, 4.0), (1.0, 0.0, 0.0, 1.0), (0.0, 5.0, 0.0, 0.0),
                                     (2.0, 2.0, 2.0, 2.0), (1e-3, 7.0, -7.0, 1e-3)])
def test_2x2_closed_form(a, b, c, d):
    # sigma_{1,2}^2 = (S +- sqrt(S^2 - 4 D^2)) / 2 with S = ||A||_F^2 and D = det A.
    A = np.array([[a, b], [c, d]])
    S = a * a + b * b + c * c + d * d
    D = a * d - b * c
    disc = math.sqrt(max(S * S - 4 * D * D, 0.0))
    s1 = math.sqrt((S + disc) / 2)
    s2 = math.sqrt(max((S - disc) / 2, 0.0))
    U, s, V = jacobi_svd(A)
    assert s[0] == pytest.approx(s1, rel=1e-14, abs=1e-14)
    assert s[1] == pytest.approx(s2, rel=1e-12, abs=1e-13)
    _check_factorisation(A, U, s, V)


def test_diagonal_and_permuted_diagonal():
    d = np.array([3.0, -7.0, 0.5, 2.0, -1e-3, 0.0])
    U, s, V = jacobi_svd(np.diag(d))
    assert np.array_equal(s, np.sort(np.abs(d))[::-1])
    rng = np.random.default_rng(1)
    P1 = np.eye(6)[rng.permutation(6)]
    P2 = np.eye(6)[rng.permutation(6)]
    A = P1 @ np.diag(d) @ P2
    U, s, V = jacobi_svd(A)
    assert np.array_equal(s, np.sort(np.abs(d))[::-1])
    _check_factorisation(A, U, s, V)


def _householder(rng, n):
    v = rng.standard_normal(n)
    v /= np.linalg.norm(v)
    return np.eye(n) - 2.0 * np.outer(v, v)


@pytest.mark.parametrize("m,n", [(9, 6), (6, 9), (12, 12)])
def test_known_spectrum(m, n):
    # A = H1 [diag(sigma); 0] H2 with Householder reflectors H1, H2: singular values are sigma.
    rng = np.random.default_rng(m * 100 + n)
    k = min(m, n)
    sigma = np.sort(rng.uniform(0.1, 10.0, k))[::-1]
    S = np.zeros((m, n))
    S[:k, :k] = np.diag(sigma)
    A = _householder(rng, m) @ _householder(rng, m) @ S @ _householder(rng, n)
    U, s, V = jacobi_svd(A)
    assert np.abs(s - sigma).max() <= 1e-13 * sigma[0]
    _check_factorisation(A, U, s, V)


@pytest.mark.parametrize("m,n,seed", [(1, 1, 0), (1, 5, 1), (5, 1, 2), (40, 25, 3), (25, 40, 4), (64, 64, 5)])
def test_against_lapack(m, n, seed):
    # A special case that reduces to a library routine: numpy.linalg.svd (LAPACK gesdd).
    A = np.random.default_rng(seed).standard_normal((m, n))
    U, s, V = jacobi_svd(A)
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.abs(s - ref).max() <= 1e-13 * max(1.0, ref[0])
    _check_factorisation(A, U, s, V)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_brute_force_small(n):
    # sigma_i^2 are the eigenvalues of A^T A (symmetric eigensolver, independent of Jacobi SVD).
    A = np.random.default_rng(10 + n).standard_normal((n, n))
    _, s, _ = jacobi_svd(A)
    ev = np.sort(np.linalg.eigvalsh(A.T @ A))[::-1]
    assert np.abs(s * s - ev).max() <= 1e-12 * ev[0]


def test_rank_deficient_and_zero():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((10, 3)) @ rng.standard_normal((3, 8))
    U, s, V = jacobi_svd(A)
    assert np.all(s[3:] <= 1e-13 * s[0])
    assert np.abs((U * s) @ V.T - A).max() <= 1e-12
    U, s, V = jacobi_svd(np.zeros((4, 3)))
    assert np.array_equal(s, np.zeros(3))
