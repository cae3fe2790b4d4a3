"""Pins of the oracle's shrink operator D_tau (Sec. 2.1).

* eq. (2.2) on inputs whose SVD is known (scalar, diagonal): soft thresholding of sigma.
* Theorem 2.1: D_tau(Y) is the prox of tau ||.||_*; the subgradient certificate
  Y - X = tau (U0 V0^T + W) with U0^T W = 0, W V0 = 0, ||W||_2 <= 1 (eq. (2.6)), and
  optimality of h0(X) = tau ||X||_* + 1/2 ||X - Y||_F^2 against random perturbations.
* A planted mistake (no positive part) is caught by the certificate.
"""
import numpy as np
import pytest

from oracle import svt as osvt


def _nuclear(X):
    return float(np.linalg.svd(X, compute_uv=False).sum())


def test_scalar_soft_threshold():
    for y, tau in [(5.0, 2.0), (-5.0, 2.0), (1.0, 2.0), (2.0, 2.0), (-0.5, 0.0)]:
        X = osvt.shrink_dense(np.array([[y]]), tau)
        assert X[0, 0] == pytest.approx(np.sign(y) * max(abs(y) - tau, 0.0), abs=1e-15)


def test_diagonal_soft_threshold():
    d = np.array([9.0, -4.0, 3.0, 0.5, -7.5])
    tau = 3.5
    X = osvt.shrink_dense(np.diag(d), tau)
    assert np.abs(X - np.diag(np.sign(d) * np.maximum(np.abs(d) - tau, 0.0))).max() <= 1e-14


def _certificate(Y, tau, shrink_fn):
    """W of eq. (2.6) for X = shrink_fn(Y, tau), using X's own SVD (numpy, independent of the
    shrink): U0, V0 span the singular vectors of X with nonzero singular values."""
    U, dd, V, _ = shrink_fn(Y, tau)
    X = (U * dd) @ V.T
    Ux, sx, Vxt = np.linalg.svd(X, full_matrices=False)
    keep = sx > 1e-10 * max(1.0, sx[0] if sx.size else 1.0)
    U0, V0 = Ux[:, keep], Vxt[keep].T
    W = (Y - X) / tau - U0 @ V0.T
    return U0, V0, W, X


@pytest.mark.parametrize("shape,tau,seed", [((12, 9), 2.5, 0), ((9, 12), 2.5, 1), ((20, 20), 4.0, 2),
                                            ((30, 18), 0.3, 3)])
def test_theorem_2_1_certificate(shape, tau, seed):
    Y = np.random.default_rng(seed).standard_normal(shape) * 2.0
    U0, V0, W, X = _certificate(Y, tau, osvt.shrink)
    assert np.abs(U0.T @ W).max() <= 1e-12
    assert np.abs(W @ V0).max() <= 1e-12
    assert np.linalg.norm(W, 2) <= 1.0 + 1e-12


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_prox_optimality(seed):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((10, 7)) * 3.0
    tau = 2.0
    X = osvt.shrink_dense(Y, tau)

    def h0(Z):
        return tau * _nuclear(Z) + 0.5 * float(np.sum((Z - Y) ** 2))

    base = h0(X)
    for _ in range(40):
        Z = rng.standard_normal(Y.shape)
        for t in (1e-4, 1e-2, 1.0):
            assert h0(X + t * Z) >= base - 1e-10


def test_planted_mistake_is_caught():
    """A shrink without the positive part (sigma - tau instead of (sigma - tau)_+) breaks eq. (2.6)."""
    def wrong_shrink(Y, tau):
        U, s, V = osvt.svd(Y)
        return U, s - tau, V, s

    Y = np.random.default_rng(5).standard_normal((10, 8)) * 2.0
    U0, V0, W, X = _certificate(Y, 2.0, wrong_shrink)
    ok = (np.abs(U0.T @ W).max() <= 1e-12 and np.abs(W @ V0).max() <= 1e-12
          and np.linalg.norm(W, 2) <= 1.0 + 1e-12)
    assert not ok
