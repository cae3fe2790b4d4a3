"""ctypes binding of the oracle's C routines (test infrastructure only)."""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            L.oracle_jacobi_svd.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ctypes.c_double,
                                            ctypes.c_int]
            L.oracle_jacobi_svd.restype = ctypes.c_int
            L.oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.oracle_splitmix64.restype = ctypes.c_uint64
            ip = ctypes.POINTER(ctypes.c_int32)
            L.oracle_sample_omega.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                              ip, ip]
            L.oracle_sample_omega.restype = ctypes.c_int
            _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def jacobi_svd(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Thin SVD A = U diag(s) V^T by one-sided Jacobi (float64); s sorted decreasing."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    k = min(m, n)
    U = np.zeros((m, k))
    s = np.zeros(k)
    V = np.zeros((n, k))
    if k == 0:
        return U, s, V
    sweeps = lib().oracle_jacobi_svd(m, n, _dptr(A), _dptr(U), _dptr(s), _dptr(V), tol, max_sweeps)
    if sweeps < 0:
        raise RuntimeError("oracle_jacobi_svd failed (code %d)" % sweeps)
    return U, s, V


def splitmix64(seed: int, index: int) -> int:
    return int(lib().oracle_splitmix64(seed & (2**64 - 1), index & (2**64 - 1)))


def sample_omega(n1: int, n2: int, m: int, seed: int):
    rows = np.zeros(m, dtype=np.int32)
    cols = np.zeros(m, dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int32)
    rc = lib().oracle_sample_omega(n1, n2, m, seed & (2**64 - 1), rows.ctypes.data_as(ip), cols.ctypes.data_as(ip))
    if rc != 0:
        raise ValueError("oracle_sample_omega failed (code %d)" % rc)
    return rows, cols
