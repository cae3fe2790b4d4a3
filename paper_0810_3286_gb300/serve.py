"""Python binding of the serving runtime (include/svt_serve.h): argument marshalling only.

    srv = Server(slots=8)                       # device budget: 90 % of the free memory
    jid = srv.submit(m, n, rows, cols, vals)    # host arrays, copied
    res = srv.wait(jid)                         # blocks; {"status", "iterations", "rank", ...}
    srv.stats()                                 # {"p50_ms", "p99_ms", "solves_per_s", ...}
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import SVT_BF16, SVT_FP32, SVT_FP64, SVTError


class Server:
    def __init__(self, slots: int = 8, device_budget: int = 0, keep_factors: bool = False, dry_run: bool = False):
        from . import library
        self._L = library()
        o = _abi.svt_server_options()
        self._L.svt_server_default_options(ctypes.byref(o))
        o.slots = int(slots)
        o.device_budget = int(device_budget)
        o.keep_factors = 1 if keep_factors else 0
        o.dry_run = 1 if dry_run else 0
        h = ctypes.c_void_p()
        st = self._L.svt_server_create(ctypes.byref(o), ctypes.byref(h))
        if st != 0:
            raise SVTError(st, "svt_server_create", "")
        self._h = h
        self._keep = keep_factors
        self._shapes = {}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.svt_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, m: int, n: int, rows=None, cols=None, vals=None, tau: float = 0.0, delta: float = 0.0,
               eps: float = 1e-4, max_rank: int = 64, precision: str = "fp32", noise_sigma: float = 0.0,
               noise_eps: float = 0.0, dry_run_us: int = 0, dry_run_bytes: int = 0, nnz: int = 0,
               k_max: int = 1000) -> int:
        j = _abi.svt_job()
        keep = []
        if rows is not None:
            r = np.ascontiguousarray(rows, dtype=np.int32)
            c = np.ascontiguousarray(cols, dtype=np.int32)
            v = np.ascontiguousarray(vals, dtype=np.float64)
            keep = [r, c, v]
            j.rows, j.cols, j.vals = r.ctypes.data, c.ctypes.data, v.ctypes.data
            nnz = r.shape[0]
        j.m, j.n, j.nnz = int(m), int(n), int(nnz)
        j.tau, j.delta, j.eps, j.max_rank = float(tau), float(delta), float(eps), int(max_rank)
        j.noise_sigma, j.noise_eps = float(noise_sigma), float(noise_eps)
        self._L.svt_default_options(ctypes.byref(j.opt))
        j.opt.precision = {"fp64": SVT_FP64, "fp32": SVT_FP32, "bf16": SVT_BF16}[precision]
        j.opt.k_max = int(k_max)
        j.dry_run_us, j.dry_run_bytes = int(dry_run_us), int(dry_run_bytes)
        jid = ctypes.c_int64()
        st = self._L.svt_server_submit(self._h, ctypes.byref(j), ctypes.byref(jid))
        del keep
        if st != 0:
            raise SVTError(st, "svt_server_submit", "")
        self._shapes[jid.value] = (int(m), int(n))
        return jid.value

    def wait(self, job_id: int):
        """Result dict; with keep_factors also U, d (sigma - tau), V."""
        res = _abi.svt_job_result()
        m, n = self._shapes.pop(job_id, (0, 0))
        cap = 64
        U = np.zeros((m, cap)) if self._keep else None
        d = np.zeros(cap) if self._keep else None
        V = np.zeros((n, cap)) if self._keep else None
        st = self._L.svt_server_wait(self._h, job_id, ctypes.byref(res),
                                     U.ctypes.data if U is not None else None,
                                     d.ctypes.data if d is not None else None,
                                     V.ctypes.data if V is not None else None, cap)
        if st != 0:
            raise SVTError(st, "svt_server_wait", "")
        out = {f: getattr(res, f) for f, _ in _abi.svt_job_result._fields_}
        if self._keep:
            r = res.rank
            out["U"], out["d"], out["V"] = U[:, :r].copy(), d[:r].copy(), V[:, :r].copy()
        return out

    def drain(self):
        self._L.svt_server_drain(self._h)

    def stats(self):
        s = _abi.svt_server_stats()
        self._L.svt_server_stats_get(self._h, ctypes.byref(s))
        return {f: getattr(s, f) for f, _ in _abi.svt_server_stats._fields_}
