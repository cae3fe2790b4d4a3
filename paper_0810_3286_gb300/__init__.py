"""GB300-native Singular Value Thresholding (Cai, Candes & Shen 2008): Python binding of libsvt.

Thin marshalling layer over the C-ABI in include/svt.h.  Every step of the SVT hot path runs in
the library's CUDA kernels; PyTorch is used here only to hold device buffers and to name the
CUDA stream.  If libsvt.so is missing, the calls raise (there is no CPU fallback).

    from paper_0810_3286_gb300 import Solver
    s = Solver(m, n, rows, cols, m_vals, precision="fp64")   # numpy or torch inputs
    res = s.solve(tau, delta, eps=1e-4, max_rank=20)
    U, d, V = s.factors()                                    # X = U diag(d) V^T
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _abi
from ._abi import (SVT_BF16, SVT_ERR_NOT_CONVERGED, SVT_FP32, SVT_FP64, SVT_OK, SVT_STOPPED, SVTError, svt_options,
                   svt_result, svt_step_info)

__all__ = ["Solver", "SVTError", "sample_omega", "library", "SVT_FP64", "SVT_FP32", "SVT_BF16", "StepInfo",
           "SolveResult"]


def library():
    """The loaded libsvt (raises if it has not been built)."""
    return _abi.load()


def _check(status: int, where: str, ctx=None, allow=()):
    if status == SVT_OK or status in allow:
        return status
    L = library()
    msg = L.svt_last_error(ctx).decode(errors="replace")
    raise SVTError(status, where, msg)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _ptr(a) -> int:
    """Address of a contiguous numpy array (host) or torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError("expected numpy array or torch tensor")


class StepInfo(dict):
    pass


class SolveResult(dict):
    pass


class Solver:
    """One completion problem: Omega, the sampled entries and the SVT state (svt_ctx)."""

    def __init__(self, m: int, n: int, rows, cols, m_vals, precision: str = "fp64", stream=None, ell: int = 5,
                 k_max: int = 1000, lanczos_steps: int = 3, lanczos_tol: float = 0.0, seed: int = 0x5EED5EED,
                 max_cycles: int = 40, use_graphs: bool = True, fused_orth: bool = True, block: int = 0,
                 restart_steps: int = 0, bf16_switch: float = 1e-2, orth_grid: int = 0, orth_repass: float = 0.0,
                 allocator=None, shrink_engine: str = "lanczos", rsvd_oversample: int = 8, rsvd_power: int = 1,
                 rsvd_seed: int = 0, device_loop: bool = True, orth_tf32: Optional[bool] = None,
                 jacobi_cluster: int = 0):
        L = library()
        opt = svt_options()
        L.svt_default_options(ctypes.byref(opt))
        opt.precision = {"fp64": SVT_FP64, "fp32": SVT_FP32, "bf16": SVT_BF16}[precision]
        opt.ell = ell
        opt.k_max = k_max
        opt.lanczos_steps = lanczos_steps
        opt.lanczos_tol = lanczos_tol
        opt.seed = seed
        opt.max_cycles = max_cycles
        opt.use_graphs = 1 if use_graphs else 0
        opt.fused_orth = 1 if fused_orth else 0
        opt.block = int(block)
        opt.restart_steps = int(restart_steps)
        opt.bf16_switch = float(bf16_switch)
        opt.orth_grid = int(orth_grid)
        opt.orth_repass = float(orth_repass)
        opt.shrink_engine = {"lanczos": _abi.SVT_SHRINK_LANCZOS, "randomized": _abi.SVT_SHRINK_RANDOMIZED}[shrink_engine]
        opt.rsvd_oversample = int(rsvd_oversample)
        opt.rsvd_power = int(rsvd_power)
        opt.rsvd_seed = int(rsvd_seed) & (2**64 - 1)
        opt.device_loop = 1 if device_loop else 0
        opt.orth_tf32 = 0 if orth_tf32 is None else (1 if orth_tf32 else -1)
        opt.jacobi_cluster = jacobi_cluster
        if allocator is not None:
            # (alloc(bytes) -> int device pointer or 0, free(ptr)); the ctypes thunks must outlive
            # the context
            self._alloc_cbs = (_abi.ALLOC_FN(lambda nbytes, _u: int(allocator[0](nbytes)) or None),
                               _abi.FREE_FN(lambda ptr, _u: allocator[1](ptr)))
            opt.device_alloc = ctypes.cast(self._alloc_cbs[0], ctypes.c_void_p)
            opt.device_free = ctypes.cast(self._alloc_cbs[1], ctypes.c_void_p)
        sh = _stream_handle(stream)
        opt.stream = sh
        on_device = hasattr(rows, "is_cuda") and rows.is_cuda
        if on_device:
            import torch
            if not (cols.is_cuda and m_vals.is_cuda):
                raise ValueError("rows, cols and m_vals must be in the same memory space")
            if rows.dtype != torch.int32 or cols.dtype != torch.int32 or m_vals.dtype != torch.float64:
                raise TypeError("device inputs must be int32, int32, float64")
            opt.indices_on_device = 1
            keep = (rows, cols, m_vals)
        else:
            if hasattr(rows, "numpy"):
                rows, cols, m_vals = rows.numpy(), cols.numpy(), m_vals.numpy()
            keep = (np.ascontiguousarray(rows, dtype=np.int32), np.ascontiguousarray(cols, dtype=np.int32),
                    np.ascontiguousarray(m_vals, dtype=np.float64))
        self.m, self.n = int(m), int(n)
        self.nnz = int(keep[0].shape[0])
        self.precision = precision
        ctx = ctypes.c_void_p()
        st = L.svt_create(self.m, self.n, self.nnz, _ptr(keep[0]), _ptr(keep[1]), _ptr(keep[2]), ctypes.byref(opt),
                          ctypes.byref(ctx))
        _check(st, "svt_create", None)
        self._ctx = ctx
        self._L = L

    # -- lifetime --------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._L.svt_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- Algorithm 1 -----------------------------------------------------------------------------
    def configure(self, tau: float = 0.0, delta: float = 0.0, eps: float = 1e-4, max_rank: int = 27, k0: int = -1):
        _check(self._L.svt_configure(self._ctx, tau, delta, eps, max_rank, k0), "svt_configure", self._ctx)

    def set_noise_stop(self, sigma: float, eps_noise: float = 0.0):
        """Stop at the first X^k with ||P_Omega(X^k - B)||_F^2 <= (1 + eps_noise) |Omega| sigma^2
        (noisy data, eq. (5.10)); sigma <= 0 restores the relative-residual rule eq. (5.5)."""
        _check(self._L.svt_set_noise_stop(self._ctx, sigma, eps_noise), "svt_set_noise_stop", self._ctx)

    def set_dantzig(self, E: float):
        """Matrix Dantzig selector (Sec. 3.3): constraints |B - X| <= E on Omega, multipliers Y_+ and
        Y_- (iteration (iterDS2)); E <= 0 returns to Algorithm 1.  Configure again afterwards."""
        _check(self._L.svt_set_dantzig(self._ctx, E), "svt_set_dantzig", self._ctx)

    def step(self) -> StepInfo:
        info = svt_step_info()
        st = self._L.svt_step(self._ctx, ctypes.byref(info))
        _check(st, "svt_step", self._ctx, allow=(SVT_STOPPED,))
        out = StepInfo({f: getattr(info, f) for f, _ in svt_step_info._fields_})
        out["stopped"] = st == SVT_STOPPED
        return out

    def solve(self, tau: float = 0.0, delta: float = 0.0, eps: float = 1e-4, max_rank: int = 27,
              raise_on_nonconvergence: bool = True) -> SolveResult:
        res = svt_result()
        st = self._L.svt_solve(self._ctx, tau, delta, eps, max_rank, ctypes.byref(res))
        allow = () if raise_on_nonconvergence else (SVT_ERR_NOT_CONVERGED,)
        _check(st, "svt_solve", self._ctx, allow=allow)
        return SolveResult({f: getattr(res, f) for f, _ in svt_result._fields_})

    def set_tau(self, tau: float):
        """Continuation (Sec. 6): tau for the following steps, keeping Y, X and the warm start."""
        _check(self._L.svt_set_tau(self._ctx, tau), "svt_set_tau", self._ctx)

    def solve_continuation(self, taus, delta: float = 0.0, eps: float = 1e-4, max_rank: int = 27,
                           raise_on_nonconvergence: bool = True):
        """Algorithm 1 at taus[0] (with the kick), then at each later tau from the previous stage's
        dual iterate (Sec. 6).  Returns (SolveResult, per-stage iterations)."""
        t = np.ascontiguousarray(taus, dtype=np.float64)
        stages = np.zeros(t.shape[0], dtype=np.int64)
        res = svt_result()
        st = self._L.svt_solve_continuation(self._ctx, t.ctypes.data, int(t.shape[0]), delta, eps, max_rank,
                                            stages.ctypes.data, ctypes.byref(res))
        allow = () if raise_on_nonconvergence else (SVT_ERR_NOT_CONVERGED,)
        _check(st, "svt_solve_continuation", self._ctx, allow=allow)
        return SolveResult({f: getattr(res, f) for f, _ in svt_result._fields_}), stages.tolist()

    def shrink(self, tau: float = 0.0):
        """D_tau of the current Y; returns (rank, singular values > tau)."""
        r = ctypes.c_int()
        sig = np.zeros(64)
        _check(self._L.svt_shrink(self._ctx, tau, ctypes.byref(r), sig.ctypes.data), "svt_shrink", self._ctx)
        return r.value, sig[:r.value].copy()

    # -- state access ----------------------------------------------------------------------------
    def rank(self) -> int:
        r = ctypes.c_int()
        _check(self._L.svt_get_rank(self._ctx, ctypes.byref(r)), "svt_get_rank", self._ctx)
        return r.value

    def factors(self):
        r = self.rank()
        U = np.zeros((self.m, max(r, 1)))
        d = np.zeros(max(r, 1))
        V = np.zeros((self.n, max(r, 1)))
        _check(self._L.svt_get_factors(self._ctx, U.ctypes.data, d.ctypes.data, V.ctypes.data, max(r, 1)),
               "svt_get_factors", self._ctx)
        return U[:, :r].copy(), d[:r].copy(), V[:, :r].copy()

    def get_Y(self) -> np.ndarray:
        y = np.zeros(self.nnz)
        _check(self._L.svt_get_Y(self._ctx, y.ctypes.data), "svt_get_Y", self._ctx)
        return y

    def set_Y(self, y) -> None:
        y = np.ascontiguousarray(y, dtype=np.float64)
        if y.shape != (self.nnz,):
            raise ValueError("y must have nnz entries")
        _check(self._L.svt_set_Y(self._ctx, y.ctypes.data), "svt_set_Y", self._ctx)

    def structure(self):
        rp = np.zeros(self.m + 1, np.int32)
        ci = np.zeros(self.nnz, np.int32)
        cp = np.zeros(self.n + 1, np.int32)
        ri = np.zeros(self.nnz, np.int32)
        c2r = np.zeros(self.nnz, np.int32)
        _check(self._L.svt_get_structure(self._ctx, rp.ctypes.data, ci.ctypes.data, cp.ctypes.data, ri.ctypes.data,
                                         c2r.ctypes.data), "svt_get_structure", self._ctx)
        return rp, ci, cp, ri, c2r

    # -- kernel-level entry points (torch device tensors, float64, contiguous) -------------------
    def apply_Y(self, V, W):
        _check(self._L.svt_apply_Y(self._ctx, _ptr(V), int(V.shape[1]), _ptr(W)), "svt_apply_Y", self._ctx)

    def apply_Yt(self, U, Z):
        _check(self._L.svt_apply_Yt(self._ctx, _ptr(U), int(U.shape[1]), _ptr(Z)), "svt_apply_Yt", self._ctx)

    def sddmm_update(self, Ut, V, delta: float, y_in, y_out) -> float:
        res2 = ctypes.c_double()
        r = int(Ut.shape[1]) if Ut is not None else 0
        _check(self._L.svt_sddmm_update(self._ctx, _ptr(Ut) if r else None, _ptr(V) if r else None, r, delta,
                                        _ptr(y_in), _ptr(y_out), ctypes.byref(res2)), "svt_sddmm_update", self._ctx)
        return res2.value

    def save_state(self) -> bytes:
        n = ctypes.c_size_t()
        _check(self._L.svt_save_state(self._ctx, None, ctypes.byref(n)), "svt_save_state", self._ctx)
        buf = ctypes.create_string_buffer(n.value)
        _check(self._L.svt_save_state(self._ctx, buf, ctypes.byref(n)), "svt_save_state", self._ctx)
        return buf.raw[:n.value]

    def load_state(self, blob: bytes) -> None:
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(self._L.svt_load_state(self._ctx, buf, len(blob)), "svt_load_state", self._ctx)

    def kernel_launches(self) -> int:
        return int(self._L.svt_kernel_launches(self._ctx))

    def counters(self):
        """Cumulative solver counters (see svt_get_counters)."""
        n = len(_abi.COUNTER_NAMES)
        out = np.zeros(n)
        _check(self._L.svt_get_counters(self._ctx, out.ctypes.data, n), "svt_get_counters", self._ctx)
        return dict(zip(_abi.COUNTER_NAMES, out.tolist()))

    def set_profile(self, classes=()):
        """Bracket the launches of the named kernel classes with CUDA events (see PROF_CLASSES)."""
        mask = 0
        for c in classes:
            mask |= 1 << _abi.PROF_CLASSES.index(c)
        _check(self._L.svt_set_profile(self._ctx, mask), "svt_set_profile", self._ctx)

    def profile(self):
        """{class: (launch groups, total ms, algorithmic bytes, flops)} since the last set_profile."""
        n = len(_abi.PROF_CLASSES)
        launches = np.zeros(n, np.int64)
        ms = np.zeros(n)
        by = np.zeros(n)
        fl = np.zeros(n)
        _check(self._L.svt_get_profile(self._ctx, launches.ctypes.data, ms.ctypes.data, by.ctypes.data,
                                       fl.ctypes.data), "svt_get_profile", self._ctx)
        return {c: (int(launches[i]), float(ms[i]), float(by[i]), float(fl[i]))
                for i, c in enumerate(_abi.PROF_CLASSES)}


def batch_solve(solvers, tau=None, delta=None, eps: float = 1e-4, max_rank: int = 27, autotune: bool = False,
                spmm_grid: int = 0, update_grid: int = 0, concurrent: bool = True):
    """svt_batch_solve: Algorithm 1 for the problems of `solvers` (1 to 32 Solver objects of one
    precision) at once, in lockstep, with the sparse products and the fused updates of all jobs as
    single launches over the job list.  tau / delta: per-job sequences or None (defaults).  Returns
    (list of SolveResult, list of per-job status codes); raises SVTError on a bad batch."""
    L = library()
    n = len(solvers)
    ctxs = (ctypes.c_void_p * n)(*[s._ctx.value for s in solvers])
    t = None if tau is None else np.ascontiguousarray(tau, dtype=np.float64)
    d = None if delta is None else np.ascontiguousarray(delta, dtype=np.float64)
    opt = _abi.svt_batch_options()
    L.svt_batch_default_options(ctypes.byref(opt))
    opt.autotune = 1 if autotune else 0
    opt.spmm_grid = spmm_grid
    opt.update_grid = update_grid
    opt.concurrent = 1 if concurrent else 0
    res = (svt_result * n)()
    st = np.zeros(n, dtype=np.int32)
    rc = L.svt_batch_solve(ctypes.cast(ctxs, ctypes.c_void_p), n, None if t is None else t.ctypes.data,
                           None if d is None else d.ctypes.data, eps, max_rank, ctypes.byref(opt),
                           ctypes.cast(res, ctypes.c_void_p), st.ctypes.data)
    if rc == _abi.SVT_ERR_ARG:
        _check(rc, "svt_batch_solve", solvers[0]._ctx if n else None)
    out = [SolveResult({f: getattr(r, f) for f, _ in svt_result._fields_}) for r in res]
    return out, st.tolist()


def sample_omega(m: int, n: int, nnz: int, seed: int, rows_out, cols_out, stream=None) -> None:
    """Device random-keys sampler of Omega into int32 device tensors rows_out/cols_out."""
    L = library()
    _check(L.svt_sample_omega(m, n, nnz, seed & (2**64 - 1), _ptr(rows_out), _ptr(cols_out),
                              _stream_handle(stream)), "svt_sample_omega", None)
