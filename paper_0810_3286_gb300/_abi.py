"""ctypes declarations of the libsvt C-ABI (include/svt.h).  Argument marshalling only.

The shared library is loaded from paper_0810_3286_gb300/_build/libsvt.so.  There is no fallback:
if the library is missing or cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsvt.so")

SVT_OK = 0
SVT_ERR_ARG = 1
SVT_ERR_DUP_INDEX = 2
SVT_ERR_OOM = 3
SVT_ERR_CUDA = 4
SVT_ERR_RANK_LIMIT = 5
SVT_ERR_NOT_CONVERGED = 6
SVT_ERR_NUMERIC = 7
SVT_ERR_TIMEOUT = 8
SVT_ERR_INTERNAL = 9
SVT_STOPPED = 10

STATUS_NAMES = {
    0: "SVT_OK", 1: "SVT_ERR_ARG", 2: "SVT_ERR_DUP_INDEX", 3: "SVT_ERR_OOM", 4: "SVT_ERR_CUDA",
    5: "SVT_ERR_RANK_LIMIT", 6: "SVT_ERR_NOT_CONVERGED", 7: "SVT_ERR_NUMERIC", 8: "SVT_ERR_TIMEOUT",
    9: "SVT_ERR_INTERNAL", 10: "SVT_STOPPED",
}

SVT_FP64 = 0
SVT_FP32 = 1
SVT_BF16 = 2

SVT_SHRINK_LANCZOS = 0
SVT_SHRINK_RANDOMIZED = 1


class svt_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("block", ctypes.c_int),
        ("ell", ctypes.c_int),
        ("k_max", ctypes.c_int),
        ("lanczos_steps", ctypes.c_int),
        ("max_cycles", ctypes.c_int),
        ("lanczos_tol", ctypes.c_double),
        ("indices_on_device", ctypes.c_int),
        ("use_graphs", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("stream", ctypes.c_void_p),
        ("fused_orth", ctypes.c_int),
        ("restart_steps", ctypes.c_int),
        ("bf16_switch", ctypes.c_double),
        ("orth_grid", ctypes.c_int),
        ("orth_repass", ctypes.c_double),
        ("device_alloc", ctypes.c_void_p),
        ("device_free", ctypes.c_void_p),
        ("alloc_user", ctypes.c_void_p),
        ("shrink_engine", ctypes.c_int),
        ("rsvd_oversample", ctypes.c_int),
        ("rsvd_power", ctypes.c_int),
        ("rsvd_seed", ctypes.c_uint64),
        ("device_loop", ctypes.c_int),
        ("orth_tf32", ctypes.c_int),
        ("jacobi_cluster", ctypes.c_int),
    ]


class svt_step_info(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int64),
        ("r", ctypes.c_int),
        ("s", ctypes.c_int),
        ("passes", ctypes.c_int),
        ("lanczos_cycles", ctypes.c_int),
        ("spmm_calls", ctypes.c_int),
        ("residual", ctypes.c_double),
        ("sigma1", ctypes.c_double),
        ("ms", ctypes.c_double),
    ]


class svt_result(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int64),
        ("k0", ctypes.c_int64),
        ("rank", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("residual", ctypes.c_double),
        ("norm2_M", ctypes.c_double),
        ("normF_M", ctypes.c_double),
        ("ms", ctypes.c_double),
        ("spmm_calls", ctypes.c_int64),
        ("lanczos_cycles", ctypes.c_int64),
    ]


class svt_batch_options(ctypes.Structure):
    _fields_ = [
        ("spmm_grid", ctypes.c_int),
        ("update_grid", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("concurrent", ctypes.c_int),
    ]


_vp = ctypes.c_void_p
# svt_options.device_alloc / device_free
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_i32p = ctypes.POINTER(ctypes.c_int32)
_dp = ctypes.POINTER(ctypes.c_double)
_ctxp = ctypes.c_void_p

# name -> (restype, argtypes)
class svt_server_options(ctypes.Structure):
    _fields_ = [
        ("slots", ctypes.c_int),
        ("device_budget", ctypes.c_size_t),
        ("keep_factors", ctypes.c_int),
        ("dry_run", ctypes.c_int),
    ]


class svt_job(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64),
        ("n", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("rows", ctypes.c_void_p),
        ("cols", ctypes.c_void_p),
        ("vals", ctypes.c_void_p),
        ("tau", ctypes.c_double),
        ("delta", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("max_rank", ctypes.c_int),
        ("noise_sigma", ctypes.c_double),
        ("noise_eps", ctypes.c_double),
        ("opt", svt_options),
        ("dry_run_us", ctypes.c_int64),
        ("dry_run_bytes", ctypes.c_size_t),
    ]


class svt_job_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("iterations", ctypes.c_int64),
        ("rank", ctypes.c_int),
        ("residual", ctypes.c_double),
        ("t_submit_ms", ctypes.c_double),
        ("t_start_ms", ctypes.c_double),
        ("t_end_ms", ctypes.c_double),
        ("device_bytes", ctypes.c_size_t),
    ]


class svt_server_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64),
        ("completed", ctypes.c_int64),
        ("failed", ctypes.c_int64),
        ("queued", ctypes.c_int64),
        ("running", ctypes.c_int64),
        ("p50_ms", ctypes.c_double),
        ("p99_ms", ctypes.c_double),
        ("mean_ms", ctypes.c_double),
        ("solves_per_s", ctypes.c_double),
        ("peak_bytes", ctypes.c_size_t),
        ("peak_running", ctypes.c_int),
    ]


PROTOTYPES = {
    "svt_default_options": (None, [ctypes.POINTER(svt_options)]),
    "svt_create": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp,
                                  ctypes.POINTER(svt_options), ctypes.POINTER(_ctxp)]),
    "svt_destroy": (None, [_ctxp]),
    "svt_last_error": (ctypes.c_char_p, [_ctxp]),
    "svt_configure": (ctypes.c_int, [_ctxp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int64]),
    "svt_step": (ctypes.c_int, [_ctxp, ctypes.POINTER(svt_step_info)]),
    "svt_solve": (ctypes.c_int, [_ctxp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                 ctypes.POINTER(svt_result)]),
    "svt_get_rank": (ctypes.c_int, [_ctxp, ctypes.POINTER(ctypes.c_int)]),
    "svt_get_factors": (ctypes.c_int, [_ctxp, _vp, _vp, _vp, ctypes.c_int]),
    "svt_get_Y": (ctypes.c_int, [_ctxp, _vp]),
    "svt_set_Y": (ctypes.c_int, [_ctxp, _vp]),
    "svt_get_structure": (ctypes.c_int, [_ctxp, _vp, _vp, _vp, _vp, _vp]),
    "svt_shrink": (ctypes.c_int, [_ctxp, ctypes.c_double, ctypes.POINTER(ctypes.c_int), _vp]),
    "svt_apply_Y": (ctypes.c_int, [_ctxp, _vp, ctypes.c_int, _vp]),
    "svt_apply_Yt": (ctypes.c_int, [_ctxp, _vp, ctypes.c_int, _vp]),
    "svt_sddmm_update": (ctypes.c_int, [_ctxp, _vp, _vp, ctypes.c_int, ctypes.c_double, _vp, _vp, _dp]),
    "svt_sample_omega": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, _vp, _vp,
                                        _vp]),
    "svt_save_state": (ctypes.c_int, [_ctxp, _vp, ctypes.POINTER(ctypes.c_size_t)]),
    "svt_load_state": (ctypes.c_int, [_ctxp, _vp, ctypes.c_size_t]),
    "svt_kernel_launches": (ctypes.c_int64, [_ctxp]),
    "svt_set_profile": (ctypes.c_int, [_ctxp, ctypes.c_uint]),
    "svt_estimate_device_bytes": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                    ctypes.POINTER(svt_options)]),
    "svt_server_default_options": (None, [ctypes.POINTER(svt_server_options)]),
    "svt_server_create": (ctypes.c_int, [ctypes.POINTER(svt_server_options), ctypes.POINTER(ctypes.c_void_p)]),
    "svt_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(svt_job), ctypes.POINTER(ctypes.c_int64)]),
    "svt_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(svt_job_result), _vp, _vp, _vp,
                                       ctypes.c_int]),
    "svt_server_drain": (ctypes.c_int, [ctypes.c_void_p]),
    "svt_server_stats_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(svt_server_stats)]),
    "svt_server_destroy": (None, [ctypes.c_void_p]),
    "svt_set_dantzig": (ctypes.c_int, [_ctxp, ctypes.c_double]),
    "svt_set_noise_stop": (ctypes.c_int, [_ctxp, ctypes.c_double, ctypes.c_double]),
    "svt_get_profile": (ctypes.c_int, [_ctxp, _vp, _vp, _vp, _vp]),
    "svt_get_counters": (ctypes.c_int, [_ctxp, _vp, ctypes.c_int]),
    "svt_set_barrier_spins": (ctypes.c_int, [_ctxp, ctypes.c_int]),
    "svt_set_tau": (ctypes.c_int, [_ctxp, ctypes.c_double]),
    "svt_batch_default_options": (None, [ctypes.POINTER(svt_batch_options)]),
    "svt_batch_solve": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(svt_batch_options), _vp, _vp]),
    "svt_selftest_math": (ctypes.c_int, [ctypes.c_int64, _vp, _vp, _vp]),
    "svt_solve_continuation": (ctypes.c_int, [_ctxp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int, _vp, ctypes.POINTER(svt_result)]),
    "svt_sddmm_update_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _vp, _vp, _vp, _vp,
                                                _vp, ctypes.c_int, ctypes.c_double, _vp, _vp, _dp, _vp]),
    "svt_noalloc_last_error": (ctypes.c_char_p, []),
}

COUNTER_NAMES = ["lanczos_cycles", "spmm_calls", "svd_calls", "jacobi_sweeps", "deflated_columns",
                 "max_orth_defect", "kernel_launches", "relaxed_shrinks", "orth_repasses", "max_first_pass_defect", "device_loop_iterations"]

# kernel classes of svt_set_profile / svt_get_profile
PROF_CLASSES = ["spmm", "spmm_t", "gram", "block_update", "small", "jacobi", "combine", "sddmm_update", "orth"]

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libsvt.so and declare every entry point.  Raises OSError if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise OSError("libsvt.so not found at %s: build it with paper_0810_3286_gb300.build.build() "
                              "(there is no CPU fallback)" % path)
            L = ctypes.CDLL(path)
            for name, (res, args) in PROTOTYPES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class SVTError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES.get(status, status), message))
