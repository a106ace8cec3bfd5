"""ctypes declarations of the C ABI in include/mdhp.h (argument marshalling only).

Loading fails loudly: there is no CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "_build", "libmdhp.so")

NOALLOC_MAX_WINDOWS = 65536  # MDHP_NOALLOC_MAX_WINDOWS in include/mdhp.h

OK, E_ARG, E_UNSORTED, E_ID_RANGE, E_TIME_RANGE, E_NONFINITE, E_MAXITER, E_TIMEOUT, E_CUDA, \
    E_NOMEM, E_UNSUPPORTED, E_SIM_STALLED = range(12)
STATUS_NAMES = ["OK", "E_ARG", "E_UNSORTED", "E_ID_RANGE", "E_TIME_RANGE", "E_NONFINITE",
                "E_MAXITER", "E_TIMEOUT", "E_CUDA", "E_NOMEM", "E_UNSUPPORTED",
                "E_SIM_STALLED"]

P = ctypes.c_void_p


class MdhpBatch(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("M", ctypes.c_int32), ("n_events", ctypes.c_int64),
                ("offsets", P), ("t", P), ("id", P), ("T_span", P), ("weights", P),
                ("beta_mode", ctypes.c_int32), ("max_events", ctypes.c_int32)]


class MdhpLstmDims(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("L", ctypes.c_int32), ("D", ctypes.c_int32),
                ("H", ctypes.c_int32), ("M", ctypes.c_int32), ("nb", ctypes.c_int32),
                ("O", ctypes.c_int32)]


class MdhpFitOpts(ctypes.Structure):
    _fields_ = [("optimizer", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("fit_beta", ctypes.c_int32), ("patience", ctypes.c_int32),
                ("lr", ctypes.c_float), ("mu_floor", ctypes.c_float),
                ("alpha_floor", ctypes.c_float), ("beta_floor", ctypes.c_float),
                ("adam_b1", ctypes.c_float), ("adam_b2", ctypes.c_float),
                ("adam_eps", ctypes.c_float), ("init", ctypes.c_int32), ("tol", ctypes.c_double)]


# (name, restype, argtypes) for every symbol include/mdhp.h declares
SIGNATURES = [
    ("mdhp_loglik_grad", ctypes.c_int, [ctypes.POINTER(MdhpBatch), P, P, P, P, P, P, P, P, P, P, P]),
    ("mdhp_fit_opts_default", None, [ctypes.POINTER(MdhpFitOpts)]),
    ("mdhp_plan_create", ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int64, ctypes.c_char_p]),
    ("mdhp_plan_destroy", None, [P]),
    ("mdhp_fit_batch", ctypes.c_int, [P, ctypes.POINTER(MdhpBatch), ctypes.POINTER(MdhpFitOpts),
                                      P, P, P, P, P, P, P]),
    ("mdhp_plan_set_timing", ctypes.c_int, [P, ctypes.c_int32]),
    ("mdhp_plan_last_fit_ms", ctypes.c_float, [P]),
    ("mdhp_plan_get_shape", ctypes.c_int, [P, P, P, P]),
    ("mdhp_plan_set_shape", ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    ("mdhp_plan_set_path", ctypes.c_int, [P, ctypes.c_int32]),
    ("mdhp_fit_batch_noalloc", ctypes.c_int, [ctypes.POINTER(MdhpBatch), ctypes.POINTER(MdhpFitOpts),
                                              P, P, P, P, P, P, P]),
    ("mdhp_plan_autotune", ctypes.c_int, [P, ctypes.POINTER(MdhpBatch), ctypes.POINTER(MdhpFitOpts),
                                          P, P, P, P, P, P, ctypes.c_int32, P, P, P]),
    ("mdhp_plan_set_pipeline", ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32]),
    ("mdhp_plan_set_feature_store", ctypes.c_int, [P, ctypes.c_int32]),
    ("mdhp_plan_get_feature_store", ctypes.c_int32, [P]),
    ("mdhp_plan_get_pipeline", ctypes.c_int, [P, P, P]),
    ("mdhp_plan_set_split", ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    ("mdhp_plan_get_split", ctypes.c_int, [P, P, P, P]),
    ("mdhp_plan_last_launches", ctypes.c_int32, [P]),
    ("mdhp_simulate", ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P, P, P,
                                     ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, P, P, P, P, P]),
    ("mdhp_init_model_create", ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_uint64]),
    ("mdhp_init_model_destroy", None, [P]),
    ("mdhp_init_model_info", ctypes.c_int, [P, P, P, P]),
    ("mdhp_init_model_get", ctypes.c_int, [P, ctypes.c_int32, P, P]),
    ("mdhp_init_model_set_params", ctypes.c_int, [P, P, P]),
    ("mdhp_init_features", ctypes.c_int, [ctypes.POINTER(MdhpBatch), P, P, P, P]),
    ("mdhp_init_forward", ctypes.c_int, [P, P, ctypes.c_int32, P, P]),
    ("mdhp_init_predict", ctypes.c_int, [P, ctypes.POINTER(MdhpBatch), P, P, P, P]),
    ("mdhp_init_train_step", ctypes.c_int, [P, P, P, P, ctypes.c_int32, P, P, ctypes.c_int32,
                                            ctypes.c_float, ctypes.c_float, P, P]),
    ("mdhp_init_backward", ctypes.c_int, [P, P, P, P, ctypes.c_int32, P, P, ctypes.c_int32, P, P]),
    ("mdhp_init_set_grads", ctypes.c_int, [P, P, P]),
    ("mdhp_init_apply", ctypes.c_int, [P, ctypes.c_float, ctypes.c_float, P]),
    ("mdhp_plan_set_init_model", ctypes.c_int, [P, P]),
    ("mdhp_lstm_forward", ctypes.c_int, [ctypes.POINTER(MdhpLstmDims)] + [P] * 18),
    ("mdhp_lstm_backward", ctypes.c_int, [ctypes.POINTER(MdhpLstmDims)] + [P] * 30),
    ("mdhp_probe_peak", ctypes.c_int, [ctypes.c_int32, P, P, P]),
    ("mdhp_plan_set_event_ring", ctypes.c_int, [P, ctypes.c_int32]),
    ("mdhp_plan_set_wait_limit", ctypes.c_int, [P, ctypes.c_int32]),
    ("mdhp_init_model_set_gemm", ctypes.c_int, [P, ctypes.c_int32]),
    ("mdhp_gemm_bf16", ctypes.c_int, [P, ctypes.c_int64, ctypes.c_int32, P, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, ctypes.c_int32,
                                      P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, P]),
    ("mdhp_gemm_check", ctypes.c_int, [P]),
    ("mdhp_last_error", ctypes.c_char_p, []),
    ("mdhp_version", ctypes.c_int32, []),
]

_lib = None


def load(path: str | None = None):
    """Load libmdhp.so (built by ``build.py``); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIBPATH
    if not os.path.exists(p):
        raise RuntimeError(f"MDHP CUDA library not built: {p} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class MdhpError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.mdhp_last_error().decode(errors="replace")
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")
        self.status = status


def check(status: int, where: str):
    if status != OK:
        raise MdhpError(status, where)
