"""ctypes wrapper of the FP64 C oracle (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this module.  The product path never does: it has no CPU
fallback.  See ``mdhp_oracle.c`` for the definitions and their sources in
arXiv 2411.10258 (MDHP intensity, closed-form lnL and App. B).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdhp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBPATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

OK, E_ARG, E_UNSORTED, E_ID_RANGE, E_TIME_RANGE, E_NONFINITE, E_MAXITER = 0, 1, 2, 3, 4, 5, 6


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, no fast-math, OpenMP over windows)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        tmp = _LIBPATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


class FitOpts(ctypes.Structure):
    _fields_ = [("optimizer", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("fit_beta", ctypes.c_int32), ("patience", ctypes.c_int32),
                ("lr", ctypes.c_double), ("tol", ctypes.c_double),
                ("mu_floor", ctypes.c_double), ("alpha_floor", ctypes.c_double),
                ("beta_floor", ctypes.c_double), ("adam_b1", ctypes.c_double),
                ("adam_b2", ctypes.c_double), ("adam_eps", ctypes.c_double)]


def fit_opts(optimizer=0, max_iters=200, fit_beta=0, lr=1e-2, tol=0.0, patience=3,
             mu_floor=1e-10, alpha_floor=0.0, beta_floor=1e-6, adam_b1=0.9, adam_b2=0.999,
             adam_eps=1e-8) -> FitOpts:
    return FitOpts(optimizer, max_iters, fit_beta, patience, lr, tol, mu_floor, alpha_floor,
                   beta_floor, adam_b1, adam_b2, adam_eps)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.oracle_validate.restype = I
        lib.oracle_validate.argtypes = [I, I64, P, P, P, D]
        lib.oracle_loglik_grad.restype = I
        lib.oracle_loglik_grad.argtypes = [I, I, I64, P, P, P, D, P, P, P, P, P, P, P, P, P]
        lib.oracle_cold_init.restype = None
        lib.oracle_cold_init.argtypes = [I, I, I64, P, D, P, P, P]
        lib.oracle_fit.restype = I
        lib.oracle_fit.argtypes = [I, I, I64, P, P, P, D, ctypes.POINTER(FitOpts), P, P, P, P, P]
        lib.oracle_fit_batch.restype = I
        lib.oracle_fit_batch.argtypes = [I, I, I, P, P, P, P, P, ctypes.POINTER(FitOpts),
                                         P, P, P, P, P, P, I]
        lib.oracle_num_threads.restype = I
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def beta_mode_of(beta, M: int, mode: int | None) -> int:
    if mode is not None:
        return mode
    n = np.asarray(beta).size
    return 0 if n == 1 else (1 if n == M else 2)


def validate(t, ids, T, M, w=None) -> int:
    t = _f64(t); ids = np.ascontiguousarray(ids, dtype=np.int32); w = _f64(w)
    return _load().oracle_validate(M, len(t), _p(t), _p(ids), _p(w), float(T))


def loglik_grad(t, ids, T, mu, alpha, beta, w=None, mode=None):
    """lnL and its gradient for one window, in FP64.

    Returns dict(status, lnL, g_mu [M], g_alpha [M, M], g_beta (shape of beta),
    g_w [N] (only if w is given), r [N] = 1/lambda at each event)."""
    mu = _f64(mu).reshape(-1)
    M = mu.shape[0]
    alpha = _f64(alpha).reshape(M * M)
    beta = _f64(beta).reshape(-1)
    mode = beta_mode_of(beta, M, mode)
    t = _f64(t).reshape(-1)
    ids = np.ascontiguousarray(ids, dtype=np.int32).reshape(-1)
    w = _f64(w)
    N = t.shape[0]
    lnl = np.zeros(1)
    gm, ga, gb = np.zeros(M), np.zeros(M * M), np.zeros(beta.shape[0])
    gw = np.zeros(N) if w is not None else None
    r = np.zeros(max(N, 1))
    st = _load().oracle_loglik_grad(M, mode, N, _p(t), _p(ids), _p(w), float(T), _p(mu),
                                    _p(alpha), _p(beta), _p(lnl), _p(gm), _p(ga), _p(gb),
                                    _p(gw), _p(r))
    return dict(status=st, lnL=float(lnl[0]), g_mu=gm, g_alpha=ga.reshape(M, M), g_beta=gb,
                g_w=gw, r=r[:N])


def cold_init(ids, T, M, beta, mode=None):
    beta = _f64(beta).reshape(-1)
    mode = beta_mode_of(beta, M, mode)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    mu, alpha = np.zeros(M), np.zeros(M * M)
    _load().oracle_cold_init(M, mode, len(ids), _p(ids), float(T), _p(beta), _p(mu), _p(alpha))
    return mu, alpha.reshape(M, M)


def fit(t, ids, T, mu, alpha, beta, opts: FitOpts, w=None, mode=None):
    """Projected ascent for one window; returns dict(status, lnL, iters, mu, alpha, beta)."""
    mu = _f64(mu).reshape(-1).copy()
    M = mu.shape[0]
    alpha = _f64(alpha).reshape(M * M).copy()
    beta = _f64(beta).reshape(-1).copy()
    mode = beta_mode_of(beta, M, mode)
    t = _f64(t).reshape(-1)
    ids = np.ascontiguousarray(ids, dtype=np.int32).reshape(-1)
    w = _f64(w)
    lnl = np.zeros(1)
    it = np.zeros(1, dtype=np.int32)
    st = _load().oracle_fit(M, mode, len(t), _p(t), _p(ids), _p(w), float(T), ctypes.byref(opts),
                            _p(mu), _p(alpha), _p(beta), _p(lnl), _p(it))
    return dict(status=st, lnL=float(lnl[0]), iters=int(it[0]), mu=mu, alpha=alpha.reshape(M, M),
                beta=beta)


def fit_batch(offsets, t32, id16, T32, M, mode, mu, alpha, beta, opts: FitOpts, w32=None,
              nthreads: int = 0):
    """Batched fit over CSR windows (FP32/int16 inputs widened to FP64 inside).
    mu [B, M], alpha [B, M, M], beta [B, nb] are copied; returns dict of arrays."""
    B = len(T32)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    t32 = np.ascontiguousarray(t32, dtype=np.float32)
    id16 = np.ascontiguousarray(id16, dtype=np.int16)
    T32 = np.ascontiguousarray(T32, dtype=np.float32)
    w32 = None if w32 is None else np.ascontiguousarray(w32, dtype=np.float32)
    mu = _f64(mu).reshape(B, M).copy()
    alpha = _f64(alpha).reshape(B, M, M).copy()
    beta = _f64(beta).reshape(B, -1).copy()
    lnl = np.zeros(B)
    it = np.zeros(B, dtype=np.int32)
    st = np.zeros(B, dtype=np.int32)
    _load().oracle_fit_batch(B, M, mode, _p(offsets), _p(t32), _p(id16), _p(w32), _p(T32),
                             ctypes.byref(opts), _p(mu), _p(alpha), _p(beta), _p(lnl), _p(it),
                             _p(st), nthreads)
    return dict(status=st, lnL=lnl, iters=it, mu=mu, alpha=alpha, beta=beta)


def num_threads() -> int:
    return _load().oracle_num_threads()
