"""GB300 (sm_103a) MDHP-GDS: batched gradient-descent fitting of exponential
multi-dimensional Hawkes processes (arXiv 2411.10258, Sec. IV-B) behind a C ABI
(include/mdhp.h).  Python is marshalling only; the computation is in
``_build/libmdhp.so``.
"""
from .api import (DeviceBatch, FitOptions, InitModel, LoglikGrad, MdhpLSTM, MdhpLSTMFunction,  # noqa: F401
                  Plan, loglik_grad, simulate)
from ._lib import MdhpError  # noqa: F401

__all__ = ["DeviceBatch", "FitOptions", "InitModel", "LoglikGrad", "Plan", "loglik_grad", "simulate", "MdhpError",
           "MdhpLSTM", "MdhpLSTMFunction"]
