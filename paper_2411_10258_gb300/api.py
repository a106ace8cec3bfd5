"""Python surface of the MDHP-GDS library: torch tensors in, C ABI calls out.

Every computation runs in the CUDA library (``libmdhp.so``); this module only
moves pointers, shapes and the current CUDA stream across the boundary.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib


def _ptr(x):
    return None if x is None else ctypes.c_void_p(x.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def nbeta(beta_mode: int, M: int) -> int:
    return 1 if beta_mode == 0 else (M if beta_mode == 1 else M * M)


@dataclass
class DeviceBatch:
    """CSR windows resident on the GPU (see include/mdhp.h, mdhp_batch)."""

    M: int
    beta_mode: int
    offsets: torch.Tensor  # int64 [B+1]
    t: torch.Tensor  # float32 [n]
    id: torch.Tensor  # int16 [n]
    T: torch.Tensor  # float32 [B]
    weights: torch.Tensor | None = None  # float32 [n]
    max_events: int = 0

    @property
    def B(self) -> int:
        return int(self.T.shape[0])

    @property
    def n_events(self) -> int:
        return int(self.t.shape[0])

    def c_struct(self, weights: torch.Tensor | None = None) -> _lib.MdhpBatch:
        w = self.weights if weights is None else weights
        return _lib.MdhpBatch(self.B, self.M, self.n_events, _ptr(self.offsets), _ptr(self.t),
                              _ptr(self.id), _ptr(self.T), _ptr(w), self.beta_mode,
                              int(self.max_events))

    @staticmethod
    def from_host(batch, device="cuda", max_events: int | None = None, non_blocking=False):
        """Copy a host batch (workload.Batch or anything with the same fields)."""
        dev = torch.device(device)

        def up(a):
            return torch.from_numpy(np.ascontiguousarray(a)).to(dev, non_blocking=non_blocking)

        cnt = np.diff(batch.offsets)
        me = int(cnt.max()) if (max_events is None and len(cnt)) else int(max_events or 0)
        return DeviceBatch(batch.M, batch.beta_mode, up(batch.offsets), up(batch.t), up(batch.id),
                           up(batch.T), None if batch.weights is None else up(batch.weights), me)


def loglik_grad(db: DeviceBatch, mu: torch.Tensor, alpha: torch.Tensor, beta: torch.Tensor,
                beta_grad: bool = False, weight_grad: bool = False,
                weights: torch.Tensor | None = None, stream=None) -> dict:
    """lnL and its gradient per window (mdhp_loglik_grad).  Returns tensors
    loglik [B] f64, g_mu [B,M], g_alpha [B,M,M], g_beta or None, g_w or None,
    status [B] int32."""
    lib = _lib.load()
    B, M = db.B, db.M
    dev = db.t.device
    f32 = dict(dtype=torch.float32, device=dev)
    mu = mu.contiguous().float(); alpha = alpha.contiguous().float(); beta = beta.contiguous().float()
    out = dict(loglik=torch.empty(B, dtype=torch.float64, device=dev),
               g_mu=torch.empty(B, M, **f32), g_alpha=torch.empty(B, M, M, **f32),
               g_beta=torch.empty(B, nbeta(db.beta_mode, M), **f32) if beta_grad else None,
               g_w=torch.empty(db.n_events, **f32) if weight_grad else None,
               status=torch.empty(B, dtype=torch.int32, device=dev))
    r_work = torch.empty(db.n_events, **f32) if weight_grad else None
    st = db.c_struct(weights)
    rc = lib.mdhp_loglik_grad(ctypes.byref(st), _ptr(mu), _ptr(alpha), _ptr(beta),
                              _ptr(out["loglik"]), _ptr(out["g_mu"]), _ptr(out["g_alpha"]),
                              _ptr(out["g_beta"]), _ptr(out["g_w"]), _ptr(r_work),
                              _ptr(out["status"]), _stream(stream))
    _lib.check(rc, "mdhp_loglik_grad")
    out["_keep"] = (r_work, mu, alpha, beta)
    return out


def simulate(M: int, beta_mode: int, mu, alpha, beta, counts, seed: int, stream_id: int,
             first_window: int = 0, device="cuda", stream=None):
    """Simulate windows with exactly counts[b] events each on the GPU
    (mdhp_simulate, Ogata thinning in FP64).  mu [B,M], alpha [B,M,M] and beta
    [B,nb] are float64 (host arrays or device tensors); counts is a host int
    array.  Windows run longest first.  Returns (DeviceBatch, status int32[B])."""
    lib = _lib.load()
    dev = torch.device(device)
    counts = np.asarray(counts, dtype=np.int64)
    B = len(counts)
    offsets = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    order = np.argsort(-counts, kind="stable").astype(np.int32)

    def dev64(x, shape):
        x = torch.as_tensor(x, dtype=torch.float64, device=dev)
        return x.reshape(shape).contiguous()

    mu = dev64(mu, (B, M))
    alpha = dev64(alpha, (B, M, M))
    beta = dev64(beta, (B, nbeta(beta_mode, M)))
    n = int(offsets[-1])
    off_d = torch.from_numpy(offsets).to(dev)
    order_d = torch.from_numpy(order).to(dev)
    t = torch.empty(max(n, 1), dtype=torch.float32, device=dev)
    ids = torch.empty(max(n, 1), dtype=torch.int16, device=dev)
    T = torch.empty(B, dtype=torch.float32, device=dev)
    status = torch.empty(B, dtype=torch.int32, device=dev)
    _lib.check(lib.mdhp_simulate(M, beta_mode, B, _ptr(mu), _ptr(alpha), _ptr(beta), _ptr(off_d),
                                 _ptr(order_d), int(seed), int(stream_id), int(first_window),
                                 _ptr(t), _ptr(ids), _ptr(T), _ptr(status), _stream(stream)),
               "mdhp_simulate")
    me = int(counts.max()) if B else 0
    return DeviceBatch(M, beta_mode, off_d, t[:n], ids[:n], T, None, me), status


PEAK_KINDS = ("fp32_fma", "mufu_ex2", "mufu_lg2", "mufu_rcp")


def probe_peak(kind: str, stream=None) -> tuple[float, float]:
    """Measured throughput of one arithmetic pipe of the current GPU
    (mdhp_probe_peak): (operations per second, best time in ms).  fp32_fma
    counts an FMA as two floating-point operations."""
    lib = _lib.load()
    rate, ms = ctypes.c_double(0.0), ctypes.c_float(0.0)
    _lib.check(lib.mdhp_probe_peak(PEAK_KINDS.index(kind), ctypes.byref(rate), ctypes.byref(ms),
                                   _stream(stream)), "mdhp_probe_peak")
    return rate.value, ms.value


def gemm_bf16(A: torch.Tensor, B: torch.Tensor, M: int, N: int, K: int, a_mn: bool = False,
              b_mn: bool = False, bias: torch.Tensor | None = None, relu: bool = False,
              C: torch.Tensor | None = None, C_bf16: torch.Tensor | None = None, accumulate: bool = False,
              engine: int = 0, stream=None):
    """C (+)= A B (mdhp_gemm_bf16).  A: bfloat16 [M, K] (a_mn False) or [K, M];
    B: bfloat16 [N, K] (b_mn False) or [K, N]; C float32 [M, N] and/or C_bf16
    bfloat16 [M, N] (row pitch N).  engine 0: tcgen05 tensor cores, 1: mma.sync."""
    lib = _lib.load()
    lda = A.shape[1]
    ldb = B.shape[1]
    _lib.check(lib.mdhp_gemm_bf16(_ptr(A), lda, int(a_mn), _ptr(B), ldb, int(b_mn), M, N, K,
                                  _ptr(bias) if bias is not None else None, int(relu),
                                  _ptr(C) if C is not None else None,
                                  _ptr(C_bf16) if C_bf16 is not None else None, N, int(accumulate),
                                  engine, _stream(stream)), "mdhp_gemm_bf16")


def gemm_check() -> int:
    """Synchronise; tensor-core GEMM CTAs whose bounded waits gave up since the last call."""
    lib = _lib.load()
    n = ctypes.c_int32(0)
    _lib.check(lib.mdhp_gemm_check(ctypes.byref(n)), "mdhp_gemm_check")
    return n.value


@dataclass
class FitOptions:
    """Mirror of mdhp_fit_opts (defaults as mdhp_fit_opts_default)."""

    optimizer: int = 0
    max_iters: int = 200
    fit_beta: int = 0
    patience: int = 3
    lr: float = 1e-2
    mu_floor: float = 1e-10
    alpha_floor: float = 0.0
    beta_floor: float = 1e-6
    adam_b1: float = 0.9
    adam_b2: float = 0.999
    adam_eps: float = 1e-8
    init: int = 1
    tol: float = 0.0

    def c_struct(self) -> _lib.MdhpFitOpts:
        return _lib.MdhpFitOpts(self.optimizer, self.max_iters, self.fit_beta, self.patience,
                                self.lr, self.mu_floor, self.alpha_floor, self.beta_floor,
                                self.adam_b1, self.adam_b2, self.adam_eps, self.init, self.tol)


class Plan:
    """Owns the device scratch of batched fitting (mdhp_plan)."""

    def __init__(self, M: int, beta_mode: int, max_windows: int, max_events: int = 0,
                 autotune_cache: str | None = None):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        rc = self.lib.mdhp_plan_create(ctypes.byref(h), M, beta_mode, max_windows, max_events,
                                       None if autotune_cache is None else autotune_cache.encode())
        _lib.check(rc, "mdhp_plan_create")
        self.h = h
        self.M, self.beta_mode, self.max_windows = M, beta_mode, max_windows

    def close(self):
        if getattr(self, "h", None):
            self.lib.mdhp_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_timing(self, on: bool):
        _lib.check(self.lib.mdhp_plan_set_timing(self.h, 1 if on else 0), "mdhp_plan_set_timing")

    def last_fit_ms(self) -> float:
        return float(self.lib.mdhp_plan_last_fit_ms(self.h))

    def last_launches(self) -> int:
        """Kernels launched by the last fit (mdhp_plan_last_launches)."""
        return int(self.lib.mdhp_plan_last_launches(self.h))

    def shape(self):
        v = [ctypes.c_int32() for _ in range(3)]
        _lib.check(self.lib.mdhp_plan_get_shape(self.h, *[ctypes.byref(x) for x in v]), "get_shape")
        return tuple(x.value for x in v)

    def set_path(self, path: str):
        """'auto' (decoupled features for fixed beta when possible) or 'recursion'."""
        code = {"auto": 0, "recursion": 1}[path]
        _lib.check(self.lib.mdhp_plan_set_path(self.h, code), "mdhp_plan_set_path")

    def set_shape(self, threads_per_window: int, threads_per_chunk: int, cutoff: int):
        _lib.check(self.lib.mdhp_plan_set_shape(self.h, threads_per_window, threads_per_chunk, cutoff),
                   "mdhp_plan_set_shape")

    def autotune(self, db: DeviceBatch, opts: FitOptions, mu: torch.Tensor, alpha: torch.Tensor,
                 beta: torch.Tensor, tune_iters: int = 20, stream=None) -> dict:
        """mdhp_plan_autotune: time the candidate launch shapes on this batch and
        keep the fastest (written to the plan's cache file, if any).  mu/alpha/beta
        are restored on return.  Returns the choice and its device time."""
        B = db.B
        dev = db.t.device
        for x in (mu, alpha, beta):
            assert x.is_contiguous() and x.dtype == torch.float32 and x.device == dev
        scratch = dict(loglik=torch.empty(B, dtype=torch.float64, device=dev),
                       iters=torch.empty(B, dtype=torch.int32, device=dev),
                       status=torch.empty(B, dtype=torch.int32, device=dev))
        chosen = (ctypes.c_int32 * 9)()
        best = ctypes.c_float(-1.0)
        st = db.c_struct()
        o = opts.c_struct()
        rc = self.lib.mdhp_plan_autotune(self.h, ctypes.byref(st), ctypes.byref(o), _ptr(mu),
                                         _ptr(alpha), _ptr(beta), _ptr(scratch["loglik"]),
                                         _ptr(scratch["iters"]), _ptr(scratch["status"]),
                                         int(tune_iters), chosen, ctypes.byref(best), _stream(stream))
        _lib.check(rc, "mdhp_plan_autotune")
        return dict(path=("decoupled", "recursion")[chosen[0]], threads_per_window=chosen[1],
                    threads_per_chunk=chosen[2], cutoff=chosen[3], pipe_steps=chosen[4],
                    pipe_stages=chosen[5], split=bool(chosen[6]), split_threads=chosen[7],
                    split_ctas=chosen[8], feature_store=self.get_feature_store(), ms=best.value)

    def set_event_ring(self, enable: bool):
        """Streamed events through the bulk-copy ring (mdhp_plan_set_event_ring)."""
        _lib.check(self.lib.mdhp_plan_set_event_ring(self.h, 1 if enable else 0),
                   "mdhp_plan_set_event_ring")

    def set_wait_limit(self, polls: int):
        """Bound of the bulk-copy rings' consumer waits (mdhp_plan_set_wait_limit); 0 = default."""
        _lib.check(self.lib.mdhp_plan_set_wait_limit(self.h, polls), "mdhp_plan_set_wait_limit")

    def set_feature_store(self, store: int):
        """Where the decoupled kernels keep each thread's first feature steps
        (mdhp_plan_set_feature_store): 0 the scratch only, 1 tensor memory,
        2 tensor memory and then shared memory, 3 as 2 with 384 threads."""
        _lib.check(self.lib.mdhp_plan_set_feature_store(self.h, int(store)),
                   "mdhp_plan_set_feature_store")

    def get_feature_store(self) -> int:
        return int(self.lib.mdhp_plan_get_feature_store(self.h))

    def set_pipeline(self, steps_per_stage: int, stages: int):
        """Feature ring of the decoupled kernels (mdhp_plan_set_pipeline); stages=0: none."""
        _lib.check(self.lib.mdhp_plan_set_pipeline(self.h, steps_per_stage, stages),
                   "mdhp_plan_set_pipeline")

    def set_split(self, enable: bool, long_threads: int = 256, long_ctas_per_sm: int = 1):
        """Two launches over one queue (mdhp_plan_set_split)."""
        _lib.check(self.lib.mdhp_plan_set_split(self.h, 1 if enable else 0, long_threads,
                                                long_ctas_per_sm), "mdhp_plan_set_split")

    def split(self):
        v = [ctypes.c_int32() for _ in range(3)]
        _lib.check(self.lib.mdhp_plan_get_split(self.h, *[ctypes.byref(x) for x in v]),
                   "mdhp_plan_get_split")
        return (bool(v[0].value), v[1].value, v[2].value)

    def pipeline(self):
        v = [ctypes.c_int32() for _ in range(2)]
        _lib.check(self.lib.mdhp_plan_get_pipeline(self.h, *[ctypes.byref(x) for x in v]),
                   "mdhp_plan_get_pipeline")
        return tuple(x.value for x in v)

    def fit(self, db: DeviceBatch, opts: FitOptions, mu: torch.Tensor, alpha: torch.Tensor,
            beta: torch.Tensor, out: dict | None = None, stream=None) -> dict:
        """mdhp_fit_batch; mu/alpha/beta are updated in place (float32, contiguous)."""
        B = db.B
        dev = db.t.device
        if out is None:
            out = dict(loglik=torch.empty(B, dtype=torch.float64, device=dev),
                       iters=torch.empty(B, dtype=torch.int32, device=dev),
                       status=torch.empty(B, dtype=torch.int32, device=dev))
        for x in (mu, alpha, beta):
            assert x.is_contiguous() and x.dtype == torch.float32 and x.device == dev
        st = db.c_struct()
        o = opts.c_struct()
        rc = self.lib.mdhp_fit_batch(self.h, ctypes.byref(st), ctypes.byref(o), _ptr(mu),
                                     _ptr(alpha), _ptr(beta), _ptr(out["loglik"]),
                                     _ptr(out["iters"]), _ptr(out["status"]), _stream(stream))
        _lib.check(rc, "mdhp_fit_batch")
        out.update(mu=mu, alpha=alpha, beta=beta)
        return out


class LoglikGrad(torch.autograd.Function):
    """lnL per window as a differentiable function of (mu, alpha, beta, weights).

    forward returns lnL [B] (float64); the gradients are computed by the
    library in the same call (one recursion pass, plus the reverse-time pass
    for event weights), and backward scales them by grad_output per window.
    As a loss use -LoglikGrad.apply(...).sum()."""

    @staticmethod
    def forward(ctx, db: DeviceBatch, mu, alpha, beta, weights=None):
        need_b = ctx.needs_input_grad[3]
        need_w = weights is not None and ctx.needs_input_grad[4]
        out = loglik_grad(db, mu.detach(), alpha.detach(), beta.detach(), beta_grad=need_b,
                          weight_grad=need_w, weights=None if weights is None else weights.detach())
        bad = out["status"] != 0
        ctx.save_for_backward(out["g_mu"], out["g_alpha"],
                              out["g_beta"] if need_b else torch.empty(0, device=mu.device),
                              out["g_w"] if need_w else torch.empty(0, device=mu.device),
                              db.offsets)
        ctx.need_b, ctx.need_w = need_b, need_w
        ctx.beta_shape = beta.shape
        ll = out["loglik"]
        ctx.mark_non_differentiable(bad)
        return ll, bad

    @staticmethod
    def backward(ctx, g_ll, _g_bad):
        g_mu, g_alpha, g_beta, g_w, offsets = ctx.saved_tensors
        go = g_ll.to(torch.float32)
        d_mu = g_mu * go[:, None]
        d_alpha = g_alpha * go[:, None, None]
        d_beta = (g_beta * go[:, None]).reshape(ctx.beta_shape) if ctx.need_b else None
        d_w = None
        if ctx.need_w:
            counts = offsets[1:] - offsets[:-1]
            d_w = g_w * torch.repeat_interleave(go, counts)
        return None, d_mu, d_alpha, d_beta, d_w


class InitModel:
    """Learned warm start (mdhp_init_model): features -> 4-layer BF16 MLP -> (mu, alpha).

    Training runs on the GPU through mdhp_init_train_step; this class only
    allocates the torch buffers the C ABI writes into."""

    def __init__(self, M: int, hidden: int = 256, max_batch: int = 256, seed: int = 1024):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(self.lib.mdhp_init_model_create(ctypes.byref(h), M, hidden, max_batch, seed),
                   "mdhp_init_model_create")
        self.h = h
        self.M, self.hidden, self.max_batch = M, hidden, max_batch
        fd, od, npar = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _lib.check(self.lib.mdhp_init_model_info(self.h, ctypes.byref(fd), ctypes.byref(od),
                                                 ctypes.byref(npar)), "mdhp_init_model_info")
        self.feature_dim, self.out_dim, self.num_params = fd.value, od.value, npar.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.mdhp_init_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self, what: str = "params", stream=None) -> torch.Tensor:
        out = torch.empty(self.num_params, dtype=torch.float32, device="cuda")
        _lib.check(self.lib.mdhp_init_model_get(self.h, 0 if what == "params" else 1, _ptr(out),
                                                _stream(stream)), "mdhp_init_model_get")
        return out

    def set_params(self, params: torch.Tensor, stream=None):
        params = params.contiguous().float().cuda()
        assert params.numel() == self.num_params
        _lib.check(self.lib.mdhp_init_model_set_params(self.h, _ptr(params), _stream(stream)),
                   "mdhp_init_model_set_params")

    def features(self, db: DeviceBatch, beta: torch.Tensor, stream=None):
        """(features bfloat16 [B, feature_dim], mu_cold float32 [B, M])."""
        feat = torch.empty(db.B, self.feature_dim, dtype=torch.bfloat16, device=db.t.device)
        mu_cold = torch.empty(db.B, db.M, dtype=torch.float32, device=db.t.device)
        st = db.c_struct()
        beta = beta.contiguous().float()
        _lib.check(self.lib.mdhp_init_features(ctypes.byref(st), _ptr(beta), _ptr(feat),
                                               _ptr(mu_cold), _stream(stream)), "mdhp_init_features")
        return feat, mu_cold

    def forward(self, feat: torch.Tensor, stream=None) -> torch.Tensor:
        out = torch.empty(feat.shape[0], self.out_dim, dtype=torch.float32, device=feat.device)
        _lib.check(self.lib.mdhp_init_forward(self.h, _ptr(feat.contiguous()), feat.shape[0],
                                              _ptr(out), _stream(stream)), "mdhp_init_forward")
        return out

    def predict(self, db: DeviceBatch, beta: torch.Tensor, stream=None):
        mu = torch.empty(db.B, db.M, dtype=torch.float32, device=db.t.device)
        alpha = torch.empty(db.B, db.M, db.M, dtype=torch.float32, device=db.t.device)
        st = db.c_struct()
        _lib.check(self.lib.mdhp_init_predict(self.h, ctypes.byref(st), _ptr(beta.contiguous().float()),
                                              _ptr(mu), _ptr(alpha), _stream(stream)),
                   "mdhp_init_predict")
        return mu, alpha

    def train_step(self, feat, mu_cold, beta, mu_target, alpha_target, lr=3e-4, weight_decay=5e-5,
                   loss_out: torch.Tensor | None = None, stream=None):
        B = feat.shape[0]
        beta = beta.contiguous().float()
        bstride = 1 if beta.numel() == B else self.M
        if loss_out is None:
            loss_out = torch.empty(1, dtype=torch.float32, device=feat.device)
        _lib.check(self.lib.mdhp_init_train_step(
            self.h, _ptr(feat.contiguous()), _ptr(mu_cold.contiguous()), _ptr(beta), bstride,
            _ptr(mu_target.contiguous().float()), _ptr(alpha_target.contiguous().float()), B,
            float(lr), float(weight_decay), _ptr(loss_out), _stream(stream)), "mdhp_init_train_step")
        return loss_out

    def backward(self, feat, mu_cold, beta, mu_target, alpha_target, loss_out=None, stream=None):
        """Loss and gradient of this process's windows (mdhp_init_backward); no update."""
        B = feat.shape[0]
        beta = beta.contiguous().float()
        bstride = 1 if beta.numel() == B else self.M
        if loss_out is None:
            loss_out = torch.empty(1, dtype=torch.float32, device=feat.device)
        _lib.check(self.lib.mdhp_init_backward(
            self.h, _ptr(feat.contiguous()), _ptr(mu_cold.contiguous()), _ptr(beta), bstride,
            _ptr(mu_target.contiguous().float()), _ptr(alpha_target.contiguous().float()), B,
            _ptr(loss_out), _stream(stream)), "mdhp_init_backward")
        return loss_out

    def set_grads(self, grads: torch.Tensor, stream=None):
        _lib.check(self.lib.mdhp_init_set_grads(self.h, _ptr(grads.contiguous().float()), _stream(stream)),
                   "mdhp_init_set_grads")

    def apply(self, lr=3e-4, weight_decay=5e-5, stream=None):
        """AdamW step with the current gradient buffer (mdhp_init_apply)."""
        _lib.check(self.lib.mdhp_init_apply(self.h, float(lr), float(weight_decay), _stream(stream)),
                   "mdhp_init_apply")

    def train_step_dp(self, feat, mu_cold, beta, mu_target, alpha_target, lr=3e-4, weight_decay=5e-5):
        """Data-parallel step: local gradient, mean over the ranks of the default
        process group, then AdamW on every rank (identical parameters after it)."""
        from . import shard

        loss = self.backward(feat, mu_cold, beta, mu_target, alpha_target)
        g = self.get("grads")
        shard.allreduce_mean_(g)
        self.set_grads(g)
        self.apply(lr, weight_decay)
        return loss

    def set_gemm(self, engine: int):
        """0: tensor-core (tcgen05) products where they apply; 1: mma.sync for all."""
        _lib.check(self.lib.mdhp_init_model_set_gemm(self.h, engine), "mdhp_init_model_set_gemm")

    def attach(self, plan: "Plan"):
        """Use this model for FitOptions(init=2) fits of `plan`."""
        _lib.check(self.lib.mdhp_plan_set_init_model(plan.h, self.h), "mdhp_plan_set_init_model")


class MdhpLSTMFunction(torch.autograd.Function):
    """The MDHP-LSTM cell over whole sequences (mdhp_lstm_forward /
    mdhp_lstm_backward): inputs x [B, L, D], the windows' fitted MDHP
    parameters mu [B, M], alpha [B, M, M], beta [B, nb] and T_span [B], and
    the weights W [4H, D], U [4H, H], b [4H], A [H, M*M], Bm [H, nb],
    C [H, M], Wy [O, H]; returns y [B, L, O].  Gradients flow to x, the
    weights and (mu, alpha, beta); T_span gets none."""

    @staticmethod
    def forward(ctx, x, mu, alpha, beta, T, W, U, b, A, Bm, C, Wy):
        lib = _lib.load()
        c32 = lambda t: t.detach().contiguous().float()
        x, mu, alpha, beta, T, W, U, b, A, Bm, C, Wy = map(c32, (x, mu, alpha, beta, T, W, U, b, A, Bm, C, Wy))
        Bn, L, D = x.shape
        H, M, O = U.shape[1], mu.shape[1], Wy.shape[0]
        beta = beta.reshape(Bn, -1)
        dims = _lib.MdhpLstmDims(Bn, L, D, H, M, beta.shape[1], O)
        f32 = dict(dtype=torch.float32, device=x.device)
        y = torch.empty(Bn, L, O, **f32)
        hs, cs = torch.empty(Bn, L, H, **f32), torch.empty(Bn, L, H, **f32)
        gates, hks = torch.empty(Bn, L, 4 * H, **f32), torch.empty(Bn, H, **f32)
        _lib.check(lib.mdhp_lstm_forward(ctypes.byref(dims), *map(_ptr, (x, mu, alpha, beta, T, W, U, b, A, Bm,
                                                                          C, Wy, y, hs, cs, gates, hks)),
                                         _stream()), "mdhp_lstm_forward")
        ctx.dims = (Bn, L, D, H, M, beta.shape[1], O)
        ctx.save_for_backward(x, mu, alpha, beta, T, W, U, A, Bm, C, Wy, hs, cs, gates, hks)
        return y

    @staticmethod
    def backward(ctx, dy):
        lib = _lib.load()
        x, mu, alpha, beta, T, W, U, A, Bm, C, Wy, hs, cs, gates, hks = ctx.saved_tensors
        Bn, L, D, H, M, nb, O = ctx.dims
        dims = _lib.MdhpLstmDims(Bn, L, D, H, M, nb, O)
        dy = dy.contiguous().float()
        z = lambda *shape: torch.empty(*shape, dtype=torch.float32, device=x.device)
        dz, dpre = z(Bn, L, 4 * H), z(Bn, H)
        dx, dW, dU, db = z(Bn, L, D), z(4 * H, D), z(4 * H, H), z(4 * H)
        dA, dBm, dC, dWy = z(H, M * M), z(H, nb), z(H, M), z(max(O, 1), H)
        dmu, dalpha, dbeta = z(Bn, M), z(Bn, M, M), z(Bn, nb)
        _lib.check(lib.mdhp_lstm_backward(ctypes.byref(dims), *map(_ptr, (
            x, mu, alpha, beta, T, W, U, A, Bm, C, Wy, hs, cs, gates, hks, dy, dz, dpre, dx, dW, dU, db,
            dA, dBm, dC, dWy, dmu, dalpha, dbeta)), _stream()), "mdhp_lstm_backward")
        return dx, dmu, dalpha, dbeta, None, dW, dU, db, dA, dBm, dC, dWy[:O]


class MdhpLSTM(torch.nn.Module):
    """MDHP-LSTM cell with its own weights (uniform +-1/sqrt(H) initialisation)."""

    def __init__(self, D: int, H: int, M: int, nb: int = 1, O: int = 1, seed: int = 0):
        super().__init__()
        g = torch.Generator().manual_seed(seed)
        k = 1.0 / np.sqrt(H)
        u = lambda *shape: torch.nn.Parameter((torch.rand(*shape, generator=g) * 2 - 1) * k)
        self.W, self.U, self.b = u(4 * H, D), u(4 * H, H), u(4 * H)
        self.A, self.Bm, self.C, self.Wy = u(H, M * M), u(H, nb), u(H, M), u(O, H)

    def forward(self, x, mu, alpha, beta, T_span):
        return MdhpLSTMFunction.apply(x, mu, alpha, beta, T_span, self.W, self.U, self.b, self.A,
                                      self.Bm, self.C, self.Wy)
