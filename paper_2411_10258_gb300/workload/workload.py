"""Seeded synthetic MDHP workloads (inputs only; no likelihood arithmetic here).

The paper's windows (STEIA9, 128 SOME/IP messages per window) are not
available, so windows are simulated from known exponential-kernel MDHP
parameters by Ogata thinning (``hawkes_sim.c``).  Shapes follow the five
workloads the library is measured on:

==== ========================================================================
name what
==== ========================================================================
1    one window, M=4, scalar beta=1, T=100 s, ~2,000 events (mu~U(0.1,1)
     scaled by a common factor so the expected count is 2,000), rho(alpha/beta)=0.5
2    4,096 windows, M=16, counts log-uniform [200, 5000], rho ~ U(0.2, 0.8),
     scalar beta in {0.5, 1, 2} for the whole batch
3    512 long windows, M=64, counts log-uniform [2e4, 1e5], beta per source
     (log-uniform [0.5, 2]), rho ~ U(0.2, 0.8)
4    initializer training/eval windows, M=16, counts log-uniform [500, 5000],
     beta per window in {0.5, 1, 2}
5    65,536 windows, M=32, counts log-uniform [100, 10000], 10 % carry one
     injected self-exciting component (alpha_kk = 0.9 beta, mu_k x 5)
6    the shapes of workload 2 with the full decay matrix: beta_ij log-uniform
     [0.5, 2] per window and pair, rho(alpha / beta) ~ U(0.2, 0.8)
==== ========================================================================

Layout produced (what the C ABI consumes): CSR ``offsets`` int64[B+1],
``t`` float32[sum N] (seconds from window start, sorted), ``id`` int16[sum N],
``T`` float32[B].  Parameters use row = target, column = source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hawkes_sim.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBPATH = os.path.join(_BUILD, "libhawkes_sim.so")
_lib = None

BASE_SEED = 2024  # the seed the paper's GDS timing runs use (Sec. V-C)


def build(force: bool = False) -> str:
    """Compile the simulator (plain C + OpenMP) in-tree; returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIBPATH) or os.path.getmtime(_LIBPATH) < os.path.getmtime(_SRC):
        tmp = _LIBPATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.sim_window_key.restype = ctypes.c_uint64
        lib.sim_window_key.argtypes = [ctypes.c_uint64] * 3
        lib.sim_window.restype = ctypes.c_int64
        lib.sim_window.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_int64,
                                   ctypes.c_double, ctypes.c_uint64, ctypes.c_int64, P, P, P]
        lib.sim_batch.restype = ctypes.c_int
        lib.sim_batch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P, P,
                                  ctypes.c_uint64, ctypes.c_uint64, P, P, P, ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def nbeta(mode: int, M: int) -> int:
    return 1 if mode == 0 else (M if mode == 1 else M * M)


def beta_matrix(beta: np.ndarray, mode: int, M: int) -> np.ndarray:
    """beta_ij for every (target i, source j); beta has a trailing axis of size nb."""
    beta = np.asarray(beta, dtype=np.float64)
    lead = beta.shape[:-1]
    if mode == 0:
        return np.broadcast_to(beta[..., None], lead + (M, M)).copy()
    if mode == 1:
        return np.broadcast_to(beta[..., None, :], lead + (M, M)).copy()
    return beta.reshape(lead + (M, M)).copy()


def spectral_radius(G: np.ndarray) -> np.ndarray:
    return np.max(np.abs(np.linalg.eigvals(G)), axis=-1)


@dataclass
class Batch:
    """A CSR batch of windows plus the parameters that generated it."""

    M: int
    beta_mode: int
    offsets: np.ndarray  # int64 [B+1]
    t: np.ndarray  # float32 [sum N]
    id: np.ndarray  # int16 [sum N]
    T: np.ndarray  # float32 [B]
    beta: np.ndarray  # float32 [B, nb]  (the decay the fit uses / starts from)
    mu_true: np.ndarray  # float64 [B, M]
    alpha_true: np.ndarray  # float64 [B, M, M]
    beta_true: np.ndarray  # float64 [B, nb]
    weights: np.ndarray | None = None  # float32 [sum N] or None
    meta: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return int(self.T.shape[0])

    @property
    def counts(self) -> np.ndarray:
        return np.diff(self.offsets)

    @property
    def n_events(self) -> int:
        return int(self.offsets[-1])

    def window(self, b: int):
        """(t float32, id int16, T float32, weights or None) of window b."""
        s, e = int(self.offsets[b]), int(self.offsets[b + 1])
        w = None if self.weights is None else self.weights[s:e]
        return self.t[s:e], self.id[s:e], np.float32(self.T[b]), w

    def subset(self, idx) -> "Batch":
        idx = np.asarray(idx, dtype=np.int64)
        cnt = self.counts[idx]
        off = np.zeros(len(idx) + 1, dtype=np.int64)
        np.cumsum(cnt, out=off[1:])
        sl = np.concatenate([np.arange(self.offsets[b], self.offsets[b + 1]) for b in idx]) \
            if len(idx) else np.zeros(0, dtype=np.int64)
        return Batch(self.M, self.beta_mode, off, self.t[sl].copy(), self.id[sl].copy(),
                     self.T[idx].copy(), self.beta[idx].copy(), self.mu_true[idx].copy(),
                     self.alpha_true[idx].copy(), self.beta_true[idx].copy(),
                     None if self.weights is None else self.weights[sl].copy(), dict(self.meta))


def sample_params(rng: np.random.Generator, B: int, M: int, mode: int, beta: np.ndarray,
                  rho: np.ndarray, mu_lo: float = 0.1, mu_hi: float = 1.0):
    """mu ~ U(mu_lo, mu_hi), alpha ~ U(0, 1) rescaled so that rho(alpha / beta) = rho."""
    mu = rng.uniform(mu_lo, mu_hi, size=(B, M))
    alpha = rng.uniform(0.0, 1.0, size=(B, M, M))
    G = alpha / beta_matrix(beta, mode, M)
    sr = spectral_radius(G)
    alpha *= (np.asarray(rho, dtype=np.float64) / sr)[:, None, None]
    return mu, alpha


def inject_component(rng: np.random.Generator, mu, alpha, beta, mode, M, frac):
    """Raise one self-excitation per chosen window: alpha_kk = 0.9 beta_kk, mu_k x 5;
    if rho(alpha/beta) >= 0.98, shrink row k's off-diagonal entries until rho = 0.95."""
    B = mu.shape[0]
    chosen = rng.random(B) < frac
    ks = rng.integers(0, M, size=B)
    bm = beta_matrix(beta, mode, M)
    for b in np.nonzero(chosen)[0]:
        k = int(ks[b])
        alpha[b, k, k] = 0.9 * bm[b, k, k]
        mu[b, k] *= 5.0
        G = alpha[b] / bm[b]
        if spectral_radius(G) >= 0.98:
            lo, hi = 0.0, 1.0
            off = alpha[b, k].copy()
            for _ in range(60):
                s = 0.5 * (lo + hi)
                a2 = alpha[b].copy()
                a2[k] = off * s
                a2[k, k] = off[k]
                if spectral_radius(a2 / bm[b]) > 0.95:
                    hi = s
                else:
                    lo = s
            alpha[b, k] = off * lo
            alpha[b, k, k] = off[k]
    return chosen, ks


def simulate(M: int, mode: int, mu, alpha, beta, counts, seed: int, stream: int,
             nthreads: int = 0) -> Batch:
    """Simulate B windows with exactly counts[b] events each."""
    lib = _load()
    B = len(counts)
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    off = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(B, nbeta(mode, M)))
    t = np.empty(int(off[-1]), dtype=np.float32)
    ids = np.empty(int(off[-1]), dtype=np.int16)
    T = np.empty(B, dtype=np.float32)
    rc = lib.sim_batch(B, M, mode, _ptr(mu), _ptr(alpha), _ptr(beta), _ptr(counts), _ptr(off),
                       seed, stream, _ptr(t), _ptr(ids), _ptr(T), nthreads)
    if rc != 0:
        raise RuntimeError("simulation failed")
    return Batch(M, mode, off, t, ids, T, beta.astype(np.float32), mu, alpha, beta.copy())


def simulate_fixed_T(M: int, mode: int, mu, alpha, beta, T: float, seed: int, stream: int,
                     cap: int = 1 << 22) -> Batch:
    """One window observed on [0, T] (random count)."""
    lib = _load()
    mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(M)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64).reshape(M * M)
    beta = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(nbeta(mode, M)))
    t = np.empty(cap, dtype=np.float64)
    ids = np.empty(cap, dtype=np.int32)
    Tout = np.zeros(1, dtype=np.float64)
    key = lib.sim_window_key(seed, stream, 0)
    n = lib.sim_window(M, mode, _ptr(mu), _ptr(alpha), _ptr(beta), 0, float(T), key, cap,
                       _ptr(t), _ptr(ids), _ptr(Tout))
    if n < 0:
        raise RuntimeError("capacity exceeded")
    off = np.array([0, n], dtype=np.int64)
    return Batch(M, mode, off, t[:n].astype(np.float32), ids[:n].astype(np.int16),
                 np.array([T], dtype=np.float32), beta.astype(np.float32)[None, :],
                 mu[None, :], alpha.reshape(1, M, M), beta[None, :])


def log_uniform_counts(rng, B, lo, hi):
    return np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), size=B))).astype(np.int64)


def make_params(name: int, B: int | None = None, seed: int = BASE_SEED, beta: float = 1.0) -> dict:
    """Parameters and event counts of workload 2..5 (see module docstring) without
    simulating: dict(M, mode, mu, alpha, beta, counts, meta).  Feeds the CPU
    generator here and the library's GPU simulator alike."""
    rng = np.random.default_rng([seed, name])
    meta = dict(name=name)
    if name == 2:
        B = 4096 if B is None else B
        M, mode = 16, 0
        betas = np.full((B, 1), float(beta))
        rho = rng.uniform(0.2, 0.8, size=B)
        mu, alpha = sample_params(rng, B, M, mode, betas, rho)
        counts = log_uniform_counts(rng, B, 200, 5000)
    elif name == 3:
        B = 512 if B is None else B
        M, mode = 64, 1
        betas = np.exp(rng.uniform(np.log(0.5), np.log(2.0), size=(B, M)))
        rho = rng.uniform(0.2, 0.8, size=B)
        mu, alpha = sample_params(rng, B, M, mode, betas, rho)
        counts = log_uniform_counts(rng, B, 20000, 100000)
    elif name == 4:
        B = 16384 if B is None else B
        M, mode = 16, 0
        betas = rng.choice(np.array([0.5, 1.0, 2.0]), size=(B, 1))
        rho = rng.uniform(0.2, 0.8, size=B)
        mu, alpha = sample_params(rng, B, M, mode, betas, rho)
        counts = log_uniform_counts(rng, B, 500, 5000)
    elif name == 6:
        B = 4096 if B is None else B
        M, mode = 16, 2
        betas = np.exp(rng.uniform(np.log(0.5), np.log(2.0), size=(B, M * M)))
        rho = rng.uniform(0.2, 0.8, size=B)
        mu, alpha = sample_params(rng, B, M, mode, betas, rho)
        counts = log_uniform_counts(rng, B, 200, 5000)
    elif name == 5:
        B = 65536 if B is None else B
        M, mode = 32, 0
        betas = np.full((B, 1), float(beta))
        rho = rng.uniform(0.2, 0.8, size=B)
        mu, alpha = sample_params(rng, B, M, mode, betas, rho)
        injected, ks = inject_component(rng, mu, alpha, betas, mode, M, 0.10)
        counts = log_uniform_counts(rng, B, 100, 10000)
        meta.update(injected=injected, injected_k=ks)
    else:
        raise ValueError(f"unknown workload {name}")
    return dict(M=M, mode=mode, mu=mu, alpha=alpha, beta=betas, counts=counts, meta=meta)


def make_workload(name: int, B: int | None = None, seed: int = BASE_SEED, beta: float = 1.0,
                  nthreads: int = 0) -> Batch:
    """Build one of the five workloads (see module docstring); B overrides the
    window count (the shapes and distributions stay those of the workload)."""
    if name == 1:
        rng = np.random.default_rng([seed, name])
        M, mode = 4, 0
        mu = rng.uniform(0.1, 1.0, size=(1, M))
        alpha = rng.uniform(0.0, 1.0, size=(1, M, M))
        alpha *= 0.5 / spectral_radius(alpha / 1.0)[:, None, None]
        G = alpha[0] / 1.0
        rate = np.linalg.solve(np.eye(M) - G, mu[0]).sum()
        c = 2000.0 / (100.0 * rate)
        mu *= c
        bt = simulate_fixed_T(M, mode, mu[0], alpha[0], np.array([1.0]), 100.0, seed, name)
        bt.meta.update(name=1, mu_scale=float(c))
        return bt
    p = make_params(name, B, seed, beta)
    bt = simulate(p["M"], p["mode"], p["mu"], p["alpha"], p["beta"], p["counts"], seed, name, nthreads)
    bt.meta.update(p["meta"])
    return bt
