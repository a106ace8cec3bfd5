"""Time-exciting injection attacks (inputs only; no likelihood arithmetic).

The attack rate functions of the paper's table of attack strategies (Sec.
"Time-exciting attack strategies") and its three ways of drawing injection
times (App. "Sampling algorithm"), written from their definitions:

  PLA  power-law acceleration       g(t) = a t^b
  DEA  delayed escalation           g(t) = W1 a1 t^(a1-1)          for t < t1
                                         = W2 a2 exp(gamma (t - t1)) for t >= t1
  ASA  adaptive stealth-oriented     g(t) = C exp(gamma t) / (1 + exp(gamma (t - t0)))^2
  DAM  multi-strategy integration   g(t) = w a1 t^(a1-1) + (1 - w) a2 exp(a2 t)

  NPP  candidates at exponential gaps of mean 1/512 (normalized time), each
       kept with probability g(t) / g_max (thinning of a Poisson process)
  ND   the same with gaps |Normal(1/512, 1/1024)|
  DRP  DAM with a weight w drawn per third of the interval (U(0, 1/3),
       U(1/3, 2/3), U(2/3, 1)), a1 = 3, a2 = 4, then NPP thinning

Times are on the normalized interval [0, 1) of a window; `inject` maps them
onto a simulated window's [0, T_span) as extra events of one message ID.
"""
from __future__ import annotations

import numpy as np

STRATEGIES = ("PLA", "DEA", "ASA", "DAM")
SAMPLERS = ("NPP", "ND", "DRP")
CANDIDATE_GAP = 1.0 / 512.0


def rate(strategy: str, t, p: dict):
    """g(t) of an attack strategy with parameters p (t may be an array)."""
    t = np.asarray(t, dtype=np.float64)
    if strategy == "PLA":
        return p["a"] * np.power(t, p["b"])
    if strategy == "DEA":
        early = p["W1"] * p["a1"] * np.power(np.maximum(t, 1e-300), p["a1"] - 1.0)
        late = p["W2"] * p["a2"] * np.exp(p["gamma"] * (t - p["t1"]))
        return np.where(t < p["t1"], early, late)
    if strategy == "ASA":
        return p["C"] * np.exp(p["gamma"] * t) / (1.0 + np.exp(p["gamma"] * (t - p["t0"]))) ** 2
    if strategy == "DAM":
        return (p["w"] * p["a1"] * np.power(np.maximum(t, 1e-300), p["a1"] - 1.0)
                + (1.0 - p["w"]) * p["a2"] * np.exp(p["a2"] * t))
    raise ValueError(strategy)


def default_params(strategy: str, rng: np.random.Generator) -> dict:
    """A random member of each strategy's family (ranges chosen so every
    strategy injects on the order of a hundred messages per window)."""
    if strategy == "PLA":
        return dict(a=rng.uniform(0.5, 2.0), b=rng.uniform(1.0, 3.0))
    if strategy == "DEA":
        return dict(W1=rng.uniform(0.2, 0.5), a1=rng.uniform(1.5, 2.5), W2=rng.uniform(0.2, 0.5),
                    a2=rng.uniform(1.0, 2.0), gamma=rng.uniform(2.0, 5.0), t1=rng.uniform(0.4, 0.7))
    if strategy == "ASA":
        return dict(C=rng.uniform(1.0, 3.0), gamma=rng.uniform(5.0, 15.0), t0=rng.uniform(0.3, 0.7))
    if strategy == "DAM":
        return dict(w=rng.uniform(0.0, 1.0), a1=3.0, a2=4.0)
    raise ValueError(strategy)


def _g_max(g, lo: float, hi: float, n: int = 4097) -> float:
    """Largest value of g on a fine grid of [lo, hi] (the rate functions are
    smooth and at most unimodal there; the grid maximum is the thinning bound)."""
    return float(np.max(g(np.linspace(lo, hi, n))))


def _thin(rng, g, g_max: float, lo: float, hi: float, gaps: str) -> np.ndarray:
    """Candidates from `lo` at the given gap law until `hi`; keep t with
    probability g(t) / g_max."""
    out = []
    t = lo
    while True:
        if gaps == "exp":
            t += rng.exponential(CANDIDATE_GAP)
        else:  # |Normal(1/512, 1/1024)|
            t += abs(rng.normal(CANDIDATE_GAP, CANDIDATE_GAP / 2.0))
        if t > hi:
            break
        if rng.uniform(0.0, g_max) < g(t):
            out.append(t)
    return np.asarray(out, dtype=np.float64)


def sample(sampler: str, strategy: str, rng: np.random.Generator, p: dict | None = None,
           lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Injection times on [lo, hi) (normalized time)."""
    if sampler == "DRP":  # DAM with one random weight per third of the interval
        edges = lo + (hi - lo) * np.array([1.0 / 3.0, 2.0 / 3.0])
        w = np.array([rng.uniform(0.0, 1 / 3), rng.uniform(1 / 3, 2 / 3), rng.uniform(2 / 3, 1.0)])

        def g(t):
            k = np.searchsorted(edges, t, side="right")
            return rate("DAM", t, dict(w=w[k], a1=3.0, a2=4.0))

        gm = max(_g_max(lambda t: rate("DAM", t, dict(w=wk, a1=3.0, a2=4.0)), lo, hi) for wk in w)
        return _thin(rng, g, gm, lo, hi, "exp")
    p = default_params(strategy, rng) if p is None else p
    g = lambda t: rate(strategy, t, p)
    return _thin(rng, g, _g_max(g, lo, hi), lo, hi, "exp" if sampler == "NPP" else "normal")


def inject(t: np.ndarray, ids: np.ndarray, T: float, attack_times01: np.ndarray, attack_id: int):
    """Merge injection times (normalized to [0, 1)) into a window as events of
    `attack_id`; returns (t, ids) sorted by time (stable: background first on ties)."""
    ta = np.asarray(attack_times01, dtype=np.float64) * float(T)
    t_all = np.concatenate([np.asarray(t, dtype=np.float64), ta])
    id_all = np.concatenate([np.asarray(ids, dtype=np.int64), np.full(len(ta), attack_id)])
    order = np.argsort(t_all, kind="stable")
    return t_all[order], id_all[order]
