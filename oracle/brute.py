"""O(N^2) brute-force definitions in numpy (test infrastructure only).

These are the plain definitions of arXiv 2411.10258, written without any
recursion, used to pin the C oracle's recursion on tiny inputs:

* ``intensity`` -- Sec. II, MDHP intensity eq.: lambda_i(v) = theta_i +
  sum_j sum_{k: T_j^k < v} w_k alpha_ij exp(-beta_ij (v - T_j^k)).
* ``loglik_brute`` -- Sec. IV-B.1 closed-form lnL (Part1 + Part2 + Part3).
* ``compensator_quadrature`` -- Gamma of the log-likelihood eq. (the integral
  of the total intensity over [0, T_span]) by adaptive quadrature between
  consecutive event times, independent of App. B's closed form.
"""
from __future__ import annotations

import numpy as np


def _bm(beta, M, mode):
    beta = np.asarray(beta, dtype=np.float64).reshape(-1)
    if mode == 0:
        return np.full((M, M), beta[0])
    if mode == 1:
        return np.broadcast_to(beta[None, :], (M, M)).copy()
    return beta.reshape(M, M)


def intensity(v, t, ids, mu, alpha, beta, mode, w=None, i=None):
    """lambda_i(v) (all i if i is None) from the definition (strict t_k < v)."""
    t = np.asarray(t, dtype=np.float64)
    ids = np.asarray(ids, dtype=np.int64)
    M = len(mu)
    bm = _bm(beta, M, mode)
    w = np.ones_like(t) if w is None else np.asarray(w, dtype=np.float64)
    past = t < v
    lam = np.array(mu, dtype=np.float64).copy()
    for k in np.nonzero(past)[0]:
        j = ids[k]
        lam += w[k] * alpha[:, j] * np.exp(-bm[:, j] * (v - t[k]))
    return lam if i is None else lam[i]


def loglik_brute(t, ids, T, mu, alpha, beta, mode, w=None):
    """Part1 + Part2 + Part3 from the definitions (double sum for Part1)."""
    t = np.asarray(t, dtype=np.float64)
    ids = np.asarray(ids, dtype=np.int64)
    M = len(mu)
    alpha = np.asarray(alpha, dtype=np.float64).reshape(M, M)
    bm = _bm(beta, M, mode)
    w = np.ones_like(t) if w is None else np.asarray(w, dtype=np.float64)
    part1 = 0.0
    for n in range(len(t)):
        i = ids[n]
        part1 += np.log(intensity(t[n], t, ids, mu, alpha, beta, mode, w, i))
    part2 = -T * np.sum(mu)
    part3 = 0.0
    for i in range(M):
        for j in range(M):
            sel = ids == j
            part3 += alpha[i, j] / bm[i, j] * np.sum(w[sel] * (np.exp(-bm[i, j] * (T - t[sel])) - 1.0))
    return part1 + part2 + part3


def compensator_quadrature(t, ids, T, mu, alpha, beta, mode, w=None):
    """sum_i int_0^T lambda_i(v) dv by scipy quad on each inter-event interval."""
    from scipy.integrate import quad

    t = np.asarray(t, dtype=np.float64)
    M = len(mu)
    alpha = np.asarray(alpha, dtype=np.float64).reshape(M, M)
    edges = np.unique(np.concatenate([[0.0], t, [T]]))
    total = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        if b <= a:
            continue
        f = lambda v: float(np.sum(intensity(v, t, ids, mu, alpha, beta, mode, w)))
        val, _ = quad(f, a, b, epsabs=1e-13, epsrel=1e-12, limit=200)
        total += val
    return total


def event_weight_grad_brute(t, ids, T, mu, alpha, beta, mode, w=None):
    """d lnL / d w_k from the definition: sum over later events n of
    r_n alpha_{u_n u_k} exp(-beta (t_n - t_k)) minus the compensator term."""
    t = np.asarray(t, dtype=np.float64)
    ids = np.asarray(ids, dtype=np.int64)
    M = len(mu)
    alpha = np.asarray(alpha, dtype=np.float64).reshape(M, M)
    bm = _bm(beta, M, mode)
    w = np.ones_like(t) if w is None else np.asarray(w, dtype=np.float64)
    r = np.array([1.0 / intensity(t[n], t, ids, mu, alpha, beta, mode, w, ids[n])
                  for n in range(len(t))])
    g = np.zeros(len(t))
    for k in range(len(t)):
        j = ids[k]
        later = t > t[k]
        acc = np.sum(r[later] * alpha[ids[later], j] * np.exp(-bm[ids[later], j] * (t[later] - t[k])))
        comp = np.sum(alpha[:, j] * (1.0 - np.exp(-bm[:, j] * (T - t[k]))) / bm[:, j])
        g[k] = acc - comp
    return g
