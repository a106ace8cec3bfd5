"""Checks of the synthetic workload generator and statistical pins of the oracle.

* time-rescaling theorem (Brown et al. 2002): integrated-intensity increments
  between consecutive events of each type are i.i.d. Exp(1);
* the long-run event rate of a stable MDHP is (I - G)^{-1} mu with G = alpha / beta;
* recovery: the oracle's maximum-likelihood estimate on a long window lies
  within 4 asymptotic standard errors (observed Fisher information, by central
  differences of the oracle gradient) of the generating parameters.
"""
import numpy as np
import pytest
from scipy import stats


def integrated_intensity(t, ids, mu, alpha, beta, M):
    """Lambda_i(t_n) for all i and n (scalar beta), vectorised O(N^2)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros((len(t), M))
    for n in range(len(t)):
        past = t[: n] < t[n]
        d = t[n] - t[:n][past]
        src = ids[:n][past]
        contrib = (1.0 - np.exp(-beta * d)) / beta
        out[n] = mu * t[n] + alpha[:, src] @ contrib
    return out


def test_time_rescaling(wl):
    M = 3
    mu = np.array([0.4, 0.2, 0.3])
    alpha = np.array([[0.3, 0.2, 0.0], [0.1, 0.4, 0.2], [0.2, 0.0, 0.3]])
    beta = 1.5
    bt = wl.simulate(M, 0, mu[None], alpha[None], np.array([[beta]]), np.array([2500]), 7, 1)
    t, ids, T, _ = bt.window(0)
    t = t.astype(np.float64); ids = ids.astype(np.int64)
    L = integrated_intensity(t, ids, mu, alpha, beta, M)
    incs = []
    for i in range(M):
        sel = np.nonzero(ids == i)[0]
        li = L[sel, i]
        incs.append(np.diff(np.concatenate([[0.0], li])))
    incs = np.concatenate(incs)
    p = stats.kstest(incs, "expon").pvalue
    assert p > 1e-3, p


def test_stationary_rate(wl):
    M = 2
    mu = np.array([0.5, 0.3])
    alpha = np.array([[0.4, 0.3], [0.2, 0.5]])
    beta = 2.0
    G = alpha / beta
    rate = np.linalg.solve(np.eye(M) - G, mu)
    bt = wl.simulate_fixed_T(M, 0, mu, alpha, np.array([beta]), 20000.0, 3, 2)
    ids = bt.id.astype(np.int64)
    emp = np.bincount(ids, minlength=M) / 20000.0
    np.testing.assert_allclose(emp, rate, rtol=0.05)


def test_per_source_beta_simulation_rate(wl):
    M = 3
    mu = np.array([0.3, 0.2, 0.4])
    alpha = np.array([[0.2, 0.3, 0.1], [0.1, 0.2, 0.4], [0.3, 0.1, 0.2]])
    beta = np.array([0.8, 1.5, 2.5])
    G = alpha / beta[None, :]
    rate = np.linalg.solve(np.eye(M) - G, mu)
    bt = wl.simulate_fixed_T(M, 1, mu, alpha, beta, 20000.0, 5, 3)
    emp = np.bincount(bt.id.astype(np.int64), minlength=M) / 20000.0
    np.testing.assert_allclose(emp, rate, rtol=0.06)


def test_recovery_within_four_standard_errors(orc, wl):
    from scipy.optimize import minimize

    M = 2
    mu = np.array([0.4, 0.25])
    alpha = np.array([[0.5, 0.2], [0.3, 0.4]])
    beta = np.array([1.0])
    bt = wl.simulate(M, 0, mu[None], alpha[None], beta[None], np.array([20000]), 21, 4)
    t, ids, T, _ = bt.window(0)
    t = t.astype(np.float64); ids = ids.astype(np.int32); T = float(T)

    def f(x):
        out = orc.loglik_grad(t, ids, T, x[:M], x[M:].reshape(M, M), beta)
        return -out["lnL"], -np.concatenate([out["g_mu"], out["g_alpha"].ravel()])

    mu0, a0 = orc.cold_init(ids, T, M, beta)
    sol = minimize(f, np.concatenate([mu0, a0.ravel()]), jac=True, method="L-BFGS-B",
                   bounds=[(1e-8, None)] * (M + M * M), options=dict(maxiter=5000, gtol=1e-9))
    x = sol.x
    # observed information by central differences of the oracle gradient
    H = np.zeros((x.size, x.size))
    for q in range(x.size):
        h = 1e-5 * max(1.0, abs(x[q]))
        xp, xm = x.copy(), x.copy()
        xp[q] += h
        xm[q] -= h
        H[:, q] = (f(xp)[1] - f(xm)[1]) / (2 * h)
    H = 0.5 * (H + H.T)
    se = np.sqrt(np.diag(np.linalg.inv(H)))
    truth = np.concatenate([mu, alpha.ravel()])
    z = np.abs(x - truth) / se
    assert np.all(z < 4.0), z
