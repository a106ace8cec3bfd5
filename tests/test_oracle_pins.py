"""Pins of the FP64 oracle to things other than itself (CPU only).

Each check ties the oracle to the paper's definitions or to mathematics a
plausible mistake would violate: the O(N^2) brute-force double sum
(closed-form lnL, Sec. IV-B.1), quadrature of the compensator (Gamma of the
log-likelihood eq.; App. B), the alpha = 0 closed form, the univariate
(Ozaki 1979) recursion, central finite differences, invariances, a 40-digit
evaluation and the KKT conditions of the fitted optimum.
"""
import numpy as np
import pytest

from oracle import brute


def tiny_window(rng, M, N, T=5.0, ties=True, empty_dim=None, edge=True):
    t = np.sort(rng.uniform(0.0, 0.95 * T, N))
    ids = rng.integers(0, M, N)
    if ties and N >= 10:
        t[3] = t[2]
        t[8] = t[7]
        t[9] = t[7]
        ids[8] = ids[7]  # a same-id tie too
    if edge and N >= 2:
        t[0] = 0.0
        t[-1] = T
    if empty_dim is not None:
        ids[ids == empty_dim] = (empty_dim + 1) % M
    return t, ids.astype(np.int32), T


def params(rng, M, mode):
    mu = rng.uniform(0.2, 1.0, M)
    alpha = rng.uniform(0.0, 0.5, (M, M))
    nb = 1 if mode == 0 else (M if mode == 1 else M * M)
    beta = rng.uniform(0.5, 2.0, nb)
    return mu, alpha, beta


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("weighted", [False, True])
def test_recursion_matches_bruteforce(orc, mode, weighted):
    rng = np.random.default_rng(10 + mode + 3 * weighted)
    for trial in range(3):
        M = 3
        t, ids, T = tiny_window(rng, M, 40, empty_dim=2 if trial == 1 else None)
        w = rng.uniform(0.5, 1.5, len(t)) if weighted else None
        mu, alpha, beta = params(rng, M, mode)
        out = orc.loglik_grad(t, ids, T, mu, alpha, beta, w=w, mode=mode)
        assert out["status"] == 0
        ref = brute.loglik_brute(t, ids, T, mu, alpha, beta, mode, w)
        assert abs(out["lnL"] - ref) <= 1e-12 * max(1.0, abs(ref))
        if weighted:
            gw = brute.event_weight_grad_brute(t, ids, T, mu, alpha, beta, mode, w)
            np.testing.assert_allclose(out["g_w"], gw, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("mode", [0, 2])
def test_compensator_matches_quadrature(orc, mode):
    """Part2 + Part3 = -(integral of the total intensity over [0, T]); pins the
    sign and the '-1' term of App. B."""
    rng = np.random.default_rng(77 + mode)
    M = 2
    t, ids, T = tiny_window(rng, M, 25, T=4.0)
    mu, alpha, beta = params(rng, M, mode)
    out = orc.loglik_grad(t, ids, T, mu, alpha, beta, mode=mode)
    part1 = float(np.sum(np.log(1.0 / out["r"])))
    gamma = brute.compensator_quadrature(t, ids, T, mu, alpha, beta, mode)
    assert abs((out["lnL"] - part1) + gamma) <= 1e-9 * max(1.0, gamma)


def test_alpha_zero_closed_form(orc):
    """alpha = 0: the MLE is mu_i = N_i / T and lnL* = sum N_i log(N_i / T) - N."""
    rng = np.random.default_rng(5)
    M, T = 4, 37.0
    t = np.sort(rng.uniform(0, T, 300))
    ids = rng.integers(0, M, 300).astype(np.int32)
    Ni = np.bincount(ids, minlength=M).astype(float)
    mu = Ni / T
    out = orc.loglik_grad(t, ids, T, mu, np.zeros((M, M)), np.array([1.3]))
    ref = float(np.sum(Ni * np.log(Ni / T)) - Ni.sum())
    assert abs(out["lnL"] - ref) <= 1e-12 * abs(ref)
    np.testing.assert_allclose(out["g_mu"], 0.0, atol=1e-9)
    # the gradient w.r.t. alpha at 0 is sum_n r_n R_j(t_n) - C_ij, not zero in general
    assert np.all(np.isfinite(out["g_alpha"]))


def test_univariate_ozaki(orc):
    """M = 1: Ozaki's recursion A_n = exp(-beta (t_n - t_{n-1})) (1 + A_{n-1})."""
    rng = np.random.default_rng(6)
    T, mu, a, b = 50.0, 0.7, 0.6, 1.4
    t = np.sort(rng.uniform(0, T, 200))
    A, ll = 0.0, 0.0
    for n in range(len(t)):
        if n > 0:
            A = np.exp(-b * (t[n] - t[n - 1])) * (1.0 + A)
        ll += np.log(mu + a * A)
    ll += -mu * T - (a / b) * np.sum(1.0 - np.exp(-b * (T - t)))
    out = orc.loglik_grad(t, np.zeros(200, np.int32), T, [mu], [[a]], [b])
    assert abs(out["lnL"] - ll) <= 1e-11 * abs(ll)


def test_high_precision_value(orc):
    """A hand-sized window (ties, an event at 0-excluded history, the end T)
    evaluated in 40-digit arithmetic with mpmath: log-intensities at the events
    and tanh-sinh quadrature of the intensity between events -- no closed form."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    ev = [(mp.mpf(1) / 2, 0), (mp.mpf(1), 1), (mp.mpf(1), 0), (mp.mpf(7) / 4, 1)]
    T = mp.mpf(5) / 2
    mu = [mp.mpf(3) / 10, mp.mpf(1) / 5]
    al = [[mp.mpf(1) / 2, mp.mpf(1) / 10], [mp.mpf(2) / 5, mp.mpf(1) / 5]]
    be = [[mp.mpf(1), mp.mpf(3) / 2], [mp.mpf(1) / 2, mp.mpf(2)]]

    def lam(i, x, before):
        s = mu[i]
        for tk, j in ev:
            if tk < before:
                s += al[i][j] * mp.exp(-be[i][j] * (x - tk))
        return s

    part1 = mp.fsum(mp.log(lam(i, tk, tk)) for tk, i in ev)
    cuts = sorted({mp.mpf(0), T} | {tk for tk, _ in ev})
    gamma = mp.fsum(mp.quad(lambda x: lam(i, x, b), [a, b])
                    for a, b in zip(cuts[:-1], cuts[1:]) for i in range(2))
    exact = float(part1 - gamma)
    t = np.array([float(x) for x, _ in ev])
    ids = np.array([j for _, j in ev], dtype=np.int32)
    out = orc.loglik_grad(t, ids, 2.5, [0.3, 0.2], [[0.5, 0.1], [0.4, 0.2]],
                          np.array([[1.0, 1.5], [0.5, 2.0]]), mode=2)
    assert abs(out["lnL"] - exact) <= 1e-13 * abs(exact)


def _fd(f, x, h):
    g = np.zeros_like(x)
    for q in range(x.size):
        xp, xm = x.copy(), x.copy()
        step = h * max(1.0, abs(x.flat[q]))
        xp.flat[q] += step
        xm.flat[q] -= step
        g.flat[q] = (f(xp) - f(xm)) / (2 * step)
    return g


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_gradient_central_differences(orc, mode):
    rng = np.random.default_rng(40 + mode)
    M = 3
    t, ids, T = tiny_window(rng, M, 60, T=6.0)
    w = rng.uniform(0.5, 1.5, len(t))
    mu, alpha, beta = params(rng, M, mode)
    out = orc.loglik_grad(t, ids, T, mu, alpha, beta, w=w, mode=mode)
    L = lambda m, a, b, ww: orc.loglik_grad(t, ids, T, m, a, b, w=ww, mode=mode)["lnL"]
    h = 1e-5
    np.testing.assert_allclose(out["g_mu"], _fd(lambda x: L(x, alpha, beta, w), mu, h), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(out["g_alpha"], _fd(lambda x: L(mu, x, beta, w), alpha, h), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(out["g_beta"], _fd(lambda x: L(mu, alpha, x, w), beta, h), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(out["g_w"], _fd(lambda x: L(mu, alpha, beta, x), w, h), rtol=1e-6, atol=1e-7)


def test_invariances(orc):
    rng = np.random.default_rng(8)
    M = 3
    t, ids, T = tiny_window(rng, M, 50, T=8.0)
    mu, alpha, _ = params(rng, M, 1)
    beta = rng.uniform(0.5, 2.0, M)
    base = orc.loglik_grad(t, ids, T, mu, alpha, beta, mode=1)
    # relabel ids by a permutation: parameters permute, lnL is unchanged
    perm = np.array([2, 0, 1])  # new label of old id j is perm[j]
    inv = np.argsort(perm)
    p2 = orc.loglik_grad(t, perm[ids].astype(np.int32), T, mu[inv], alpha[np.ix_(inv, inv)], beta[inv], mode=1)
    assert abs(p2["lnL"] - base["lnL"]) <= 1e-12 * abs(base["lnL"])
    np.testing.assert_allclose(p2["g_alpha"], base["g_alpha"][np.ix_(inv, inv)], rtol=1e-12, atol=1e-13)
    # time scaling t -> c t maps (mu, alpha, beta) -> (mu, alpha, beta) / c and shifts lnL by -N log c
    c = 2.5
    s = orc.loglik_grad(t * c, ids, T * c, mu / c, alpha / c, beta / c, mode=1)
    assert abs(s["lnL"] - (base["lnL"] - len(t) * np.log(c))) <= 1e-11 * abs(base["lnL"])
    # block-diagonal alpha: lnL is the sum over independent sub-processes
    a_bd = alpha.copy()
    a_bd[0, 1:] = 0
    a_bd[1:, 0] = 0
    full = orc.loglik_grad(t, ids, T, mu, a_bd, beta, mode=1)["lnL"]
    s0 = ids == 0
    part_a = orc.loglik_grad(t[s0], np.zeros(s0.sum(), np.int32), T, mu[:1], a_bd[:1, :1], beta[:1])["lnL"]
    s12 = ~s0
    part_b = orc.loglik_grad(t[s12], (ids[s12] - 1).astype(np.int32), T, mu[1:], a_bd[1:, 1:], beta[1:], mode=1)["lnL"]
    assert abs(full - (part_a + part_b)) <= 1e-12 * abs(full)


def test_validation_codes(orc):
    t = np.array([0.1, 0.5, 0.4]); ids = np.array([0, 1, 0], np.int32)
    assert orc.validate(t, ids, 1.0, 2) == orc.E_UNSORTED
    assert orc.validate(np.array([0.1, 0.2]), np.array([0, 2], np.int32), 1.0, 2) == orc.E_ID_RANGE
    assert orc.validate(np.array([0.1, 1.2]), np.array([0, 1], np.int32), 1.0, 2) == orc.E_TIME_RANGE
    assert orc.validate(np.array([0.1, np.nan]), np.array([0, 1], np.int32), 1.0, 2) == orc.E_NONFINITE
    # smallest code wins when several are violated
    assert orc.validate(np.array([0.5, 0.2, 3.0]), np.array([0, 5, 0], np.int32), 1.0, 2) == orc.E_UNSORTED
    # empty window: lnL = -T sum mu
    out = orc.loglik_grad(np.zeros(0), np.zeros(0, np.int32), 3.0, [0.5, 0.25], np.ones((2, 2)), [1.0])
    assert out["status"] == 0 and abs(out["lnL"] + 3.0 * 0.75) < 1e-15
    np.testing.assert_array_equal(out["g_mu"], [-3.0, -3.0])
    np.testing.assert_array_equal(out["g_alpha"], 0.0)


def test_fit_reaches_kkt_point(orc, wl):
    """Fixed beta: lnL is concave in (mu, alpha); the projected-ascent fit must
    land on the same KKT point as an independent bound-constrained optimiser
    (scipy L-BFGS-B on the oracle's value and gradient)."""
    from scipy.optimize import minimize

    M = 4
    mu_t = np.array([0.3, 0.5, 0.2, 0.4])
    a_t = np.array([[0.3, 0.1, 0.0, 0.2], [0.1, 0.2, 0.1, 0.0], [0.0, 0.3, 0.2, 0.1], [0.2, 0.0, 0.1, 0.3]])
    bt = wl.simulate(M, 0, mu_t[None], a_t[None], np.array([[1.0]]), np.array([600]), 11, 99)
    t, ids, T, _ = bt.window(0)
    t = t.astype(np.float64); ids = ids.astype(np.int32); T = float(T)
    beta = np.array([1.0])
    mu0, a0 = orc.cold_init(ids, T, M, beta)
    o = orc.fit_opts(optimizer=1, max_iters=4000, lr=2e-2, tol=1e-13, patience=3)
    res = orc.fit(t, ids, T, mu0, a0, beta, o)
    assert res["status"] in (orc.OK, orc.E_MAXITER)

    def f(x):
        out = orc.loglik_grad(t, ids, T, x[:M], x[M:].reshape(M, M), beta)
        return -out["lnL"], -np.concatenate([out["g_mu"], out["g_alpha"].ravel()])

    x0 = np.concatenate([mu0, a0.ravel()])
    bounds = [(1e-10, None)] * M + [(0.0, None)] * (M * M)
    sol = minimize(f, x0, jac=True, method="L-BFGS-B", bounds=bounds,
                   options=dict(maxiter=20000, ftol=1e-15, gtol=1e-10))
    assert abs(res["lnL"] + sol.fun) <= 1e-6 * abs(sol.fun)
    g = orc.loglik_grad(t, ids, T, res["mu"], res["alpha"], beta)
    ga = g["g_alpha"]
    at_bound = res["alpha"] <= 1e-8
    scale = np.sum(1.0 / np.abs(g["r"]))  # magnitude of the gradient's terms
    assert np.all(ga[at_bound] <= 1e-4 * scale)
    assert np.all(np.abs(ga[~at_bound]) <= 1e-4 * scale)
    assert np.all(np.abs(g["g_mu"]) <= 1e-4 * scale)
