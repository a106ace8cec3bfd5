"""Pins of the oracle's fit iteration, stopping rule and cold start (CPU).

The fit (projected ascent on f = lnL / max(N, 1), Sec. IV-B.2 leaves the
optimiser open; the library's reading is the iteration stated in
include/mdhp.h) is pinned on a window whose optimum and whole trajectory are
known in closed form: events so sparse against 1/beta that d lnL / d alpha_ij
is negative at alpha = 0 everywhere on the path, so the projection holds every
alpha_ij at its floor 0 and the problem reduces to the alpha = 0 likelihood

    lnL(mu) = sum_i N_i log mu_i - T sum_i mu_i,   d lnL / d mu_i = N_i / mu_i - T

(Sec. IV-B.1 closed form with Part3 = 0).  The expected iterates are written
out step by step from that closed form, so a wrong 1/N scale, a step of the
wrong sign, a projection that lets alpha go negative, an off-by-one in the
evaluation count, in the patience streak or in the restore rule each fail a
check here.
"""
import numpy as np
import pytest

M = 2
BETA = 6.0


def sparse_window():
    """40 events one second apart (type pattern 0, 0, 1), T = 40.5 s."""
    N = 40
    t = 0.5 + np.arange(N, dtype=np.float64)
    ids = np.array([1 if n % 3 == 2 else 0 for n in range(N)], dtype=np.int32)
    return t, ids, 40.5


def closed_lnl(mu, Ni, T):
    return float(np.sum(Ni * np.log(mu)) - T * np.sum(mu))


def closed_grad(mu, Ni, T):
    return Ni / mu - T


@pytest.fixture(scope="module")
def win(orc):
    t, ids, T = sparse_window()
    Ni = np.bincount(ids, minlength=M).astype(np.float64)
    return t, ids, T, Ni


def _assert_alpha_grad_negative(orc, t, ids, T, mus):
    # precondition of the reduction: at alpha = 0 the alpha-gradient is < 0 on
    # every point of the trajectory, so projected steps keep alpha at 0
    for mu in mus:
        g = orc.loglik_grad(t, ids, T, mu, np.zeros((M, M)), [BETA])
        assert np.all(g["g_alpha"] < 0.0), g["g_alpha"]


def test_pgd_two_steps_by_hand(orc, win):
    t, ids, T, Ni = win
    N = len(t)
    lr = 0.1
    mu0 = np.array([0.3, 0.1])
    # theta_{k+1} = max(theta_k + lr * g_k / N, floor) with g_k = N_i / mu_i - T
    mu1 = mu0 + lr * closed_grad(mu0, Ni, T) / N
    mu2 = mu1 + lr * closed_grad(mu1, Ni, T) / N
    assert np.all(mu1 > 0) and np.all(mu2 > 0)
    _assert_alpha_grad_negative(orc, t, ids, T, [mu0, mu1, mu2])
    o = orc.fit_opts(optimizer=0, max_iters=3, lr=lr)
    res = orc.fit(t, ids, T, mu0, np.zeros((M, M)), [BETA], o)
    assert res["status"] == orc.OK
    assert res["iters"] == 3  # evaluations at theta_0, theta_1, theta_2
    np.testing.assert_allclose(res["mu"], mu2, rtol=1e-13)
    assert np.all(res["alpha"] == 0.0)
    assert abs(res["lnL"] - closed_lnl(mu2, Ni, T)) <= 1e-12 * abs(res["lnL"])
    # max_iters = 1 evaluates theta_0 only and returns it unchanged
    res1 = orc.fit(t, ids, T, mu0, np.zeros((M, M)), [BETA], orc.fit_opts(max_iters=1, lr=lr))
    assert res1["iters"] == 1
    np.testing.assert_array_equal(res1["mu"], mu0)
    assert abs(res1["lnL"] - closed_lnl(mu0, Ni, T)) <= 1e-12 * abs(res1["lnL"])


def test_adam_two_steps_by_hand(orc, win):
    t, ids, T, Ni = win
    N = len(t)
    lr, b1, b2, eps = 0.05, 0.9, 0.999, 1e-8
    mu0 = np.array([0.3, 0.1])
    # step 1: m = (1 - b1) g, v = (1 - b2) g^2, bias-corrected m/(1-b1) = g, v/(1-b2) = g^2
    g0 = closed_grad(mu0, Ni, T) / N
    m, v = (1 - b1) * g0, (1 - b2) * g0 * g0
    mu1 = mu0 + lr * (m / (1 - b1)) / (np.sqrt(v / (1 - b2)) + eps)
    # the first Adam step moves every coordinate by lr (sign of its gradient)
    np.testing.assert_allclose(np.abs(mu1 - mu0), lr, rtol=1e-6)
    g1 = closed_grad(mu1, Ni, T) / N
    m, v = b1 * m + (1 - b1) * g1, b2 * v + (1 - b2) * g1 * g1
    mu2 = mu1 + lr * (m / (1 - b1 ** 2)) / (np.sqrt(v / (1 - b2 ** 2)) + eps)
    _assert_alpha_grad_negative(orc, t, ids, T, [mu0, mu1, mu2])
    o = orc.fit_opts(optimizer=1, max_iters=3, lr=lr)
    res = orc.fit(t, ids, T, mu0, np.zeros((M, M)), [BETA], o)
    assert res["status"] == orc.OK and res["iters"] == 3
    np.testing.assert_allclose(res["mu"], mu2, rtol=1e-12)
    assert np.all(res["alpha"] == 0.0)  # alpha's Adam steps are projected back to 0


def _pgd_sequence(mu0, Ni, T, N, lr, K):
    mus, lnls = [mu0], [closed_lnl(mu0, Ni, T)]
    for _ in range(K - 1):
        mus.append(mus[-1] + lr * closed_grad(mus[-1], Ni, T) / N)
        lnls.append(closed_lnl(mus[-1], Ni, T))
    return mus, np.array(lnls)


@pytest.mark.parametrize("patience", [1, 3])
def test_stopping_rule_patience(orc, win, patience):
    """Stop at the patience-th consecutive evaluation k with
    |lnL_k - lnL_{k-1}| <= tol |lnL_k|.  Along this smooth ascent the relative
    changes d_k decrease strictly, so with tol between d_{k1} and d_{k1-1} the
    first small change is at k1 and the fit ends after k1 + patience
    evaluations, returning theta at that evaluation."""
    t, ids, T, Ni = win
    N, lr, K = len(t), 0.05, 60
    mu0 = np.array([0.3, 0.1])
    mus, lnls = _pgd_sequence(mu0, Ni, T, N, lr, K)
    d = np.abs(np.diff(lnls)) / np.abs(lnls[1:])  # d[k - 1] belongs to evaluation k
    k1 = 12
    assert np.all(np.diff(d[: k1 + patience + 2]) < 0), d
    tol = float(np.sqrt(d[k1 - 1] * d[k1 - 2]))  # d_{k1} <= tol < d_{k1 - 1}
    _assert_alpha_grad_negative(orc, t, ids, T, mus[: k1 + patience + 1])
    o = orc.fit_opts(optimizer=0, max_iters=K, lr=lr, tol=tol, patience=patience)
    res = orc.fit(t, ids, T, mu0, np.zeros((M, M)), [BETA], o)
    assert res["status"] == orc.OK
    last = k1 + patience - 1
    assert res["iters"] == last + 1, (res["iters"], last + 1)
    np.testing.assert_allclose(res["mu"], mus[last], rtol=1e-12)
    assert abs(res["lnL"] - lnls[last]) <= 1e-12 * abs(lnls[last])
    # a tolerance never met runs out the evaluations and reports it
    o2 = orc.fit_opts(optimizer=0, max_iters=20, lr=lr, tol=1e-30, patience=patience)
    res2 = orc.fit(t, ids, T, mu0, np.zeros((M, M)), [BETA], o2)
    assert res2["status"] == orc.E_MAXITER and res2["iters"] == 20
    np.testing.assert_allclose(res2["mu"], mus[19], rtol=1e-12)


def test_restore_on_nonfinite(orc, win):
    """With mu_floor = 0 a long step clamps mu_i to 0; the next evaluation has
    lambda = 0 at the type-i events (ln 0 = -inf), so the fit stops, restores
    the previous point and reports its lnL and MDHP_E_NONFINITE."""
    t, ids, T, Ni = win
    N, lr = len(t), 50.0
    mu0 = 3.0 * Ni / T  # above the optimum: both gradients are -2T/3
    mu1 = np.maximum(mu0 + lr * closed_grad(mu0, Ni, T) / N, 0.0)
    assert np.all(mu1 == 0.0)
    o = orc.fit_opts(optimizer=0, max_iters=10, lr=lr, mu_floor=0.0)
    res = orc.fit(t, ids, T, mu0, np.zeros((M, M)), [BETA], o)
    assert res["status"] == orc.E_NONFINITE
    assert res["iters"] == 1  # one finite evaluation (theta_0) was kept
    np.testing.assert_array_equal(res["mu"], mu0)
    assert np.all(res["alpha"] == 0.0)
    assert abs(res["lnL"] - closed_lnl(mu0, Ni, T)) <= 1e-12 * abs(res["lnL"])


def test_cold_start_rule(orc):
    """mu_i = 0.5 max(N_i, 1) / T (a type with no events counts as one) and
    alpha_ij = 0.5 beta_ij / M, i.e. alpha / beta has spectral radius 0.5."""
    ids = np.array([0] * 5 + [2] * 12, dtype=np.int32)
    T, Mm = 7.0, 3
    np.random.default_rng(0).shuffle(ids)
    for mode, beta in ((0, np.array([1.7])), (1, np.array([0.5, 1.0, 2.0])),
                       (2, np.random.default_rng(1).uniform(0.3, 3.0, 9))):
        mu, alpha = orc.cold_init(ids, T, Mm, beta, mode=mode)
        np.testing.assert_allclose(mu, [5 * 0.5 / 7.0, 0.5 / 7.0, 12 * 0.5 / 7.0], rtol=1e-15)
        bm = np.broadcast_to(beta.reshape(-1), (Mm, Mm)) if mode != 2 else beta.reshape(Mm, Mm)
        if mode == 0:
            bm = np.full((Mm, Mm), beta[0])
        rho = np.max(np.abs(np.linalg.eigvals(alpha / bm)))
        assert abs(rho - 0.5) <= 1e-12, (mode, rho)
        # per-source: column j is scaled by beta_j (source j's decay)
        if mode == 1:
            np.testing.assert_allclose(alpha[1] / alpha[1, 0], beta / beta[0], rtol=1e-15)
