"""The MDHP-LSTM oracle pinned by central finite differences (every weight,
the inputs and the MDHP parameters), and by special cases that reduce to
known cells: hks = 1 everywhere gives the plain LSTM recursion written out
step by step; a zero forget gate with hks = 1 makes c_t depend on step t
alone."""
import numpy as np

from oracle import lstm


def _params(rng, B=3, L=5, D=4, H=3, M=2, nb=2, O=2, scale=0.5):
    p = dict(x=rng.normal(size=(B, L, D)), mu=rng.uniform(0.1, 1, (B, M)),
             alpha=rng.uniform(0, 0.5, (B, M, M)), beta=rng.uniform(0.5, 2, (B, nb)),
             T=rng.uniform(5, 20, B), W=rng.normal(scale=scale, size=(4 * H, D)),
             U=rng.normal(scale=scale, size=(4 * H, H)), b=rng.normal(scale=scale, size=4 * H),
             A=rng.normal(scale=scale, size=(H, M * M)), Bm=rng.normal(scale=0.05, size=(H, nb)),
             C=rng.normal(scale=scale, size=(H, M)), Wy=rng.normal(scale=scale, size=(O, H)))
    return p


def _loss(p, dy):
    y, _ = lstm.forward(**p)
    return float(np.sum(y * dy))


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    p = _params(rng)
    y, cache = lstm.forward(**p)
    dy = rng.normal(size=y.shape)
    g = lstm.backward(cache, dy)
    names = dict(x="dx", W="dW", U="dU", b="db", A="dA", Bm="dBm", C="dC", Wy="dWy", mu="dmu",
                 alpha="dalpha", beta="dbeta")
    h = 1e-6
    for k, gk in names.items():
        base = p[k]
        num = np.zeros(base.size)
        flat = base.reshape(-1)
        for j in range(base.size):
            orig = flat[j]
            flat[j] = orig + h
            lp = _loss(p, dy)
            flat[j] = orig - h
            lm = _loss(p, dy)
            flat[j] = orig
            num[j] = (lp - lm) / (2 * h)
        got = np.asarray(g[gk]).reshape(-1)
        np.testing.assert_allclose(got, num, rtol=1e-5, atol=1e-7, err_msg=k)


def test_unit_hawkes_gate_is_the_plain_lstm():
    rng = np.random.default_rng(1)
    p = _params(rng, M=2, nb=2)
    p["A"][:] = 0.0; p["Bm"][:] = 0.0; p["C"][:] = 0.0
    # tanh(0) = 0 would zero the cell: shift by a constant large enough that hks = 1 in float64
    p["C"][:, 0] = 40.0 / p["mu"][:, 0].min()
    y, cache = lstm.forward(**p)
    assert np.allclose(cache["hks"], 1.0)
    B, L, D = p["x"].shape
    H = p["U"].shape[1]
    sig = lambda z: 1 / (1 + np.exp(-z))
    h = np.zeros((B, H)); c = np.zeros((B, H))
    for t in range(L):
        z = p["x"][:, t] @ p["W"].T + h @ p["U"].T + p["b"]
        c = sig(z[:, H:2 * H]) * c + sig(z[:, :H]) * np.tanh(z[:, 2 * H:3 * H])
        h = sig(z[:, 3 * H:]) * np.tanh(c)
        np.testing.assert_allclose(y[:, t], h @ p["Wy"].T, rtol=1e-12)


def test_zero_forget_gate_forgets():
    rng = np.random.default_rng(2)
    p = _params(rng)
    H = p["U"].shape[1]
    p["b"][H:2 * H] = -1e3  # f = sigmoid(-1000) = 0
    _, cache = lstm.forward(**p)
    G = cache["gates"]
    i, g = G[:, :, :H], G[:, :, 2 * H:3 * H]
    np.testing.assert_allclose(cache["c"], cache["hks"][:, None, :] * i * g, rtol=1e-12, atol=1e-300)
