"""Pins of the FP64 initializer oracle (CPU): its analytic gradient against
central finite differences of its own loss in exact FP64 arithmetic, the
feature definition on a hand-checkable window, and the AdamW step."""
import numpy as np

from oracle import mlp


def test_loss_gradient_central_differences():
    rng = np.random.default_rng(0)
    M, H, B = 2, 64, 5
    _, n = mlp.layout(M, H)
    params = rng.normal(0, 0.05, n)
    X = rng.uniform(0, 1, (B, mlp.feature_dim(M)))
    mu_cold = rng.uniform(0.1, 1, (B, M))
    beta = rng.uniform(0.5, 2, B)
    mu_t = rng.uniform(0.1, 1, (B, M))
    alpha_t = rng.uniform(0, 0.5, (B, M, M))
    loss, g = mlp.loss_and_grad(params, X, mu_cold, beta, mu_t, alpha_t, M, H, bf=False)
    offs, _ = mlp.layout(M, H)
    idx = []
    for ow, ob, din, dout in offs:
        idx += list(rng.integers(ow, ow + din * dout, 4)) + [ob, ob + dout - 1]
    for q in idx:
        h = 1e-6
        pp, pm = params.copy(), params.copy()
        pp[q] += h
        pm[q] -= h
        fd = (mlp.loss_and_grad(pp, X, mu_cold, beta, mu_t, alpha_t, M, H, bf=False)[0] -
              mlp.loss_and_grad(pm, X, mu_cold, beta, mu_t, alpha_t, M, H, bf=False)[0]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-6 * max(1.0, abs(fd)), (q, fd, g[q])


def test_features_hand_window():
    # types 0,1; events: (0.0,0) (1.0,1) (1.0,0) (3.0,1); T = 4, N = 4, scale = 1
    row, mu_cold = mlp.features([0.0, 1.0, 1.0, 3.0], [0, 1, 0, 1], 4.0, 1.5, 2)
    M, B = 2, mlp.BINS
    np.testing.assert_allclose(row[:2], [0.5, 0.5])
    h = row[M:M + M * M * B].reshape(M, M, B)
    # event 1 (t=1, type 1): gap to type 0 = 1 -> bin 16; the tie at t=1 is not seen
    # event 2 (t=1, type 0): gap to type 0 = 1 -> bin 16 (type 1 at t=1 is a tie: unseen)
    # event 3 (t=3, type 1): gap to type 0 = 2 -> bin 17; to type 1 = 2 -> bin 17
    assert h[1, 0, 16] == 0.5 and h[1, 0, 17] == 0.5 and h[1, 1, 17] == 1.0
    assert h[0, 0, 16] == 1.0 and h[0, 1].sum() == 0.0
    assert row[M + M * M * B] == np.log(4) and row[M + M * M * B + 2] == 1.5
    np.testing.assert_allclose(mu_cold, [0.5 * 2 / 4, 0.5 * 2 / 4])


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159, 0.0])
    r = mlp.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0  # tie to even
    assert r[2] == 1.0 + 2 ** -7
    assert abs(r[3] + 3.140625) < 1e-12


def test_adamw_first_step():
    M, H = 1, 64
    _, n = mlp.layout(M, H)
    p = np.ones(n)
    g = np.full(n, 0.5)
    w, m, v = mlp.adamw_step(p, g, np.zeros(n), np.zeros(n), 1, 1e-3, 0.1, M, H)
    offs, _ = mlp.layout(M, H)
    ow, ob, din, dout = offs[0]
    # first step: m_hat = g, v_hat = g^2 -> step lr * sign(g); decay only on matrices
    assert abs(w[ow] - (1 - 1e-3 * 0.1 - 1e-3 * 0.5 / (0.5 + 1e-8))) < 1e-12
    assert abs(w[ob] - (1 - 1e-3 * 0.5 / (0.5 + 1e-8))) < 1e-12


def test_head_closed_form():
    """Head of the initializer: mu_i = mu_cold_i exp(clamp(y_i, -6, 6)) and
    alpha_ij = (beta_j / M) softplus(y_ij), column j scaled by source j's decay.
    Checked at points where softplus has a known value: softplus(0) = ln 2,
    softplus(y) - softplus(-y) = y, softplus(40) = 40 to double precision."""
    M, B = 2, 3
    mu_cold = np.array([[0.2, 0.4], [1.0, 3.0], [0.5, 0.5]])
    beta = np.array([[1.0, 2.0], [0.5, 0.5], [3.0, 1.0]])  # per source
    y = np.zeros((B, M + M * M))
    y[1, :M] = [10.0, -10.0]                    # clamped to +-6
    y[1, M:] = [40.0, -40.0, 3.0, -3.0]
    y[2, :M] = [0.7, -1.3]
    y[2, M:] = [1.5, -1.5, 0.0, 0.0]
    mu, alpha = mlp.head(y, mu_cold, beta, M)
    np.testing.assert_allclose(mu[0], mu_cold[0], rtol=1e-15)
    np.testing.assert_allclose(mu[1], [3.0 * np.exp(0.0) * np.exp(6.0) / 3.0, 3.0 * np.exp(-6.0)], rtol=1e-14)
    np.testing.assert_allclose(mu[2], mu_cold[2] * np.exp([0.7, -1.3]), rtol=1e-14)
    ln2 = np.log(2.0)
    np.testing.assert_allclose(alpha[0], [[ln2 / 2, 2 * ln2 / 2], [ln2 / 2, 2 * ln2 / 2]], rtol=1e-15)
    np.testing.assert_allclose(alpha[1, 0, 0], 0.25 * 40.0, rtol=1e-15)
    assert 0.0 < alpha[1, 0, 1] <= 0.25 * np.exp(-40.0) * (1 + 1e-12)
    assert abs((alpha[1, 1, 0] - alpha[1, 1, 1]) / 0.25 - 3.0) <= 1e-13
    # row 0 of window 2: softplus(1.5) - softplus(-1.5) = 1.5, columns scaled by beta = (3, 1)
    assert abs(alpha[2, 0, 0] / (3.0 / M) - alpha[2, 0, 1] / (1.0 / M) - 1.5) <= 1e-13
    np.testing.assert_allclose(alpha[2, 1], [3.0 / M * ln2, 1.0 / M * ln2], rtol=1e-15)
    # scalar beta broadcasts over sources
    mu_s, alpha_s = mlp.head(y, mu_cold, np.array([1.0, 0.5, 3.0]), M)
    np.testing.assert_allclose(alpha_s[0], ln2 / 2, rtol=1e-15)
