"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (FP32 arithmetic with Kahan-compensated lnL):
  lnL        |gpu - ref| <= 1e-5 |ref|
  gradients  |gpu - ref| <= 1e-4 max(|ref|, s) with s the magnitude of the
             group's terms: T for d/dmu, sum_n r_n R_j(t_n) (= g_alpha_ij + C_j)
             for d/dalpha, and the compensator's beta-derivative scale for d/dbeta
  fitted parameters after the same iteration count:
             |gpu - ref| <= 1e-4 max(|ref|, max |ref| over the group)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LL_RTOL = 1e-5
G_RTOL = 1e-4
P_RTOL = 1e-4


@pytest.fixture(scope="module")
def mdhp():
    import paper_2411_10258_gb300 as m

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return m


def _bm(beta, M, mode):
    beta = np.asarray(beta, dtype=np.float64).reshape(-1)
    return np.full(M, beta[0]) if mode == 0 else beta


def compensator(t, ids, T, M, beta, mode, w=None):
    """C_j = sum_{k in j} w_k (1 - exp(-beta_j (T - t_k))) / beta_j (tolerance scale only)."""
    b = _bm(beta, M, mode)
    w = np.ones(len(t)) if w is None else w
    C = np.zeros(M)
    for j in range(M):
        s = ids == j
        C[j] = np.sum(w[s] * -np.expm1(-b[j] * (T - t[s]))) / b[j]
    return C


def check_window(orc, bt, b, mu, alpha, beta, gpu, idx, beta_grad, weights=None, gw=None):
    t, ids, T, _ = bt.window(b)
    s0, s1 = int(bt.offsets[b]), int(bt.offsets[b + 1])
    t64 = t.astype(np.float64); ids32 = ids.astype(np.int32); T = float(T)
    w = None if weights is None else weights[s0:s1].astype(np.float64)
    M, mode = bt.M, bt.beta_mode
    ref = orc.loglik_grad(t64, ids32, T, mu.astype(np.float64), alpha.astype(np.float64),
                          beta.astype(np.float64), w=w, mode=mode)
    assert gpu["status"][idx] == ref["status"] == 0
    ll = gpu["loglik"][idx]
    assert abs(ll - ref["lnL"]) <= LL_RTOL * abs(ref["lnL"]), (b, ll, ref["lnL"])
    np.testing.assert_array_less(np.abs(gpu["g_mu"][idx] - ref["g_mu"]),
                                 G_RTOL * np.maximum(np.abs(ref["g_mu"]), T) + 1e-30)
    C = compensator(t64, ids32, T, M, beta, mode, w)
    s_alpha = np.abs(ref["g_alpha"] + C[None, :])
    s_alpha = np.maximum(s_alpha, s_alpha.max() * 1e-3)
    err = np.abs(gpu["g_alpha"][idx] - ref["g_alpha"])
    assert np.all(err <= G_RTOL * np.maximum(np.abs(ref["g_alpha"]), s_alpha)), err.max()
    if beta_grad:
        bj = _bm(beta, M, mode)
        scale = np.sum(alpha * (C / bj)[None, :], axis=0)  # per source
        if mode == 0:
            scale = np.array([scale.sum()])
        e = np.abs(gpu["g_beta"][idx] - ref["g_beta"])
        assert np.all(e <= G_RTOL * np.maximum(np.abs(ref["g_beta"]), scale)), (e, ref["g_beta"])
    if gw is not None:
        g = gw[s0:s1]
        sc = np.maximum(np.abs(ref["g_w"]), np.abs(ref["g_w"]).max())
        assert np.all(np.abs(g - ref["g_w"]) <= G_RTOL * sc)


def run_llg(mdhp, bt, mu, alpha, beta, beta_grad=False, weight_grad=False, max_events=None):
    db = mdhp.DeviceBatch.from_host(bt, "cuda", max_events=max_events)
    out = mdhp.loglik_grad(db, torch.from_numpy(mu.astype(np.float32)).cuda(),
                           torch.from_numpy(alpha.astype(np.float32)).cuda(),
                           torch.from_numpy(beta.astype(np.float32)).cuda(),
                           beta_grad=beta_grad, weight_grad=weight_grad)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()}


def perturbed_params(bt, rng, scale=0.3):
    mu = bt.mu_true * rng.uniform(1 - scale, 1 + scale, bt.mu_true.shape)
    alpha = bt.alpha_true * rng.uniform(1 - scale, 1 + scale, bt.alpha_true.shape)
    return mu.astype(np.float32), alpha.astype(np.float32)


@pytest.mark.parametrize("staged", [True, False])
@pytest.mark.parametrize("beta_grad", [False, True])
def test_loglik_grad_m16_scalar_beta(mdhp, orc, wl, staged, beta_grad):
    bt = wl.make_workload(2, B=12, seed=101)
    rng = np.random.default_rng(1)
    mu, alpha = perturbed_params(bt, rng)
    beta = bt.beta
    gpu = run_llg(mdhp, bt, mu, alpha, beta, beta_grad=beta_grad,
                  max_events=None if staged else 0)
    for b in range(bt.B):
        check_window(orc, bt, b, mu[b], alpha[b], beta[b], gpu, b, beta_grad)


@pytest.mark.parametrize("M", [1, 3, 4, 7, 8, 32])
def test_loglik_grad_other_widths(mdhp, orc, wl, M):
    rng = np.random.default_rng(M)
    B = 6
    mu_t = rng.uniform(0.1, 1.0, (B, M))
    a_t = rng.uniform(0, 1, (B, M, M))
    a_t *= (0.5 / wl.spectral_radius(a_t))[:, None, None]
    beta = np.ones((B, 1))
    counts = rng.integers(50, 3000, B)
    bt = wl.simulate(M, 0, mu_t, a_t, beta, counts, 5, 50 + M)
    mu, alpha = perturbed_params(bt, rng)
    gpu = run_llg(mdhp, bt, mu, alpha, bt.beta, beta_grad=True)
    for b in range(B):
        check_window(orc, bt, b, mu[b], alpha[b], bt.beta[b], gpu, b, True)


@pytest.mark.parametrize("staged", [True, False])
def test_loglik_grad_per_source_beta_m64(mdhp, orc, wl, staged):
    rng = np.random.default_rng(3)
    M, B = 64, 4
    betas = np.exp(rng.uniform(np.log(0.5), np.log(2.0), (B, M)))
    mu_t, a_t = wl.sample_params(rng, B, M, 1, betas, rng.uniform(0.2, 0.8, B))
    counts = np.array([300, 2500, 7000, 1])
    bt = wl.simulate(M, 1, mu_t, a_t, betas, counts, 9, 77)
    mu, alpha = perturbed_params(bt, rng)
    gpu = run_llg(mdhp, bt, mu, alpha, bt.beta, beta_grad=True, max_events=None if staged else 0)
    for b in range(B):
        check_window(orc, bt, b, mu[b], alpha[b], bt.beta[b], gpu, b, True)


def test_event_weight_gradient(mdhp, orc, wl):
    rng = np.random.default_rng(4)
    for M, mode in ((16, 0), (32, 1)):
        B = 4
        betas = np.ones((B, 1)) if mode == 0 else rng.uniform(0.5, 2, (B, M))
        mu_t, a_t = wl.sample_params(rng, B, M, mode, betas, rng.uniform(0.2, 0.8, B))
        bt = wl.simulate(M, mode, mu_t, a_t, betas, rng.integers(100, 4000, B), 13, 80 + M)
        bt.weights = rng.uniform(0.5, 1.5, bt.n_events).astype(np.float32)
        mu, alpha = perturbed_params(bt, rng)
        gpu = run_llg(mdhp, bt, mu, alpha, bt.beta, beta_grad=True, weight_grad=True)
        for b in range(B):
            check_window(orc, bt, b, mu[b], alpha[b], bt.beta[b], gpu, b, True,
                         weights=bt.weights, gw=gpu["g_w"])


def _handmade_batch(wl, windows, M, T_list, mode=0, beta=1.0):
    """Build a Batch from explicit (t, id) lists (edge cases)."""
    counts = np.array([len(w[0]) for w in windows], dtype=np.int64)
    off = np.zeros(len(windows) + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    t = np.concatenate([np.asarray(w[0], np.float32) for w in windows]) if off[-1] else np.zeros(0, np.float32)
    ids = np.concatenate([np.asarray(w[1], np.int16) for w in windows]) if off[-1] else np.zeros(0, np.int16)
    B = len(windows)
    nb = 1 if mode == 0 else M
    bt = wl.Batch(M, mode, off, t, ids, np.asarray(T_list, np.float32),
                  np.full((B, nb), beta, np.float32), np.zeros((B, M)), np.zeros((B, M, M)),
                  np.full((B, nb), beta))
    return bt


def test_edge_cases(mdhp, orc, wl):
    rng = np.random.default_rng(5)
    M = 4
    tie_heavy = np.sort(rng.choice(np.linspace(0, 10, 40), 600)).astype(np.float32)
    windows = [
        ([], []),                                            # empty window
        ([0.5], [2]),                                        # one event
        ([1.0] * 50, list(rng.integers(0, M, 50))),          # one tie group
        (list(tie_heavy), list(rng.integers(0, M, 600))),    # ties everywhere, across chunks
        ([0.0, 0.0, 3.0, 5.0], [0, 1, 0, 3]),                # events at 0 and at T
        (list(np.sort(rng.uniform(0, 9, 900))), [1] * 900),  # a single id
    ]
    bt = _handmade_batch(wl, windows, M, [2.0, 1.0, 1.0, 10.0, 5.0, 9.0])
    mu = rng.uniform(0.2, 1, (bt.B, M)).astype(np.float32)
    alpha = rng.uniform(0, 0.4, (bt.B, M, M)).astype(np.float32)
    for staged in (True, False):
        gpu = run_llg(mdhp, bt, mu, alpha, bt.beta, beta_grad=True, max_events=None if staged else 0)
        for b in range(bt.B):
            check_window(orc, bt, b, mu[b], alpha[b], bt.beta[b], gpu, b, True)


def test_invalid_windows_report_status(mdhp, orc, wl):
    M = 3
    windows = [
        ([0.1, 0.5, 0.4], [0, 1, 0]),       # unsorted
        ([0.1, 0.2], [0, 3]),               # id out of range
        ([0.1, 1.5], [0, 1]),               # t > T
        ([0.1, float("nan")], [0, 1]),      # NaN
        ([0.5, 0.2, 3.0], [0, 5, 0]),       # several problems: smallest code wins
        ([0.1, 0.2, 0.3], [0, 1, 2]),       # valid
    ]
    bt = _handmade_batch(wl, windows, M, [1.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    mu = np.full((bt.B, M), 0.5, np.float32)
    alpha = np.full((bt.B, M, M), 0.1, np.float32)
    gpu = run_llg(mdhp, bt, mu, alpha, bt.beta)
    for b in range(bt.B):
        t, ids, T, _ = bt.window(b)
        assert gpu["status"][b] == orc.validate(t.astype(np.float64), ids.astype(np.int32), float(T), M)
    assert gpu["status"][-1] == 0


@pytest.mark.parametrize("path", ["auto", "recursion"])
@pytest.mark.parametrize("optimizer", [0, 1])
def test_fit_matches_oracle_fixed_iterations(mdhp, orc, wl, optimizer, path):
    bt = wl.make_workload(2, B=10, seed=202)
    M, B = bt.M, bt.B
    iters = 60
    lr = 1e-2 if optimizer == 0 else 3e-3
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    plan = mdhp.Plan(M, 0, B, int(bt.counts.max()))
    plan.set_path(path)
    mu = torch.zeros(B, M, device="cuda")
    alpha = torch.zeros(B, M, M, device="cuda")
    beta = torch.from_numpy(bt.beta).cuda()
    out = plan.fit(db, mdhp.FitOptions(optimizer=optimizer, max_iters=iters, lr=lr, init=1),
                   mu, alpha, beta)
    torch.cuda.synchronize()
    o = orc.fit_opts(optimizer=optimizer, max_iters=iters, lr=lr)
    g_mu, g_alpha = out["mu"].cpu().numpy(), out["alpha"].cpu().numpy()
    ll, it, st = out["loglik"].cpu().numpy(), out["iters"].cpu().numpy(), out["status"].cpu().numpy()
    for b in range(B):
        t, ids, T, _ = bt.window(b)
        m0, a0 = orc.cold_init(ids, float(T), M, bt.beta[b])
        r = orc.fit(t, ids, float(T), m0, a0, bt.beta[b].astype(np.float64), o)
        assert st[b] == r["status"] and it[b] == r["iters"] == iters
        assert abs(ll[b] - r["lnL"]) <= LL_RTOL * abs(r["lnL"])
        np.testing.assert_array_less(np.abs(g_mu[b] - r["mu"]), P_RTOL * np.abs(r["mu"]).max())
        np.testing.assert_array_less(np.abs(g_alpha[b] - r["alpha"]),
                                     P_RTOL * np.abs(r["alpha"]).max() + 1e-30)


def test_fit_learned_per_source_beta(mdhp, orc, wl):
    rng = np.random.default_rng(8)
    M, B = 32, 4
    betas = rng.uniform(0.5, 2.0, (B, M))
    mu_t, a_t = wl.sample_params(rng, B, M, 1, betas, rng.uniform(0.2, 0.8, B))
    bt = wl.simulate(M, 1, mu_t, a_t, betas, np.array([800, 3000, 12000, 200]), 17, 91)
    iters = 25
    beta0 = np.full((B, M), 1.0, np.float32)
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    plan = mdhp.Plan(M, 1, B, 0)
    mu = torch.zeros(B, M, device="cuda")
    alpha = torch.zeros(B, M, M, device="cuda")
    beta = torch.from_numpy(beta0.copy()).cuda()
    out = plan.fit(db, mdhp.FitOptions(optimizer=1, max_iters=iters, lr=2e-3, fit_beta=1, init=1),
                   mu, alpha, beta)
    torch.cuda.synchronize()
    o = orc.fit_opts(optimizer=1, max_iters=iters, lr=2e-3, fit_beta=1)
    for b in range(B):
        t, ids, T, _ = bt.window(b)
        m0, a0 = orc.cold_init(ids, float(T), M, beta0[b])
        r = orc.fit(t, ids, float(T), m0, a0, beta0[b].astype(np.float64), o)
        assert out["iters"][b].item() == r["iters"]
        assert abs(out["loglik"][b].item() - r["lnL"]) <= LL_RTOL * abs(r["lnL"])
        for name, g in (("mu", out["mu"][b]), ("alpha", out["alpha"][b]), ("beta", out["beta"][b])):
            gv = g.cpu().numpy()
            np.testing.assert_array_less(np.abs(gv - r[name]), P_RTOL * np.abs(r[name]).max() + 1e-30)


def test_fit_convergence_tolerance(mdhp, orc, wl):
    """With tol > 0 both sides stop on the same rule; the stopping iteration may
    differ by rounding, the reached lnL may not."""
    bt = wl.make_workload(2, B=6, seed=303)
    M, B = bt.M, bt.B
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    plan = mdhp.Plan(M, 0, B, int(bt.counts.max()))
    mu = torch.zeros(B, M, device="cuda")
    alpha = torch.zeros(B, M, M, device="cuda")
    beta = torch.from_numpy(bt.beta).cuda()
    opts = mdhp.FitOptions(optimizer=1, max_iters=3000, lr=1e-2, tol=1e-7, init=1)
    out = plan.fit(db, opts, mu, alpha, beta)
    torch.cuda.synchronize()
    o = orc.fit_opts(optimizer=1, max_iters=3000, lr=1e-2, tol=1e-7)
    for b in range(B):
        t, ids, T, _ = bt.window(b)
        m0, a0 = orc.cold_init(ids, float(T), M, bt.beta[b])
        r = orc.fit(t, ids, float(T), m0, a0, bt.beta[b].astype(np.float64), o)
        assert out["status"][b].item() == r["status"]
        assert abs(out["loglik"][b].item() - r["lnL"]) <= 1e-5 * abs(r["lnL"])
