"""Parity at the benchmark sizes, in the launch configuration the benchmark
times: the whole batch is fitted on the GPU, a sample of windows (the longest,
the shortest and random ones) is re-fitted one by one by the FP64 oracle with
the same options, and every window is checked for the properties that hold at
any size (status, iteration count, finite lnL and parameters, floors).

Tolerances as in test_gpu_parity: lnL 1e-5 relative, fitted parameters 1e-4
of the group's scale after the same number of iterations."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LL_RTOL = 1e-5
P_RTOL = 1e-4


@pytest.fixture(scope="module")
def mdhp():
    import paper_2411_10258_gb300 as m

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return m


def _sample(counts, k_long, k_short, k_rand, seed):
    order = np.argsort(counts, kind="stable")
    rng = np.random.default_rng(seed)
    pick = list(order[-k_long:]) + list(order[:k_short])
    pick += list(rng.choice(len(counts), k_rand, replace=False))
    return sorted(set(int(b) for b in pick))


def _host_window(db, b):
    o0, o1 = int(db.offsets[b].item()), int(db.offsets[b + 1].item())
    t = db.t[o0:o1].cpu().numpy().astype(np.float64)
    ids = db.id[o0:o1].cpu().numpy().astype(np.int32)
    return t, ids, float(db.T[b].item())


def _oracle_refit(orc, db, sample, beta0, M, mode, o):
    """Re-fit the sampled windows with the FP64 oracle from the same cold
    start, windows spread over the host cores (OpenMP)."""
    ts, ids, Ts = [], [], []
    for b in sample:
        t, u, T = _host_window(db, b)
        ts.append(t.astype(np.float32)); ids.append(u.astype(np.int16)); Ts.append(T)
    off = np.zeros(len(sample) + 1, np.int64)
    np.cumsum([len(x) for x in ts], out=off[1:])
    nb = 1 if mode == 0 else M
    b0 = np.asarray(beta0, dtype=np.float64).reshape(len(beta0), -1)[sample]
    mu0 = np.zeros((len(sample), M)); a0 = np.zeros((len(sample), M, M))
    for q in range(len(sample)):
        mu0[q], a0[q] = orc.cold_init(ids[q].astype(np.int32), Ts[q], M, b0[q], mode=mode)
    return orc.fit_batch(off, np.concatenate(ts), np.concatenate(ids), np.asarray(Ts, np.float32), M,
                         mode, mu0, a0, b0.reshape(len(sample), nb), o)


def _check(orc, db, out, mu, al, be_fit, beta0, sample, o, M, iters, fit_beta=False, mode=0):
    st = out["status"].cpu().numpy()
    it = out["iters"].cpu().numpy()
    ll = out["loglik"].cpu().numpy()
    mu_h, al_h = mu.cpu().numpy(), al.cpu().numpy()
    assert np.all(st == 0)
    assert np.all(it == iters)
    assert np.all(np.isfinite(ll)) and np.all(np.isfinite(mu_h)) and np.all(np.isfinite(al_h))
    assert np.all(mu_h >= 1e-10 * 0.999) and np.all(al_h >= 0.0)
    r = _oracle_refit(orc, db, sample, beta0, M, mode, o)
    assert np.all(r["status"] == 0) and np.all(r["iters"] == iters)
    for q, b in enumerate(sample):
        assert abs(ll[b] - r["lnL"][q]) <= LL_RTOL * abs(r["lnL"][q]), (b, ll[b], r["lnL"][q])
        # mu: relative per entry (an entry below 1e-3 of the window's largest
        # rate is compared at that scale); alpha: relative to the group's
        # largest entry, since entries at the alpha = 0 bound have no scale
        rm = r["mu"][q]
        assert np.all(np.abs(mu_h[b] - rm) <= P_RTOL * np.maximum(np.abs(rm), 1e-3 * np.abs(rm).max())), b
        assert np.all(np.abs(al_h[b] - r["alpha"][q]) <= P_RTOL * np.abs(r["alpha"][q]).max() + 1e-30), b
        if fit_beta:
            be = be_fit.cpu().numpy()[b]
            assert np.all(np.abs(be - r["beta"][q]) <= P_RTOL * np.abs(r["beta"][q])), b


def test_workload2_full_size_autotuned(mdhp, orc, wl):
    """4,096 windows x M=16, 200 PGD iterations, lr 1e-2, cold start, plan
    autotuned as the benchmark does."""
    bt = wl.make_workload(2, B=4096, seed=2024)
    M, B, iters = bt.M, bt.B, 200
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    beta = torch.from_numpy(bt.beta.astype(np.float32)).cuda()
    plan = mdhp.Plan(M, 0, B, int(bt.counts.max()))
    opts = mdhp.FitOptions(optimizer=0, max_iters=iters, lr=1e-2, init=1)
    mu = torch.zeros(B, M, device="cuda")
    al = torch.zeros(B, M, M, device="cuda")
    plan.autotune(db, opts, mu, al, beta, tune_iters=20)
    out = plan.fit(db, opts, mu, al, beta)
    torch.cuda.synchronize()
    sample = _sample(bt.counts, 4, 4, 8, seed=1)
    o = orc.fit_opts(optimizer=0, max_iters=iters, lr=1e-2)
    _check(orc, db, out, mu, al, beta, bt.beta, sample, o, M, iters)


def test_workload5_full_size(mdhp, orc, wl):
    """65,536 windows x M=32 (counts 100-10,000, 10 % injected component),
    projected Adam lr 2e-2 from the cold start, 100 iterations (tol = 0 so
    that every window runs the same count)."""
    p = wl.make_params(5, B=65536, seed=2024)
    M, B, iters = 32, 65536, 100
    db, sst = mdhp.simulate(M, 0, p["mu"], p["alpha"], p["beta"], p["counts"], seed=2024, stream_id=5)
    assert int((sst != 0).sum().item()) == 0
    beta = torch.from_numpy(p["beta"].astype(np.float32)).cuda()
    plan = mdhp.Plan(M, 0, B, int(p["counts"].max()))
    opts = mdhp.FitOptions(optimizer=1, max_iters=iters, lr=2e-2, init=1)
    mu = torch.zeros(B, M, device="cuda")
    al = torch.zeros(B, M, M, device="cuda")
    out = plan.fit(db, opts, mu, al, beta)
    torch.cuda.synchronize()
    # the longest windows (up to 10,000 events: the wide CTAs of the two-ended
    # split fit them), the shortest, random ones, and injected windows of
    # every length class
    counts = p["counts"]
    order = np.argsort(counts, kind="stable")
    rng = np.random.default_rng(5)
    inj = np.nonzero(p["meta"]["injected"])[0]
    inj_sorted = inj[np.argsort(counts[inj])]
    sample = list(order[-3:]) + list(order[:2]) + list(rng.choice(B, 4, replace=False))
    sample += [int(inj_sorted[0]), int(inj_sorted[len(inj_sorted) // 2]), int(inj_sorted[-1])]
    sample = sorted(set(int(b) for b in sample))
    assert counts[sample].max() >= 9000
    o = orc.fit_opts(optimizer=1, max_iters=iters, lr=2e-2)
    _check(orc, db, out, mu, al, beta, p["beta"].astype(np.float32), sample, o, M, iters)


def test_workload3_full_size_learned_beta(mdhp, orc, wl):
    """512 windows x M=64, 20k-100k events, beta per source learned by
    projected Adam (lr 1e-2) from the generating beta, 20 iterations; the
    three longest windows (about 100k events, where FP32 rounding along the
    recursion accumulates most) and the two shortest are re-fitted by the
    oracle (O(N M^2) per evaluation, windows in parallel on the host cores)."""
    p = wl.make_params(3, B=512, seed=2024)
    M, B, iters = 64, 512, 20
    db, sst = mdhp.simulate(M, 1, p["mu"], p["alpha"], p["beta"], p["counts"], seed=2024, stream_id=3)
    assert int((sst != 0).sum().item()) == 0
    beta0 = p["beta"].astype(np.float32)
    be = torch.from_numpy(beta0.copy()).cuda()
    plan = mdhp.Plan(M, 1, B, 0)
    opts = mdhp.FitOptions(optimizer=1, max_iters=iters, lr=1e-2, init=1, fit_beta=1)
    mu = torch.zeros(B, M, device="cuda")
    al = torch.zeros(B, M, M, device="cuda")
    out = plan.fit(db, opts, mu, al, be)
    torch.cuda.synchronize()
    order = np.argsort(p["counts"], kind="stable")
    sample = sorted(int(b) for b in list(order[:2]) + list(order[-3:]))
    assert p["counts"][sample].max() >= 95000
    o = orc.fit_opts(optimizer=1, max_iters=iters, lr=1e-2, fit_beta=1)
    _check(orc, db, out, mu, al, be, beta0, sample, o, M, iters, fit_beta=True, mode=1)
    assert np.all(be.cpu().numpy() >= 1e-6 * 0.999)
