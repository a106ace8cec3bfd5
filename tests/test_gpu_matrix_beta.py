"""The full beta_ij matrix (the paper's general form, Sec. II) on the GPU:
fixed-beta fits through the decoupled kernels against the FP64 oracle, which
implements the matrix form directly (full M x M recursion).  Same tolerances
as test_gpu_parity: lnL 1e-5 relative; fitted parameters 1e-4 of the group's
scale after the same number of iterations."""
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


def _batch(wl, M, B, seed, lo=50, hi=3000, ties=False):
    rng = np.random.default_rng(seed)
    betas = np.exp(rng.uniform(np.log(0.5), np.log(2.0), size=(B, M * M)))
    mu, alpha = wl.sample_params(rng, B, M, 2, betas, rng.uniform(0.2, 0.8, B))
    counts = wl.log_uniform_counts(rng, B, lo, hi)
    counts[0] = 1
    bt = wl.simulate(M, 2, mu, alpha, betas, counts, seed=seed, stream=40 + M)
    if ties:  # repeat timestamps inside windows (ties within and across chunks)
        for b in range(1, B):
            o0, o1 = bt.offsets[b], bt.offsets[b + 1]
            if o1 - o0 > 20:
                bt.t[o0 + 5:o0 + 9] = bt.t[o0 + 5]
                mid = (o0 + o1) // 2
                bt.t[mid:mid + 3] = bt.t[mid]
    return bt


def _gpu_fit(mdhp, bt, opts, configure=None, weights=None):
    M, B = bt.M, bt.B
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    if weights is not None:
        db.weights = torch.from_numpy(weights).cuda()
    plan = mdhp.Plan(M, 2, B, int(bt.counts.max()))
    if configure is not None:
        configure(plan)
    mu = torch.zeros(B, M, device="cuda")
    al = torch.zeros(B, M, M, device="cuda")
    be = torch.from_numpy(bt.beta.astype(np.float32)).cuda()
    out = plan.fit(db, opts, mu, al, be)
    torch.cuda.synchronize()
    return (out["loglik"].cpu().numpy(), out["iters"].cpu().numpy(), out["status"].cpu().numpy(),
            mu.cpu().numpy(), al.cpu().numpy(), be.cpu().numpy())


def _oracle_fit(orc, bt, b, o, weights=None):
    t, ids, T, _ = bt.window(b)
    M = bt.M
    beta = bt.beta[b].astype(np.float32).astype(np.float64)
    m0, a0 = orc.cold_init(ids, float(T), M, beta, mode=2)
    w = None
    if weights is not None:
        w = weights[bt.offsets[b]:bt.offsets[b + 1]].astype(np.float64)
    return orc.fit(t, ids, float(T), m0, a0, beta, o, w=w, mode=2)


def _compare(orc, bt, got, o, iters, sample, weights=None):
    ll, it, st, mu, al, be = got
    assert np.all(st == 0) and np.all(it == iters)
    np.testing.assert_array_equal(be, bt.beta.astype(np.float32))  # beta is not fitted
    for b in sample:
        r = _oracle_fit(orc, bt, b, o, weights)
        assert r["status"] == 0 and r["iters"] == iters
        assert abs(ll[b] - r["lnL"]) <= LL_RTOL * abs(r["lnL"]), (b, ll[b], r["lnL"])
        assert np.all(np.abs(mu[b] - r["mu"]) <= P_RTOL * np.abs(r["mu"]).max()), b
        assert np.all(np.abs(al[b] - r["alpha"]) <= P_RTOL * np.abs(r["alpha"]).max() + 1e-30), b


@pytest.mark.parametrize("M", [4, 16, 32])
@pytest.mark.parametrize("optimizer", [0, 1])
def test_matrix_beta_fit_matches_oracle(mdhp, orc, wl, M, optimizer):
    bt = _batch(wl, M, 24, seed=300 + M, hi=3000 if M < 32 else 1500)
    iters, lr = 40, (1e-2 if optimizer == 0 else 3e-3)
    got = _gpu_fit(mdhp, bt, mdhp.FitOptions(optimizer=optimizer, max_iters=iters, lr=lr, init=1))
    o = orc.fit_opts(optimizer=optimizer, max_iters=iters, lr=lr)
    _compare(orc, bt, got, o, iters, range(bt.B))


def test_matrix_beta_ties_and_weights(mdhp, orc, wl):
    bt = _batch(wl, 8, 16, seed=77, ties=True)
    rng = np.random.default_rng(3)
    weights = rng.uniform(0.5, 1.5, bt.n_events).astype(np.float32)
    iters = 30
    got = _gpu_fit(mdhp, bt, mdhp.FitOptions(optimizer=0, max_iters=iters, lr=1e-2, init=1), weights=weights)
    o = orc.fit_opts(optimizer=0, max_iters=iters, lr=1e-2)
    _compare(orc, bt, got, o, iters, range(bt.B), weights)


def test_matrix_beta_launch_variants(mdhp, orc, wl):
    bt = _batch(wl, 16, 160, seed=91, lo=20, hi=4000)
    iters = 25
    opts = mdhp.FitOptions(optimizer=0, max_iters=iters, lr=1e-2, init=1)
    o = orc.fit_opts(optimizer=0, max_iters=iters, lr=1e-2)
    sample = [0, 1, 2] + list(range(3, bt.B, 23))
    variants = [
        lambda p: None,  # defaults: split 256 x 1 + 64
        lambda p: p.set_split(False),
        lambda p: (p.set_split(False), p.set_shape(128, 4, 0)),
        lambda p: (p.set_split(False), p.set_shape(256, 4, 0)),
        lambda p: (p.set_split(False), p.set_shape(64, 4, 1024)),  # shared-memory class
    ]
    for conf in variants:
        _compare(orc, bt, _gpu_fit(mdhp, bt, opts, conf), o, iters, sample)


def test_matrix_beta_unsupported_requests(mdhp, wl):
    bt = _batch(wl, 4, 4, seed=5)
    M, B = bt.M, bt.B
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    plan = mdhp.Plan(M, 2, B, int(bt.counts.max()))
    mu = torch.zeros(B, M, device="cuda")
    al = torch.zeros(B, M, M, device="cuda")
    be = torch.from_numpy(bt.beta.astype(np.float32)).cuda()
    with pytest.raises(mdhp.MdhpError):  # beta cannot be learned in matrix form
        plan.fit(db, mdhp.FitOptions(max_iters=3, fit_beta=1), mu, al, be)
    with pytest.raises(mdhp.MdhpError):  # single evaluations stay scalar / per source
        mdhp.loglik_grad(db, mu + 0.5, al, be)
    with pytest.raises(mdhp.MdhpError):  # the decoupled kernels need a window bound
        mdhp.Plan(M, 2, B, 0)
