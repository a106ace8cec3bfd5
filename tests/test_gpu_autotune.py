"""Autotuner (mdhp_plan_autotune): the chosen shape is one of the candidates,
the caller's parameters survive tuning, fits with the tuned shape agree with
the default shape to rounding, and the cache file written by one plan is
applied by the next plan created with the same arguments."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdhp():
    import paper_2411_10258_gb300 as m

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return m


def _fit(mdhp, plan, db, opts, beta0, M):
    B = db.B
    mu = torch.zeros(B, M, device="cuda")
    al = torch.zeros(B, M, M, device="cuda")
    be = beta0.clone()
    out = plan.fit(db, opts, mu, al, be)
    torch.cuda.synchronize()
    return out["loglik"].cpu().numpy(), mu.cpu().numpy(), out["status"].cpu().numpy()


def test_decoupled_path_tuning_and_cache(mdhp, wl, tmp_path):
    bt = wl.make_workload(2, B=384, seed=5)
    M, B = bt.M, bt.B
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    beta0 = torch.from_numpy(bt.beta).cuda()
    # projected gradient ascent: unlike Adam it does not amplify the rounding
    # of a different summation order near a stationary point, so the fitted
    # parameters themselves can be compared
    opts = mdhp.FitOptions(optimizer=0, max_iters=60, lr=1e-2, init=1)
    cache = str(tmp_path / "tune.json")
    ref_plan = mdhp.Plan(M, 0, B, int(bt.counts.max()))
    l_ref, mu_ref, st_ref = _fit(mdhp, ref_plan, db, opts, beta0, M)
    assert np.all(st_ref == 0)

    plan = mdhp.Plan(M, 0, B, int(bt.counts.max()), autotune_cache=cache)
    g = torch.Generator(device="cuda").manual_seed(0)
    mu_in = torch.rand(B, M, device="cuda", generator=g)
    al_in = torch.rand(B, M, M, device="cuda", generator=g)
    be_in = beta0.clone()
    keep = [x.clone() for x in (mu_in, al_in, be_in)]
    res = plan.autotune(db, opts, mu_in, al_in, be_in, tune_iters=10)
    assert res["path"] == "decoupled" and res["threads_per_window"] in (64, 128, 256)
    assert res["ms"] > 0
    for a, b in zip((mu_in, al_in, be_in), keep):
        assert torch.equal(a, b)
    nt, _, cut = plan.shape()
    assert (nt, cut) == (res["threads_per_window"], res["cutoff"])

    l_t, mu_t, st_t = _fit(mdhp, plan, db, opts, beta0, M)
    assert np.all(st_t == 0)
    np.testing.assert_allclose(l_t, l_ref, rtol=1e-5)
    np.testing.assert_allclose(mu_t, mu_ref, rtol=1e-4, atol=1e-6)

    doc = json.load(open(cache))
    assert doc["format"] == "mdhp-autotune-1" and len(doc["entries"]) == 1
    e = doc["entries"][0]
    assert e["key"].endswith("|M16|mode0|W384|E%d|decoupled" % int(bt.counts.max()))
    assert e["threads_per_window"] == res["threads_per_window"]

    # a new plan with the same arguments and cache starts from the tuned shape;
    # a different window bound is another key and keeps the defaults
    again = mdhp.Plan(M, 0, B, int(bt.counts.max()), autotune_cache=cache)
    assert again.shape() == plan.shape()
    other = mdhp.Plan(M, 0, B, int(bt.counts.max()) + 1, autotune_cache=cache)
    assert other.shape() == ref_plan.shape()


def test_recursion_path_tuning_learned_beta(mdhp, wl, tmp_path):
    rng = np.random.default_rng(9)
    M, B = 8, 96
    betas = np.exp(rng.uniform(np.log(0.5), np.log(2.0), size=(B, M)))
    mu, alpha = wl.sample_params(rng, B, M, 1, betas, rng.uniform(0.2, 0.8, B))
    counts = wl.log_uniform_counts(rng, B, 200, 3000)
    bt = wl.simulate(M, 1, mu, alpha, betas, counts, seed=4, stream=4)
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    beta0 = torch.from_numpy(bt.beta).cuda()
    opts = mdhp.FitOptions(optimizer=1, max_iters=40, lr=1e-2, init=1, fit_beta=1)
    cache = str(tmp_path / "tune.json")
    ref_plan = mdhp.Plan(M, 1, B, int(counts.max()))
    l_ref, _, st_ref = _fit(mdhp, ref_plan, db, opts, beta0, M)
    plan = mdhp.Plan(M, 1, B, int(counts.max()), autotune_cache=cache)
    mu_in = torch.zeros(B, M, device="cuda")
    al_in = torch.zeros(B, M, M, device="cuda")
    be_in = beta0.clone()
    res = plan.autotune(db, opts, mu_in, al_in, be_in, tune_iters=8)
    assert res["path"] == "recursion" and res["threads_per_chunk"] >= 1
    assert torch.equal(be_in, beta0)
    l_t, _, st_t = _fit(mdhp, plan, db, opts, beta0, M)
    assert np.all(st_t == st_ref)
    np.testing.assert_allclose(l_t, l_ref, rtol=1e-5)
    again = mdhp.Plan(M, 1, B, int(counts.max()), autotune_cache=cache)
    again.set_path("recursion")
    plan.set_path("recursion")
    assert again.shape() == plan.shape()


def test_tolerance_fit_tuning_is_not_slower_than_defaults(mdhp):
    """For a fit to a tolerance the tuner runs the caller's fit itself (capped
    evaluations), so the shape it picks is no slower on that fit than the
    plan's default shape (10 % allowance for timing noise)."""
    from paper_2411_10258_gb300.workload import workload

    B, M = 16384, 32
    p = workload.make_params(5, B=B, seed=77)
    db, sst = mdhp.simulate(M, 0, p["mu"], p["alpha"], p["beta"], p["counts"], seed=77, stream_id=5)
    assert int((sst != 0).sum().item()) == 0
    beta0 = torch.from_numpy(p["beta"].astype(np.float32)).cuda()
    opts = mdhp.FitOptions(optimizer=1, lr=2e-2, max_iters=3000, tol=1e-5, init=1)

    def timed(plan):
        mu = torch.zeros(B, M, device="cuda")
        al = torch.zeros(B, M, M, device="cuda")
        plan.fit(db, opts, mu, al, beta0.clone())
        ms = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = plan.fit(db, opts, mu, al, beta0.clone())
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms)), out["loglik"].cpu().numpy()

    plan_d = mdhp.Plan(M, 0, B, int(p["counts"].max()))
    plan_t = mdhp.Plan(M, 0, B, int(p["counts"].max()))
    choice = plan_t.autotune(db, opts, torch.zeros(B, M, device="cuda"), torch.zeros(B, M, M, device="cuda"),
                             beta0.clone(), tune_iters=400)
    ms_d, ll_d = timed(plan_d)
    ms_t, ll_t = timed(plan_t)
    print("default", ms_d, "tuned", ms_t, choice)
    assert ms_t <= 1.10 * ms_d, (ms_t, ms_d, choice)
    assert np.all(np.isfinite(ll_t))
