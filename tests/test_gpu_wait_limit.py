"""Bounded waits of the bulk-copy rings, made to run out (mdhp_plan_set_wait_limit).

No GPU fault is involved: a consumer's wait is cut to one non-blocking test
of its mbarrier, which a copy issued a moment earlier has not yet completed.

* Feature ring (decoupled fit, mdhp_plan_set_pipeline): a window whose fill
  did not arrive reports MDHP_E_TIMEOUT with a NaN loglik and its parameters
  left as passed in; the fills in flight are waited out with the full bound
  before the CTA goes on, so every window gets a status, the windows that did
  not time out equal the default run bit for bit, and the same plan with the
  default bound then fits everything as before.
* Event ring (recursion fit, mdhp_plan_set_event_ring): a stage wait that
  gives up switches the CTA to global-memory reads, so the results equal the
  fit without the ring bit for bit (beta fixed, one launch shape).
"""
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


def _batch(wl, M, mode, B, seed):
    rng = np.random.default_rng(seed)
    betas = np.ones((B, 1)) if mode == 0 else rng.uniform(0.5, 2.0, (B, M))
    mu, alpha = wl.sample_params(rng, B, M, mode, betas, rng.uniform(0.2, 0.8, B))
    counts = wl.log_uniform_counts(rng, B, 200, 3000)
    return wl.simulate(M, mode, mu, alpha, betas, counts, seed=seed, stream=seed)


def _fit_x(mdhp, bt, polls):
    M, B = bt.M, bt.B
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    plan = mdhp.Plan(M, 0, B, int(bt.counts.max()))
    plan.set_split(False)
    plan.set_shape(64, 4, 0)  # every window streamed through the feature ring
    plan.set_pipeline(2, 2)
    plan.set_wait_limit(polls)
    opts = mdhp.FitOptions(optimizer=0, max_iters=30, lr=1e-2, init=1)
    mu = torch.zeros(B, M, device="cuda")
    al = torch.zeros(B, M, M, device="cuda")
    be = torch.from_numpy(bt.beta).cuda()
    out = plan.fit(db, opts, mu, al, be)
    torch.cuda.synchronize()
    res = (out["loglik"].cpu().numpy(), out["iters"].cpu().numpy(), out["status"].cpu().numpy(),
           mu.cpu().numpy(), al.cpu().numpy())
    return plan, db, res


def test_feature_ring_timeout_reports_and_recovers(mdhp, wl):
    from paper_2411_10258_gb300 import _lib

    bt = _batch(wl, 16, 0, 96, 31)
    _, _, ref = _fit_x(mdhp, bt, 0)
    assert np.all(ref[2] == _lib.OK)
    plan, db, got = _fit_x(mdhp, bt, 1)
    ll, it, st, mu, al = got
    assert set(np.unique(st)) <= {_lib.OK, _lib.E_TIMEOUT}, np.unique(st)
    to = st == _lib.E_TIMEOUT
    assert to.sum() >= 1, "no wait ran out with a one-poll bound"
    assert np.all(np.isnan(ll[to]))
    assert np.all(mu[to] == 0.0) and np.all(al[to] == 0.0)  # not written back
    ok = ~to
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a[ok], b[ok])
    # the same plan, default bound: the rings are in a consistent state again
    plan.set_wait_limit(0)
    B, M = bt.B, bt.M
    mu2 = torch.zeros(B, M, device="cuda")
    al2 = torch.zeros(B, M, M, device="cuda")
    out = plan.fit(db, mdhp.FitOptions(optimizer=0, max_iters=30, lr=1e-2, init=1), mu2, al2,
                   torch.from_numpy(bt.beta).cuda())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out["status"].cpu().numpy(), ref[2])
    np.testing.assert_array_equal(out["loglik"].cpu().numpy(), ref[0])
    np.testing.assert_array_equal(mu2.cpu().numpy(), ref[3])


def _fit_ring(mdhp, db, M, beta, ring, polls):
    B = db.B
    plan = mdhp.Plan(M, 1, B, 0)
    plan.set_path("recursion")
    plan.set_split(False)
    plan.set_event_ring(ring)
    plan.set_wait_limit(polls)
    mu = torch.zeros(B, M, device="cuda")
    al = torch.zeros(B, M, M, device="cuda")
    out = plan.fit(db, mdhp.FitOptions(optimizer=1, max_iters=10, lr=2e-3, fit_beta=0, init=1), mu, al,
                   beta.clone())
    torch.cuda.synchronize()
    return [out["loglik"].clone(), out["iters"].clone(), out["status"].clone(), mu, al]


def test_event_ring_timeout_falls_back_to_global_reads(mdhp, wl):
    from paper_2411_10258_gb300 import _lib

    M = 16
    bt = _batch(wl, M, 1, 24, 32)
    db = mdhp.DeviceBatch.from_host(bt, "cuda", max_events=0)  # streamed windows
    beta = torch.from_numpy(bt.beta).float().cuda().reshape(bt.B, M)
    off = _fit_ring(mdhp, db, M, beta, False, 0)
    assert bool(torch.all(off[2] == _lib.OK))
    for polls in (1, 0):
        on = _fit_ring(mdhp, db, M, beta, True, polls)
        for a, b in zip(on, off):
            assert torch.equal(a, b), polls
