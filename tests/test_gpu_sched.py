"""Scheduling variants of the decoupled fit give the oracle's answer: the
feature ring (bulk copies through shared memory) reproduces the register-
prefetch path bit for bit; the two-launch split over one two-ended queue,
single launches of 64/128/256 threads and the shared-memory feature class
agree with the FP64 oracle; every window is fitted exactly once whatever the
split (windows with a known answer per slot)."""
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


@pytest.fixture(scope="module")
def batch(wl):
    rng = np.random.default_rng(21)
    M, B = 16, 300
    betas = np.ones((B, 1))
    mu, alpha = wl.sample_params(rng, B, M, 0, betas, rng.uniform(0.2, 0.8, B))
    counts = wl.log_uniform_counts(rng, B, 20, 4000)
    counts[:3] = (1, 2, 3)  # ranges shorter than the block, single-event windows
    return wl.simulate(M, 0, mu, alpha, betas, counts, seed=8, stream=8)


def _fit(mdhp, bt, configure, opts):
    M, B = bt.M, bt.B
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    plan = mdhp.Plan(M, 0, B, int(bt.counts.max()))
    configure(plan)
    mu = torch.zeros(B, M, device="cuda")
    al = torch.zeros(B, M, M, device="cuda")
    be = torch.from_numpy(bt.beta).cuda()
    out = plan.fit(db, opts, mu, al, be)
    torch.cuda.synchronize()
    return (out["loglik"].cpu().numpy(), out["iters"].cpu().numpy(), out["status"].cpu().numpy(),
            mu.cpu().numpy(), al.cpu().numpy(), plan.last_launches())


OPTS = dict(optimizer=0, max_iters=40, lr=1e-2, init=1)


def test_ring_equals_register_prefetch(mdhp, batch):
    opts = mdhp.FitOptions(**OPTS)

    def base(p):
        p.set_split(False)
        p.set_shape(64, 4, 0)

    def ring(steps, stages):
        def f(p):
            base(p)
            p.set_pipeline(steps, stages)
        return f

    ref = _fit(mdhp, batch, base, opts)
    assert np.all(ref[2] == 0)
    for steps, stages in ((1, 2), (2, 3), (4, 2)):
        got = _fit(mdhp, batch, ring(steps, stages), opts)
        for a, b in zip(got[:5], ref[:5]):
            np.testing.assert_array_equal(a, b)


def test_launch_variants_match_oracle(mdhp, orc, batch):
    opts = mdhp.FitOptions(**OPTS)
    o = orc.fit_opts(optimizer=0, max_iters=OPTS["max_iters"], lr=OPTS["lr"])
    M = batch.M
    sample = sorted(set(list(range(0, batch.B, 15)) + [0, 1, 2]))
    ref = {}
    for b in sample:
        t, ids, T, _ = batch.window(b)
        m0, a0 = orc.cold_init(ids, float(T), M, batch.beta[b])
        ref[b] = orc.fit(t, ids, float(T), m0, a0, batch.beta[b].astype(np.float64), o)

    variants = {
        "split 256x1 + 64": lambda p: p.set_split(True, 256, 1),
        "split 128x2 + 64": lambda p: p.set_split(True, 128, 2),
        "single 64": lambda p: p.set_split(False),
        "single 128": lambda p: (p.set_split(False), p.set_shape(128, 4, 0)),
        "single 256": lambda p: (p.set_split(False), p.set_shape(256, 4, 0)),
        "shared-memory class": lambda p: (p.set_split(False), p.set_shape(64, 4, 1024)),
    }
    for name, conf in variants.items():
        ll, it, st, mu, al, launches = _fit(mdhp, batch, conf, opts)
        assert np.all(st == 0), name
        assert np.all(it == OPTS["max_iters"]), name
        assert launches >= 4, name
        for b in sample:
            r = ref[b]
            assert r["status"] == 0 and r["iters"] == OPTS["max_iters"]
            assert abs(ll[b] - r["lnL"]) <= 1e-5 * abs(r["lnL"]), (name, b)
            # fitted parameters within 1e-4 of the group's scale
            assert np.all(np.abs(mu[b] - r["mu"]) <= 1e-4 * np.abs(r["mu"]).max()), (name, b)
            assert np.all(np.abs(al[b] - r["alpha"]) <= 1e-4 * np.abs(r["alpha"]).max() + 1e-30), (name, b)
