"""Streamed events through the bulk-copy ring (mdhp_plan_set_event_ring).

The recursion fit with the ring gives the results of the same fit reading its
events from global memory: bit for bit with beta fixed (the same arithmetic
on the same values, one launch shape), and to rounding with beta learned
(the per-chunk d/dbeta sums meet in shared-memory atomics, whose order varies
from run to run).  Covered: windows whose copies are clamped at the end of
the batch arrays, a tie group across a stage boundary, a batch whose arrays
are not 16-byte aligned (the ring then switches itself off), and agreement of
both with the FP64 oracle (lnL 1e-5 relative, parameters 1e-4)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ITERS = 12
LR = 2e-3


def _fit(mdhp, db, M, beta0, ring, fit_beta):
    B = db.B
    plan = mdhp.Plan(M, 1, B, 0)  # no stated bound: every window is streamed
    plan.set_path("recursion")
    plan.set_split(False)  # one launch shape: which windows share a launch is fixed
    plan.set_event_ring(ring)
    mu = torch.zeros(B, M, device="cuda")
    al = torch.zeros(B, M, M, device="cuda")
    be = beta0.clone()
    out = plan.fit(db, mdhp.FitOptions(optimizer=1, max_iters=ITERS, lr=LR, fit_beta=fit_beta, init=1),
                   mu, al, be)
    torch.cuda.synchronize()
    return out["loglik"].clone(), mu, al, be, out["status"].clone()


def _same(x, y, exact):
    if exact:
        for a, b in zip(x, y):
            assert torch.equal(a, b)
        return
    ll_x, mu_x, al_x, be_x, st_x = x
    ll_y, mu_y, al_y, be_y, st_y = y
    assert torch.equal(st_x, st_y)
    assert bool(torch.all(torch.abs(ll_x - ll_y) <= 2e-6 * torch.abs(ll_y)))
    for a, b in ((mu_x, mu_y), (al_x, al_y), (be_x, be_y)):
        scale = torch.abs(b).reshape(b.shape[0], -1).amax(dim=1).reshape(-1, *([1] * (b.dim() - 1)))
        assert bool(torch.all(torch.abs(a - b) <= 2e-4 * scale))


@pytest.mark.parametrize("fit_beta", [0, 1])
@pytest.mark.parametrize("M", [16, 32])
def test_ring_matches_global_reads(wl, orc, M, fit_beta):
    import paper_2411_10258_gb300 as mdhp

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    rng = np.random.default_rng(60 + M)
    counts = np.array([5003, 130, 1, 2047, 777, 3])  # batch length not a multiple of 4 or 8
    B = len(counts)
    betas = rng.uniform(0.5, 2.0, (B, M))
    mu_t, a_t = wl.sample_params(rng, B, M, 1, betas, rng.uniform(0.2, 0.8, B))
    bt = wl.simulate(M, 1, mu_t, a_t, betas, counts, 23, 95)
    t = bt.t.copy()
    s = int(bt.offsets[0])
    t[s + 120:s + 140] = t[s + 120]  # a tie group across the first 128-event stage boundary (stays sorted)
    bt.t = t
    beta0 = torch.tensor(betas if fit_beta == 0 else np.ones((B, M)), dtype=torch.float32, device="cuda")
    db = mdhp.DeviceBatch.from_host(bt, "cuda", max_events=0)
    exact = fit_beta == 0
    on = _fit(mdhp, db, M, beta0, True, fit_beta)
    off = _fit(mdhp, db, M, beta0, False, fit_beta)
    _same(on, off, exact)
    # unaligned arrays: views starting one event in (the ring switches itself off)
    t1 = torch.cat([torch.zeros(1, device="cuda"), db.t])[1:]
    u1 = torch.cat([torch.zeros(1, dtype=torch.int16, device="cuda"), db.id])[1:]
    assert t1.data_ptr() % 16 != 0
    db1 = mdhp.DeviceBatch(M, 1, db.offsets, t1, u1, db.T, None, 0)
    un = _fit(mdhp, db1, M, beta0, True, fit_beta)
    _same(un, off, exact)
    # the oracle, same iterations
    o = orc.fit_opts(optimizer=1, max_iters=ITERS, lr=LR, fit_beta=fit_beta)
    ll, mu, al = on[0].cpu().numpy(), on[1].cpu().numpy(), on[2].cpu().numpy()
    for b in range(B):
        tb, ib, T, _ = bt.window(b)
        b0 = beta0[b].double().cpu().numpy()
        m0, a0 = orc.cold_init(ib, float(T), M, b0, mode=1)
        r = orc.fit(tb, ib, float(T), m0, a0, b0, o, mode=1)
        assert abs(ll[b] - r["lnL"]) <= 1e-5 * abs(r["lnL"]), (b, ll[b], r["lnL"])
        assert np.all(np.abs(mu[b] - r["mu"]) <= 1e-4 * np.abs(r["mu"]).max()), b
        assert np.all(np.abs(al[b] - r["alpha"]) <= 1e-4 * np.abs(r["alpha"]).max() + 1e-30), b
