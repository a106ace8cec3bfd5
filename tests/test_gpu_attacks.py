"""Time-exciting injection attacks are visible in the fitted MDHP
parameters: windows that receive a power-law (PLA) or stealth (ASA)
injection stream on one message ID get a larger fitted self-excitation
alpha_kk of that ID than untouched windows (AUC well above chance), with the
whole batch fitted by the library on the GPU.  A sample of attacked and
normal windows is re-fitted by the FP64 oracle with the same options and
compared (lnL 1e-5 relative, parameters 1e-4 of the group's scale)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _auc(pos, neg):
    pos, neg = np.asarray(pos), np.asarray(neg)
    return float(np.mean(pos[:, None] > neg[None, :]) + 0.5 * np.mean(pos[:, None] == neg[None, :]))


@pytest.mark.parametrize("sampler,strategy", [("NPP", "PLA"), ("ND", "ASA")])
def test_injection_raises_self_excitation(wl, orc, sampler, strategy):
    import paper_2411_10258_gb300 as mdhp
    from paper_2411_10258_gb300.workload import attacks

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    rng = np.random.default_rng(11)
    M, n = 8, 32
    B = 2 * n
    betas = np.ones((B, 1))
    mu, alpha = wl.sample_params(rng, B, M, 0, betas, rng.uniform(0.2, 0.8, B))
    bg = wl.simulate(M, 0, mu, alpha, betas, wl.log_uniform_counts(rng, B, 1000, 2000), 5, 6)
    ts, ids, Ts, ks = [], [], [], []
    for b in range(B):
        t, u, T, _ = bg.window(b)
        k = int(rng.integers(M))
        if b < n:
            t, u = attacks.inject(t, u, float(T), attacks.sample(sampler, strategy, rng), k)
        ts.append(np.asarray(t, np.float32)); ids.append(np.asarray(u, np.int16))
        Ts.append(max(float(T), float(ts[-1][-1]))); ks.append(k)
    off = np.zeros(B + 1, np.int64)
    np.cumsum([len(x) for x in ts], out=off[1:])
    up = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    db = mdhp.DeviceBatch(M, 0, up(off), up(np.concatenate(ts)), up(np.concatenate(ids)),
                          up(np.asarray(Ts, np.float32)), None, int(np.diff(off).max()))
    plan = mdhp.Plan(M, 0, B, int(np.diff(off).max()))
    mu_d = torch.zeros(B, M, device="cuda")
    al_d = torch.zeros(B, M, M, device="cuda")
    out = plan.fit(db, mdhp.FitOptions(optimizer=1, max_iters=1500, lr=1e-2, init=1), mu_d, al_d,
                   torch.ones(B, 1, device="cuda"))
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    a = al_d.cpu().numpy()
    # the oracle re-fits three attacked and three normal windows after the same
    # 200 iterations of a separate GPU fit (over the long 1,500-iteration run,
    # Adam's steps near the optimum amplify rounding differences between any
    # two summation orders; parity is checked along a well-conditioned stretch)
    mu_p = torch.zeros(B, M, device="cuda")
    al_p = torch.zeros(B, M, M, device="cuda")
    outp = plan.fit(db, mdhp.FitOptions(optimizer=1, max_iters=200, lr=1e-2, init=1), mu_p, al_p,
                    torch.ones(B, 1, device="cuda"))
    torch.cuda.synchronize()
    sample = [0, n // 2, n - 1, n, n + n // 2, B - 1]
    o = orc.fit_opts(optimizer=1, max_iters=200, lr=1e-2)
    sub = np.zeros(len(sample) + 1, np.int64)
    np.cumsum([len(ts[b]) for b in sample], out=sub[1:])
    mu0 = np.zeros((len(sample), M)); a0 = np.zeros((len(sample), M, M))
    for q, b in enumerate(sample):
        mu0[q], a0[q] = orc.cold_init(ids[b].astype(np.int32), float(np.float32(Ts[b])), M, [1.0])
    r = orc.fit_batch(sub, np.concatenate([ts[b] for b in sample]), np.concatenate([ids[b] for b in sample]),
                      np.asarray([Ts[b] for b in sample], np.float32), M, 0, mu0, a0,
                      np.ones((len(sample), 1)), o)
    ll, m_h, a_h = outp["loglik"].cpu().numpy(), mu_p.cpu().numpy(), al_p.cpu().numpy()
    for q, b in enumerate(sample):
        assert r["status"][q] == 0 and outp["iters"][b].item() == r["iters"][q] == 200
        assert abs(ll[b] - r["lnL"][q]) <= 1e-5 * abs(r["lnL"][q]), (b, ll[b], r["lnL"][q])
        rm, ra = r["mu"][q], r["alpha"][q]
        assert np.all(np.abs(m_h[b] - rm) <= 1e-4 * np.maximum(np.abs(rm), 1e-3 * np.abs(rm).max())), b
        assert np.all(np.abs(a_h[b] - ra) <= 1e-4 * np.abs(ra).max()), b
    score = np.array([a[b, ks[b], ks[b]] for b in range(B)])
    assert _auc(score[:n], score[n:]) > 0.9
