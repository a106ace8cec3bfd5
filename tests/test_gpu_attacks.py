"""Time-exciting injection attacks are visible in the fitted MDHP
parameters: windows that receive a power-law (PLA) or stealth (ASA)
injection stream on one message ID get a larger fitted self-excitation
alpha_kk of that ID than untouched windows (AUC well above chance), with the
whole batch fitted by the library on the GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _auc(pos, neg):
    pos, neg = np.asarray(pos), np.asarray(neg)
    return float(np.mean(pos[:, None] > neg[None, :]) + 0.5 * np.mean(pos[:, None] == neg[None, :]))


@pytest.mark.parametrize("sampler,strategy", [("NPP", "PLA"), ("ND", "ASA")])
def test_injection_raises_self_excitation(wl, sampler, strategy):
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
    score = np.array([a[b, ks[b], ks[b]] for b in range(B)])
    assert _auc(score[:n], score[n:]) > 0.9
