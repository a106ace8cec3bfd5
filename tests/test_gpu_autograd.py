"""loglik_grad as a torch.autograd.Function (LoglikGrad), checked against
central finite differences of the FP64 oracle (h = 1e-4 relative) on 8 long
windows shaped like the 512 x M=64 workload (per-source beta, learned), for
sampled mu, alpha, beta and event-weight coordinates."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_loglikgrad_vs_fp64_finite_differences(orc, wl):
    import paper_2411_10258_gb300 as mdhp

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    rng = np.random.default_rng(123)
    M, B = 64, 8
    betas = np.exp(rng.uniform(np.log(0.5), np.log(2.0), (B, M)))
    mu_t, a_t = wl.sample_params(rng, B, M, 1, betas, rng.uniform(0.2, 0.8, B))
    counts = rng.integers(20000, 30000, B)
    bt = wl.simulate(M, 1, mu_t, a_t, betas, counts, 2024, 3)
    bt.weights = rng.uniform(0.8, 1.2, bt.n_events).astype(np.float32)
    db = mdhp.DeviceBatch.from_host(bt, "cuda", max_events=0)  # streamed events
    mu = torch.tensor((mu_t * rng.uniform(0.8, 1.2, mu_t.shape)).astype(np.float32), device="cuda",
                      requires_grad=True)
    alpha = torch.tensor((a_t * rng.uniform(0.8, 1.2, a_t.shape)).astype(np.float32), device="cuda",
                         requires_grad=True)
    beta = torch.tensor(bt.beta.copy(), device="cuda", requires_grad=True)
    w = torch.tensor(bt.weights, device="cuda", requires_grad=True)
    ll, bad = mdhp.LoglikGrad.apply(db, mu, alpha, beta, w)
    assert not bool(bad.any())
    ll.sum().backward()
    g = {"mu": mu.grad.cpu().numpy(), "alpha": alpha.grad.cpu().numpy(),
         "beta": beta.grad.cpu().numpy(), "w": w.grad.cpu().numpy()}
    m64 = mu.detach().cpu().numpy().astype(np.float64)
    a64 = alpha.detach().cpu().numpy().astype(np.float64)
    b64 = bt.beta.astype(np.float64)
    for b in range(B):
        t, ids, T, wb = bt.window(b)
        s0 = int(bt.offsets[b])
        t64, i32, w64 = t.astype(np.float64), ids.astype(np.int32), wb.astype(np.float64)

        def L(mu_, al_, be_, ww_):
            return orc.loglik_grad(t64, i32, float(T), mu_, al_, be_, w=ww_, mode=1)["lnL"]

        ref = orc.loglik_grad(t64, i32, float(T), m64[b], a64[b], b64[b], w=w64, mode=1)
        assert abs(ll[b].item() - ref["lnL"]) <= 1e-5 * abs(ref["lnL"])
        picks = [("mu", rng.integers(M)), ("alpha", (rng.integers(M), rng.integers(M))),
                 ("alpha", (rng.integers(M), rng.integers(M))), ("beta", rng.integers(M)),
                 ("w", rng.integers(len(t)))]
        for kind, idx in picks:
            args = [m64[b].copy(), a64[b].copy(), b64[b].copy(), w64.copy()]
            k = {"mu": 0, "alpha": 1, "beta": 2, "w": 3}[kind]
            x0 = args[k][idx]
            h = 1e-4 * max(abs(x0), 1e-3)
            args[k][idx] = x0 + h
            lp = L(*args)
            args[k][idx] = x0 - h
            lm = L(*args)
            fd = (lp - lm) / (2 * h)
            got = g[kind][s0 + idx] if kind == "w" else g[kind][b][idx]
            # scale: the magnitude of the analytic gradient group (cancellation near optimum)
            grp = {"mu": ref["g_mu"], "alpha": ref["g_alpha"], "beta": ref["g_beta"], "w": ref["g_w"]}[kind]
            scale = max(abs(fd), 1e-2 * np.max(np.abs(grp)))
            assert abs(got - fd) <= 2e-3 * scale, (b, kind, idx, got, fd)
