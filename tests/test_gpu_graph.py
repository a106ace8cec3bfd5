"""mdhp_fit_batch inside a captured CUDA graph: no host synchronisation and no
allocation in the call, so a fixed-shape batched fit can be replayed; the
replays give the eager results."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fit_captured_in_cuda_graph(wl):
    import paper_2411_10258_gb300 as mdhp

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    bt = wl.make_workload(2, B=64, seed=77)
    M, B = bt.M, bt.B
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    beta0 = torch.from_numpy(bt.beta).cuda()
    opts = mdhp.FitOptions(max_iters=25, init=1)
    plan = mdhp.Plan(M, 0, B, int(bt.counts.max()))
    mu = torch.zeros(B, M, device="cuda")
    alpha = torch.zeros(B, M, M, device="cuda")
    beta = beta0.clone()
    out = {k: torch.empty(B, dtype=d, device="cuda") for k, d in
           (("loglik", torch.float64), ("iters", torch.int32), ("status", torch.int32))}
    plan.fit(db, opts, mu, alpha, beta, out=out)  # eager run (also sets kernel attributes)
    torch.cuda.synchronize()
    eager = out["loglik"].clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.fit(db, opts, mu, alpha, beta, out=out, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        out["loglik"].zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out["loglik"], eager)
        assert bool(torch.all(out["status"] == 0))


def test_warm_pipeline_captured_in_cuda_graph(wl):
    """The learned initializer's prediction and the fit from it (one
    mdhp_fit_batch call with init = 2) captured in one CUDA graph: the replays
    give the eager results.  With the two-launch split, which of the two
    launches fits a given window (and so the block size that sets its
    summation order) depends on timing, so lnL and the parameters are compared
    to rounding, at a fixed iteration count."""
    import paper_2411_10258_gb300 as mdhp

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    bt = wl.make_workload(2, B=96, seed=78)
    M, B = bt.M, bt.B
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    beta0 = torch.from_numpy(bt.beta).cuda()
    model = mdhp.InitModel(M, hidden=64, max_batch=40, seed=3)  # several prediction chunks
    plan = mdhp.Plan(M, 0, B, int(bt.counts.max()))
    model.attach(plan)
    opts = mdhp.FitOptions(optimizer=1, lr=1e-2, max_iters=60, init=2)
    mu = torch.zeros(B, M, device="cuda")
    alpha = torch.zeros(B, M, M, device="cuda")
    beta = beta0.clone()
    out = {k: torch.empty(B, dtype=d, device="cuda") for k, d in
           (("loglik", torch.float64), ("iters", torch.int32), ("status", torch.int32))}
    plan.fit(db, opts, mu, alpha, beta, out=out)
    torch.cuda.synchronize()
    eager = {k: v.clone() for k, v in out.items()}
    eager_mu = mu.clone()
    assert plan.last_launches() >= 3 + 6 * 3 + 1  # sort, 3 prediction chunks, the fit
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.fit(db, opts, mu, alpha, beta, out=out, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        out["loglik"].zero_()
        mu.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out["status"], eager["status"])
        assert torch.equal(out["iters"], eager["iters"])
        assert bool(torch.all(torch.abs(out["loglik"] - eager["loglik"]) <= 1e-6 * torch.abs(eager["loglik"])))
        scale = torch.abs(eager_mu).amax(dim=1, keepdim=True)
        assert bool(torch.all(torch.abs(mu - eager_mu) <= 1e-4 * scale))
    assert bool(torch.all(out["status"] == 0))
