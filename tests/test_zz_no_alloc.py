"""mdhp_fit_batch_noalloc: the batched fit for callers that may not allocate
device memory (pooled framework allocators, no-allocation-after-start-up
deployments).  Called through the C ABI and checked against the plan-based
mdhp_fit_batch on the same inputs, twice in a row, since every call shares the
library's fixed scratch array.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LL_RTOL = 1e-5
P_RTOL = 1e-4


def _p(x):
    return ctypes.c_void_p(x.data_ptr())


def test_noalloc_matches_plan_fit_twice(wl):
    import paper_2411_10258_gb300 as mdhp
    from paper_2411_10258_gb300 import _lib

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lib = _lib.load()
    bt = wl.make_workload(2, B=48, seed=909)
    M, B = bt.M, bt.B
    db = mdhp.DeviceBatch.from_host(bt, "cuda")
    beta = torch.from_numpy(bt.beta).cuda()
    opts = mdhp.FitOptions(optimizer=1, max_iters=40, lr=5e-3, init=1)

    plan = mdhp.Plan(M, 0, B, int(bt.counts.max()))
    ref_mu = torch.zeros(B, M, device="cuda")
    ref_alpha = torch.zeros(B, M, M, device="cuda")
    ref = plan.fit(db, opts, ref_mu, ref_alpha, beta.clone())
    torch.cuda.synchronize()

    runs = []
    for _ in range(2):
        mu = torch.zeros(B, M, device="cuda")
        alpha = torch.zeros(B, M, M, device="cuda")
        b = beta.clone()
        ll = torch.empty(B, dtype=torch.float64, device="cuda")
        it = torch.empty(B, dtype=torch.int32, device="cuda")
        st = torch.empty(B, dtype=torch.int32, device="cuda")
        cb = db.c_struct()
        co = opts.c_struct()
        rc = lib.mdhp_fit_batch_noalloc(ctypes.byref(cb), ctypes.byref(co), _p(mu), _p(alpha), _p(b),
                                        _p(ll), _p(it), _p(st),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        _lib.check(rc, "mdhp_fit_batch_noalloc")
        torch.cuda.synchronize()
        runs.append((mu.cpu().numpy(), alpha.cpu().numpy(), ll.cpu().numpy(), it.cpu().numpy(),
                     st.cpu().numpy()))

    r_mu, r_alpha = ref["mu"].cpu().numpy(), ref["alpha"].cpu().numpy()
    r_ll, r_it, r_st = ref["loglik"].cpu().numpy(), ref["iters"].cpu().numpy(), ref["status"].cpu().numpy()
    for mu, alpha, ll, it, st in runs:
        np.testing.assert_array_equal(st, r_st)
        np.testing.assert_array_equal(it, r_it)
        assert np.all(np.abs(ll - r_ll) <= LL_RTOL * np.abs(r_ll))
        for w in range(B):
            assert np.all(np.abs(mu[w] - r_mu[w]) <= P_RTOL * np.abs(r_mu[w]).max())
            assert np.all(np.abs(alpha[w] - r_alpha[w]) <= P_RTOL * np.abs(r_alpha[w]).max() + 1e-30)
    # the two calls in a row agree with each other exactly (same kernel, same inputs)
    np.testing.assert_array_equal(runs[0][2], runs[1][2])


def test_noalloc_rejects_oversized_batch():
    from paper_2411_10258_gb300 import _lib

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    lib = _lib.load()
    B = _lib.NOALLOC_MAX_WINDOWS + 1
    cb = _lib.MdhpBatch(B, 16, 0, None, None, None, None, None, 0, 0)
    co = _lib.MdhpFitOpts(0, 10, 0, 3, 1e-2, 1e-10, 0.0, 1e-6, 0.9, 0.999, 1e-8, 1, 0.0)
    dummy = ctypes.c_void_p(1)
    rc = lib.mdhp_fit_batch_noalloc(ctypes.byref(cb), ctypes.byref(co), dummy, dummy, dummy,
                                    dummy, dummy, dummy, None)
    assert rc == _lib.E_ARG
    assert b"exceeds" in lib.mdhp_last_error()
