"""Data-parallel training of the learned initializer: two processes on the
GPU, each with half of a batch, exchange gradients through a gloo all-reduce
(mdhp_init_backward / mdhp_init_set_grads / mdhp_init_apply).  The averaged
gradient equals the gradient of the whole batch computed in one process, and
both processes hold identical parameters after the AdamW step."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M, H, B = 8, 64, 64


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _data():
    rng = np.random.default_rng(12)
    K0 = (M + 32 * M * M + 3 + 63) // 64 * 64
    X = rng.uniform(0, 1, (B, K0)).astype(np.float32)
    mu_cold = rng.uniform(0.05, 1, (B, M)).astype(np.float32)
    beta = np.full(B, 1.0, np.float32)
    mu_t = (mu_cold * rng.uniform(0.5, 2, (B, M))).astype(np.float32)
    a_t = (rng.uniform(0, 0.3, (B, M, M)) / M).astype(np.float32)
    return X, mu_cold, beta, mu_t, a_t


def _rank(rank, port, q):
    import torch.distributed as dist

    import paper_2411_10258_gb300 as mdhp

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        X, mu_cold, beta, mu_t, a_t = _data()
        sl = slice(rank * B // 2, (rank + 1) * B // 2)
        dev = torch.device("cuda", 0)
        cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        model = mdhp.InitModel(M, hidden=H, max_batch=B, seed=5)
        feat = cu(X[sl]).to(torch.bfloat16)
        model.backward(feat, cu(mu_cold[sl]), cu(beta[sl]), cu(mu_t[sl]), cu(a_t[sl]))
        g = model.get("grads")
        from paper_2411_10258_gb300 import shard

        shard.allreduce_mean_(g)
        model.set_grads(g)
        model.apply(1e-3, 0.01)
        torch.cuda.synchronize()
        q.put((rank, g.cpu().numpy(), model.get("params").cpu().numpy()))
    finally:
        dist.destroy_process_group()


def test_two_process_data_parallel_step():
    import torch.multiprocessing as mp

    import paper_2411_10258_gb300 as mdhp

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    # the whole batch in one process: gradient of the mean loss over B windows
    X, mu_cold, beta, mu_t, a_t = _data()
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ref = mdhp.InitModel(M, hidden=H, max_batch=B, seed=5)
    ref.backward(cu(X).to(torch.bfloat16), cu(mu_cold), cu(beta), cu(mu_t), cu(a_t))
    g_ref = ref.get("grads").cpu().numpy()
    torch.cuda.synchronize()

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(2)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (_, g0, p0), (_, g1, p1) = res
    np.testing.assert_array_equal(g0, g1)
    np.testing.assert_array_equal(p0, p1)
    # mean of the two half-batch gradients = the whole-batch gradient
    scale = np.abs(g_ref).max()
    assert np.max(np.abs(g0 - g_ref)) <= 1e-4 * scale
