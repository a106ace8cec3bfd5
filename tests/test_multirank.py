"""The multi-GPU host logic on CPU ranks (gloo, world size 2): the event-
balanced partition of windows, the max-over-ranks time, and the gather of
per-window results back to the original order.  No GPU: the per-rank fit is
replaced by a known function of the window index."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, counts, q):
    import torch.distributed as dist

    from paper_2411_10258_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = shard.partition(counts, world)
        mine = parts[rank]
        # stand-in for the fit: two values per window
        local = torch.stack([torch.as_tensor(mine, dtype=torch.float64) * 2.0,
                             torch.as_tensor(counts[mine], dtype=torch.float64)], dim=1)
        full = shard.gather_windows(local, mine, len(counts))
        tmax = shard.max_over_ranks(10.0 + rank)
        g = torch.arange(5, dtype=torch.float32) * (rank + 1)  # rank r holds (r + 1) * [0..4]
        shard.allreduce_mean_(g)
        q.put((rank, [p.tolist() for p in parts], full.numpy().tolist(), tmax, g.tolist()))
    finally:
        dist.destroy_process_group()


def test_partition_balance():
    from paper_2411_10258_gb300 import shard

    rng = np.random.default_rng(0)
    counts = np.round(np.exp(rng.uniform(np.log(200), np.log(5000), 4096))).astype(np.int64)
    for world in (1, 2, 3, 8):
        parts = shard.partition(counts, world)
        allidx = np.sort(np.concatenate(parts))
        np.testing.assert_array_equal(allidx, np.arange(len(counts)))
        loads = np.array([counts[p].sum() for p in parts])
        assert loads.max() - loads.min() <= counts.max()
    # degenerate: fewer windows than ranks
    parts = shard.partition([5, 7], 4)
    assert sorted(len(p) for p in parts) == [0, 0, 1, 1]


def test_two_gloo_ranks():
    import torch.multiprocessing as mp

    rng = np.random.default_rng(1)
    counts = rng.integers(1, 1000, size=37)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, counts, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    expect = np.stack([np.arange(37) * 2.0, counts.astype(np.float64)], axis=1)
    for rank, parts, full, tmax, g in res:
        assert parts == res[0][1]
        np.testing.assert_array_equal(np.asarray(full), expect)
        assert tmax == 11.0
        np.testing.assert_allclose(g, np.arange(5) * 1.5)  # mean of 1x and 2x
