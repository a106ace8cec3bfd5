"""Windows over several GPUs: one process per GPU, no collective on the data
path.

Each window is an independent fit (Sec. IV-B), so a batch shards by windows.
The ranks' work is balanced by event count (the fit's cost is about
iterations x events), not by window count: windows are taken longest first
and each goes to the rank with the fewest events so far (the longest-
processing-time rule), which keeps every rank within one window's events of
the mean.  Collectives appear only around the data path: the max-over-ranks
time of a timed region, the gather of per-window results to every rank, and
the gradient mean of data-parallel training of the learned initializer.
"""
from __future__ import annotations

import heapq

import numpy as np
import torch


def partition(counts, world: int) -> list[np.ndarray]:
    """Window indices of each rank, ascending, with nearly equal event totals."""
    counts = np.asarray(counts, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.argsort(-counts, kind="stable")
    heap = [(0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for b in order:
        load, r = heapq.heappop(heap)
        parts[r].append(int(b))
        heapq.heappush(heap, (load + int(counts[b]), r))
    return [np.sort(np.asarray(p, dtype=np.int64)) for p in parts]


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over the ranks of the default process group (the
    whole-job time of a region every rank timed); the value itself when no
    group is initialised."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_mean_(t: torch.Tensor, group=None) -> torch.Tensor:
    """In-place mean of `t` over the ranks of the process group (the gradient
    exchange of data-parallel initializer training).  A gloo group reduces a
    host copy of a device tensor.  No-op without an initialised group."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return t
    world = dist.get_world_size(group)
    if world == 1:
        return t
    if t.is_cuda and dist.get_backend(group) == "gloo":
        h = t.detach().cpu()
        dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
        t.copy_(h.to(t.device) / world)
    else:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        t /= world
    return t


def gather_windows(local: torch.Tensor, idx_local, B: int) -> torch.Tensor:
    """Per-window rows computed by each rank for its windows `idx_local` ->
    the [B, ...] tensor in the original window order, on every rank."""
    import torch.distributed as dist

    idx_local = torch.as_tensor(np.asarray(idx_local, dtype=np.int64), device=local.device)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        out = torch.empty((B,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
        out[idx_local] = local
        return out
    world = dist.get_world_size()
    n = torch.tensor([local.shape[0]], dtype=torch.int64, device=local.device)
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n)
    cap = int(max(int(x.item()) for x in ns))
    pad = torch.zeros((cap,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    ipad = torch.full((cap,), -1, dtype=torch.int64, device=local.device)
    ipad[: local.shape[0]] = idx_local
    rows = [torch.empty_like(pad) for _ in range(world)]
    idxs = [torch.empty_like(ipad) for _ in range(world)]
    dist.all_gather(rows, pad)
    dist.all_gather(idxs, ipad)
    out = torch.empty((B,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    for r, (x, i) in enumerate(zip(rows, idxs)):
        k = int(ns[r].item())
        out[i[:k]] = x[:k]
    return out
