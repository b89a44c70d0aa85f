"""Multi-rank plumbing: shard partitions across ranks, combine their results.

SparkCL schedules one task per RDD partition across workers (Sec. 3.1.5) and
combines partition results with ReduceCL's tree reduce (Sec. 3.1.3, 3.2.2).
Here each rank (one process per GPU) owns a shard of the partitions and runs
its own launches; the only exchange is the fold of small per-partition
results, done on the host: an all-gather of the 48-byte results (and keyed
tables) over torch.distributed, then the library's host combine
(scl_combine / scl_combine_keyed).  No collective touches the data path.
"""
from __future__ import annotations

import numpy as np


def shard(sizes, rank: int, world: int) -> list[int]:
    """Indices of the partitions rank `rank` owns: greedy largest-first
    assignment to the rank with the fewest bytes so far (ties by rank), so
    every partition lands on exactly one rank and bytes stay balanced."""
    sizes = np.asarray(sizes, dtype=np.int64)
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(sizes.size, dtype=np.int64)
    for i in np.argsort(-sizes, kind="stable"):
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += sizes[i]
    return [int(i) for i in np.flatnonzero(owner == rank)]


def gather_results(results: np.ndarray, group=None) -> list[np.ndarray]:
    """All-gather each rank's scl_result array (RESULT_DTYPE, any length)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    raw = np.ascontiguousarray(results).view(np.uint8)
    n = torch.tensor([raw.size], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    cap = int(max(int(s.item()) for s in sizes))
    buf = torch.zeros(max(cap, 1), dtype=torch.uint8)
    buf[:raw.size] = torch.from_numpy(raw.copy())
    bufs = [torch.zeros(max(cap, 1), dtype=torch.uint8) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    from . import scl
    return [b[:int(s.item())].numpy().view(scl.RESULT_DTYPE) for b, s in zip(bufs, sizes)]


def combine_across_ranks(results: np.ndarray, group=None):
    """ReduceCL over every rank's partition results: all-gather, then the
    library's host tree combine.  Returns an scl_result on every rank."""
    from . import scl
    parts = np.concatenate(gather_results(results, group))
    objs = []
    for r in parts:
        o = scl.scl_result()
        for k in ("u64_sum", "f64_sum", "f32_sum", "f32_min", "f32_max", "status", "n", "kind"):
            setattr(o, k, r[k].item())
        objs.append(o)
    return scl.scl_combine(objs)


def combine_keyed_across_ranks(counts: np.ndarray, sums64: np.ndarray, group=None):
    """ReduceCL over the keyed tables of every rank: each rank's tables
    [k_local, num_keys] (count uint32, sum fp64) are all-gathered as bytes,
    then folded by the library's host merge, scl_combine_keyed, in rank order
    (counts exact, sums in fp64).  Returns (counts, sums64) on every rank."""
    import torch
    import torch.distributed as dist
    from . import scl
    counts = np.ascontiguousarray(np.atleast_2d(counts), np.uint32)
    sums64 = np.ascontiguousarray(np.atleast_2d(sums64), np.float64)
    k, nk = counts.shape
    if sums64.shape != (k, nk):
        raise ValueError("counts and sums64 must have the same shape")
    world = dist.get_world_size(group)
    rows = torch.tensor([k, nk], dtype=torch.int64)
    got = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(got, rows, group=group)
    if any(int(g[1]) != nk for g in got):
        raise ValueError("ranks disagree on num_keys")
    kmax = max(int(g[0]) for g in got)
    pack = np.zeros((max(kmax, 1), nk * 12), np.uint8)   # per row: counts, then sums
    pack[:k, :nk * 4] = counts.view(np.uint8).reshape(k, nk * 4)
    pack[:k, nk * 4:] = sums64.view(np.uint8).reshape(k, nk * 8)
    bufs = [torch.zeros(pack.shape, dtype=torch.uint8) for _ in range(world)]
    dist.all_gather(bufs, torch.from_numpy(pack), group=group)
    cs, ss = [], []
    for b, g in zip(bufs, got):
        rows_r = b.numpy()[:int(g[0])]
        cs.append(np.ascontiguousarray(rows_r[:, :nk * 4]).view(np.uint32).reshape(-1, nk))
        ss.append(np.ascontiguousarray(rows_r[:, nk * 4:]).view(np.float64).reshape(-1, nk))
    allc, alls = np.concatenate(cs), np.concatenate(ss)
    if allc.shape[0] == 0:
        return np.zeros(nk, np.uint32), np.zeros(nk, np.float64)
    return scl.scl_combine_keyed(allc, alls)
