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
    """Merge keyed tables [k_local, num_keys] of every rank into one table:
    the library's host merge of the local tables, then one sum across ranks
    (counts exact in int64, sums in fp64)."""
    import torch
    import torch.distributed as dist
    from . import scl
    lc, ls = scl.scl_combine_keyed(np.ascontiguousarray(counts, np.uint32),
                                   np.ascontiguousarray(sums64, np.float64))
    tc = torch.from_numpy(lc.astype(np.int64))
    ts = torch.from_numpy(ls.copy())
    dist.all_reduce(tc, group=group)
    dist.all_reduce(ts, group=group)
    return tc.numpy().astype(np.uint32), ts.numpy()
