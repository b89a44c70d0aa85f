"""World-size-2 gloo tests (CPU) of the multi-rank path: every partition is
owned by exactly one rank, and ReduceCL's combine across ranks equals the
oracle over all partitions.  A rank that leaves before the merge makes the
other rank's merge fail with an error instead of hanging."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import oracle
from paper_1505_01120_gb300 import dist as sdist
from paper_1505_01120_gb300 import synth


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _partitions():
    rng = np.random.default_rng(800)
    sizes = synth.lognormal_sizes(37, 4096, 1.2, 1, 200_000, rng)
    return sizes, [synth.normal_f32(int(n), np.random.default_rng(900 + i))
                   for i, n in enumerate(sizes)]


def _rank_results(rank, world):
    from paper_1505_01120_gb300 import scl
    sizes, parts = _partitions()
    mine = sdist.shard(sizes, rank, world)
    res = np.zeros(len(mine), dtype=scl.RESULT_DTYPE)
    for j, i in enumerate(mine):
        s, mn, mx = oracle.reduce_f32(parts[i], poly=True)
        res[j]["f64_sum"], res[j]["f32_min"], res[j]["f32_max"] = s, mn, mx
        res[j]["u64_sum"] = oracle.sum_u32(parts[i].view(np.uint32))
        res[j]["n"] = parts[i].size
    return mine, res


def _worker(rank, world, port, q, mode):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    try:
        if mode == "leave" and rank == 1:
            q.put((rank, "left"))
            q.close()
            q.join_thread()      # flush the message before leaving
            os._exit(0)          # leaves between steps, nothing in flight
        mine, res = _rank_results(rank, world)
        r = sdist.combine_across_ranks(res)
        keys = (np.arange(5000) % 64).astype(np.int32) + rank
        vals = np.full(5000, 0.5 + rank, np.float32)
        # rank 0 holds two partition tables, rank 1 one: uneven row counts
        cuts = [0, 2000, 5000] if rank == 0 else [0, 5000]
        tabs = [oracle.keyed_count_sum(keys[a:b], vals[a:b], 128) for a, b in zip(cuts, cuts[1:])]
        kc, ks = sdist.combine_keyed_across_ranks(np.stack([t[0] for t in tabs]),
                                                  np.stack([t[1] for t in tabs]))
        q.put((rank, (mine, r.u64_sum, r.f64_sum, r.f32_min, r.f32_max, r.n, kc, ks)))
    except Exception as e:   # the surviving rank reports the failed merge
        q.put((rank, "error: %s" % type(e).__name__))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(mode, world=2):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, mode)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
    return out


def test_shard_covers_every_partition_once():
    sizes, _ = _partitions()
    for world in (1, 2, 3, 8):
        owned = sorted(i for r in range(world) for i in sdist.shard(sizes, r, world))
        assert owned == list(range(len(sizes)))
        loads = [int(sizes[sdist.shard(sizes, r, world)].sum()) for r in range(world)]
        assert max(loads) - min(loads) <= int(sizes.max())


def test_combine_across_two_gloo_ranks():
    out = _run("normal")
    sizes, parts = _partitions()
    allx = np.concatenate(parts)
    s, mn, mx = oracle.reduce_f32(allx, poly=True)
    u = oracle.sum_u32(allx.view(np.uint32))
    for rank in (0, 1):
        mine, us, fs, fmn, fmx, n, kc, ks = out[rank]
        assert us == u and n == allx.size
        assert abs(fs - s) <= 1e-12 * float(np.abs(oracle.map_poly3(allx)).sum())
        assert fmn == mn and fmx == mx
        # keyed tables merged across ranks: keys r + (i mod 64), values 0.5 + r
        want_c = np.zeros(128, np.uint32)
        want_s = np.zeros(128)
        for r in (0, 1):
            want_c[r:r + 64] += (5000 // 64 + (np.arange(64) < 5000 % 64)).astype(np.uint32)
            want_s[r:r + 64] += (5000 // 64 + (np.arange(64) < 5000 % 64)) * (0.5 + r)
        assert np.array_equal(kc, want_c) and np.allclose(ks, want_s, rtol=1e-12)
    assert sorted(out[0][0] + out[1][0]) == list(range(len(sizes)))


def test_rank_leaving_before_merge_is_detected():
    out = _run("leave")
    assert out[1] == "left"
    assert isinstance(out[0], str) and out[0].startswith("error")
