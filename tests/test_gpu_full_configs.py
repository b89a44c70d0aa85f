"""Parity at the benchmark's full sizes, in the launch configurations it times.

* 64 x 4,194,304 fp32 poly3 sum/min/max (the headline step: one batch launch
  replayed from a CUDA graph, inputs drawn as the benchmark draws them): every
  partition against the oracle, on the first and on a later replay.
* 16 x 16,777,216 (key, value) pairs, keyed count+sum in one batch launch:
  every partition's table against the oracle.
* 16 x 4,194,304 pairs with Zipf(1.2) keys over 4096 ids, one batch launch:
  every partition's table against the oracle.
* 67,108,864 pairs over 2^20 keys (uniform and Zipf), the bucket-partitioned
  large-key reduce on device tables as the benchmark calls it: the whole table
  against the oracle.
* The 10,000-task uneven batch (log-normal sizes, kernel uniform over three),
  graph replay: every task against the oracle.
* The serving pool (240 partitions, log-normal sizes up to 2^26 elements)
  replayed open-loop at 50,000 tasks/s through both servers: every served
  result equals the same partition run alone (bitwise for uint32 / fp32, counts
  exact for keyed), and each pool partition's alone result matches the oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_common import check_f32_result, check_keyed
from paper_1505_01120_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1505_01120_gb300 import scl
    from paper_1505_01120_gb300.context import Context, current_stream
    torch.cuda.set_device(0)
    c = Context(12 << 30, device=0)
    yield c, scl, current_stream(0), torch
    c.close()


def as_result(scl, row):
    r = scl.scl_result()
    for k in ("u64_sum", "f64_sum", "f32_min", "f32_max", "status", "n"):
        setattr(r, k, row[k].item())
    return r


def test_headline_64x4194304_graph_replay(env):
    c, scl, st, torch = env
    parts_n, n = 64, 1 << 22
    host = synth.normal_f32(parts_n * n, np.random.default_rng(2)).reshape(parts_n, n)
    parts = [scl.scl_load_partition(c.handle, host[i], scl.SCL_F32, stream=st)
             for i in range(parts_n)]
    b = scl.scl_batch_create(c.handle, scl.make_tasks(
        [dict(part=p, kernel=scl.SCL_K_POLY3, reduce=scl.SCL_R_SUM_MIN_MAX) for p in parts]),
        parts_n)
    torch.cuda.synchronize()
    gs = torch.cuda.Stream().cuda_stream   # graphs are captured on a non-default stream
    scl.scl_batch_capture(b, gs)
    scl.scl_batch_launch(b, gs)
    first = scl.scl_batch_results(b, parts_n, stream=gs).copy()
    for _ in range(5):
        scl.scl_batch_launch(b, gs)
    later = scl.scl_batch_results(b, parts_n, stream=gs)
    scl.scl_batch_destroy(b)
    for p in parts:
        scl.scl_free_partition(c.handle, p)
    assert first.tobytes() == later.tobytes()
    for i in range(parts_n):
        check_f32_result(as_result(scl, first[i]), host[i], True)


def test_keyed_16x16777216_one_launch(env):
    c, scl, st, torch = env
    parts_n, m = 16, 1 << 24
    keys, vals = synth.keyed_partitions(parts_n, m, seed=3)
    outs = torch.zeros((parts_n, 4096 * 4), dtype=torch.int32, device="cuda")
    parts, tasks = [], []
    for i in range(parts_n):
        p = scl.scl_load_partition_kv(c.handle, keys[i], vals[i], stream=st)
        base = outs[i].data_ptr()
        parts.append(p)
        tasks.append(dict(part=p, kernel=scl.SCL_K_IDENT, reduce=scl.SCL_R_KEYED_COUNT_SUM,
                          num_keys=4096, counts_out=base, sums_out=base + 16384,
                          sums64_out=base + 32768))
    b = scl.scl_batch_create(c.handle, scl.make_tasks(tasks), parts_n)
    scl.scl_batch_launch(b, st)
    res = scl.scl_batch_results(b, parts_n, stream=st)
    scl.scl_batch_destroy(b)
    h = outs.cpu().numpy()
    for p in parts:
        scl.scl_free_partition(c.handle, p)
    for i in range(parts_n):
        assert int(res[i]["status"]) == 0 and int(res[i]["u64_sum"]) == m
        assert check_keyed(h[i, :4096].view(np.uint32), h[i, 4096:8192].view(np.float32),
                           h[i, 8192:].view(np.float64), keys[i], vals[i], 4096) == 0


def test_keyed_zipf_16x4194304_one_launch(env):
    c, scl, st, torch = env
    parts_n, m, nk = 16, 1 << 22, 4096
    rng = np.random.default_rng(12)
    keys = synth.zipf_keys_i32(parts_n * m, rng, nk).reshape(parts_n, m)
    vals = synth.unit_f32(parts_n * m, rng).reshape(parts_n, m)
    outs = torch.zeros((parts_n, nk * 4), dtype=torch.int32, device="cuda")
    parts, tasks = [], []
    for i in range(parts_n):
        p = scl.scl_load_partition_kv(c.handle, keys[i], vals[i], stream=st)
        base = outs[i].data_ptr()
        parts.append(p)
        tasks.append(dict(part=p, kernel=scl.SCL_K_IDENT, reduce=scl.SCL_R_KEYED_COUNT_SUM,
                          num_keys=nk, counts_out=base, sums_out=base + nk * 4,
                          sums64_out=base + nk * 8))
    b = scl.scl_batch_create(c.handle, scl.make_tasks(tasks), parts_n)
    scl.scl_batch_launch(b, st)
    res = scl.scl_batch_results(b, parts_n, stream=st)
    scl.scl_batch_destroy(b)
    h = outs.cpu().numpy()
    for p in parts:
        scl.scl_free_partition(c.handle, p)
    for i in range(parts_n):
        assert int(res[i]["status"]) == 0 and int(res[i]["u64_sum"]) == m
        assert check_keyed(h[i, :nk].view(np.uint32), h[i, nk:2 * nk].view(np.float32),
                           h[i, 2 * nk:].view(np.float64), keys[i], vals[i], nk) == 0


@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_keyed_large_1048576_keys_67108864(env, dist):
    c, scl, st, torch = env
    nk, n = 1 << 20, 1 << 26
    rng = np.random.default_rng(10)
    keys = synth.keys_i32(n, rng, nk) if dist == "uniform" else synth.zipf_keys_i32(n, rng, nk)
    vals = synth.unit_f32(n, rng)
    p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
    dc = torch.empty(nk, dtype=torch.int32, device="cuda")
    ds = torch.empty(nk, dtype=torch.float32, device="cuda")
    d64 = torch.empty(nk, dtype=torch.float64, device="cuda")
    dr = torch.empty(48, dtype=torch.uint8, device="cuda")
    for _ in range(2):   # the second call reuses the stream's bucket copy
        before = scl.scl_kernel_launches_total()
        scl.scl_keyed_reduce_large_async(c.handle, p, nk, dc, ds, d64, dr, stream=st)
        assert scl.scl_kernel_launches_total() - before == 6   # the partitioned path
        torch.cuda.synchronize()
        assert check_keyed(dc.cpu().numpy().view(np.uint32), ds.cpu().numpy(),
                           d64.cpu().numpy(), keys, vals, nk) == 0
        r = dr.cpu().numpy().view(scl.RESULT_DTYPE)[0]
        assert int(r["status"]) == 0 and int(r["u64_sum"]) == n
    scl.scl_free_partition(c.handle, p)


def test_batch_10000_graph_replay(env):
    c, scl, st, torch = env
    specs = synth.batch_tasks()
    d = synth.batch_data_packed(specs)
    du = torch.from_numpy(d["u32"].view(np.int32)).cuda()
    df = torch.from_numpy(d["f32"]).cuda()
    dk = torch.from_numpy(d["keys"]).cuda()
    dv = torch.from_numpy(d["vals"]).cuda()
    nkeyed = sum(s.kind == synth.KIND_KEYED for s in specs)
    kout = torch.zeros((nkeyed, 4096 * 2), dtype=torch.int32, device="cuda")
    tasks, parts, krow, nk = [], [], [], 0
    for s, off in zip(specs, d["offset"]):
        off = int(off)
        if s.kind == synth.KIND_MIX32:
            q = scl.scl_wrap_device(c.handle, du.data_ptr() + off * 4, None, scl.SCL_U32, s.n)
            tasks.append(dict(part=q, kernel=scl.SCL_K_MIX32, reduce=scl.SCL_R_SUM))
        elif s.kind == synth.KIND_POLY3:
            q = scl.scl_wrap_device(c.handle, df.data_ptr() + off * 4, None, scl.SCL_F32, s.n)
            tasks.append(dict(part=q, kernel=scl.SCL_K_POLY3, reduce=scl.SCL_R_SUM_MIN_MAX))
        else:
            q = scl.scl_wrap_device(c.handle, dk.data_ptr() + off * 4, dv.data_ptr() + off * 4,
                                    scl.SCL_KV_I32_F32, s.n)
            krow.append(nk)
            nk += 1
            base = kout[krow[-1]].data_ptr()
            tasks.append(dict(part=q, kernel=scl.SCL_K_IDENT, reduce=scl.SCL_R_KEYED_COUNT_SUM,
                              num_keys=4096, counts_out=base, sums_out=base + 16384))
            parts.append(q)
            continue
        krow.append(-1)
        parts.append(q)
    b = scl.scl_batch_create(c.handle, scl.make_tasks(tasks), len(tasks))
    torch.cuda.synchronize()
    gs = torch.cuda.Stream().cuda_stream
    scl.scl_batch_capture(b, gs)
    for _ in range(3):
        scl.scl_batch_launch(b, gs)
    res = scl.scl_batch_results(b, len(tasks), stream=gs)
    scl.scl_batch_destroy(b)
    h = kout.cpu().numpy()
    for q in parts:
        scl.scl_free_partition(c.handle, q)
    for i, (s, off) in enumerate(zip(specs, d["offset"])):
        off = int(off)
        assert int(res[i]["status"]) == 0 and int(res[i]["n"]) == s.n, i
        if s.kind == synth.KIND_MIX32:
            assert int(res[i]["u64_sum"]) == oracle.sum_u32(d["u32"][off:off + s.n], mix=True), i
        elif s.kind == synth.KIND_POLY3:
            check_f32_result(as_result(scl, res[i]), d["f32"][off:off + s.n], True)
        else:
            row = h[krow[i]]
            assert check_keyed(row[:4096].view(np.uint32), row[4096:].view(np.float32), None,
                               d["keys"][off:off + s.n], d["vals"][off:off + s.n], 4096) == 0, i


def test_serving_pool_both_servers(env):
    c, scl, st, torch = env
    rng = np.random.default_rng(5)
    pool = 240
    sizes = synth.lognormal_sizes(pool, 1 << 18, 1.5, 1024, 1 << 26, rng)
    kinds = np.arange(pool) % 3
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    bufs, tasks, outs = [], [], []
    for n, k in zip(sizes, kinds):
        n = int(n)
        if k == synth.KIND_MIX32:
            b = torch.randint(-2**31, 2**31 - 1, (n,), dtype=torch.int32, device="cuda",
                              generator=g)
            q = scl.scl_wrap_device(c.handle, b.data_ptr(), None, scl.SCL_U32, n)
            tasks.append(dict(part=q, kernel=scl.SCL_K_MIX32, reduce=scl.SCL_R_SUM))
            bufs.append((b,))
            outs.append(None)
        elif k == synth.KIND_POLY3:
            b = torch.randn(n, device="cuda", generator=g)
            q = scl.scl_wrap_device(c.handle, b.data_ptr(), None, scl.SCL_F32, n)
            tasks.append(dict(part=q, kernel=scl.SCL_K_POLY3, reduce=scl.SCL_R_SUM_MIN_MAX))
            bufs.append((b,))
            outs.append(None)
        else:
            kk = torch.randint(0, 4096, (n,), dtype=torch.int32, device="cuda", generator=g)
            vv = torch.rand(n, device="cuda", generator=g)
            q = scl.scl_wrap_device(c.handle, kk.data_ptr(), vv.data_ptr(),
                                    scl.SCL_KV_I32_F32, n)
            tasks.append(dict(part=q, kernel=scl.SCL_K_IDENT, reduce=scl.SCL_R_KEYED_COUNT_SUM,
                              num_keys=4096))
            bufs.append((kk, vv))
            outs.append(None)
    torch.cuda.synchronize()
    # each pool partition alone, checked against the oracle
    alone = []
    for i, t in enumerate(tasks):
        if kinds[i] == synth.KIND_KEYED:
            alone.append(None)
            continue
        r = scl.scl_map_reduce(c.handle, t["part"], t["kernel"], t["reduce"], stream=st)
        h = bufs[i][0].cpu().numpy()
        if kinds[i] == synth.KIND_MIX32:
            assert r.u64_sum == oracle.sum_u32(h.view(np.uint32), mix=True), i
        else:
            check_f32_result(r, h, True)
        alone.append(r)
    n_tasks = 10_000
    arrivals = synth.poisson_arrivals(50_000.0, n_tasks, np.random.default_rng(50_050))
    pick = np.random.default_rng(60_050).integers(0, pool, size=n_tasks)
    # keyed tasks of the trace write their tables to one scratch table per
    # pool partition (the last write wins; counts are checked once below)
    tabs = torch.zeros((pool, 4096 * 2), dtype=torch.int32, device="cuda")
    trace = []
    for i in pick:
        t = dict(tasks[i])
        if kinds[i] == synth.KIND_KEYED:
            t["counts_out"] = tabs[i].data_ptr()
            t["sums_out"] = tabs[i].data_ptr() + 16384
        trace.append(t)
    arr = scl.make_tasks(trace)
    for server in ("batched", "device_polled"):
        if server == "batched":
            scl.scl_server_start(c.handle, inflight_batches=4, max_batch_tasks=4096,
                                 hbm_budget_bytes=120 * 10**9)
            lat, res = scl.scl_server_replay(c.handle, arr, arrivals, n_tasks)
            scl.scl_server_stop(c.handle)
        else:
            scl.scl_devserver_start(c.handle)
            lat, res = scl.scl_devserver_replay(c.handle, arr, arrivals, n_tasks)
            scl.scl_devserver_stop(c.handle)
        assert np.all(res["status"] == 0) and np.all(lat > 0), server
        for j, i in enumerate(pick):
            assert int(res[j]["n"]) == int(sizes[i])
            if kinds[i] == synth.KIND_KEYED:
                assert int(res[j]["u64_sum"]) == int(sizes[i])
                continue
            a = alone[i]
            assert int(res[j]["u64_sum"]) == a.u64_sum and float(res[j]["f64_sum"]) == a.f64_sum
            assert float(res[j]["f32_min"]) == a.f32_min and float(res[j]["f32_max"]) == a.f32_max
        # keyed tables of the pool partitions the trace used
        h = tabs.cpu().numpy()
        for i in sorted(set(int(x) for x in pick if kinds[x] == synth.KIND_KEYED))[:20]:
            kk, vv = (x.cpu().numpy() for x in bufs[i])
            ocnt, _, _ = oracle.keyed_count_sum(kk, vv, 4096)
            assert np.array_equal(h[i, :4096].view(np.uint32), ocnt), (server, i)
        tabs.zero_()
    for t in tasks:
        scl.scl_free_partition(c.handle, t["part"])
