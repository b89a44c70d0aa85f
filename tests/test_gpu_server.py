"""The continuous-batching server.

Each task's result must be the same served in a mix as run alone: bitwise for
uint32 and fp32 tasks (same segment geometry and fold order), counts bitwise
and sums within 1e-5 for keyed tasks; and every result must match the oracle.
Admission must respect the HBM budget; tasks that bring new data must have
their transient partitions freed; the open-loop replay must finish every task.
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
    c = Context(4 << 30, device=0)
    st = current_stream(0)
    rng = np.random.default_rng(700)
    sizes = np.concatenate([[0, 1, 255, 4096], synth.lognormal_sizes(60, 1 << 14, 1.5, 1024,
                                                                      1 << 22, rng)])
    specs = [synth.TaskSpec(int(k), int(n), 7000 + i)
             for i, (n, k) in enumerate(zip(sizes, rng.integers(0, 3, size=sizes.size)))]
    data, tasks, outs = [], [], []
    for s in specs:
        d = synth.task_data(s)
        data.append(d)
        if s.kind == synth.KIND_MIX32:
            p = scl.scl_load_partition(c.handle, d[0], scl.SCL_U32, stream=st)
            tasks.append(dict(part=p, kernel=scl.SCL_K_MIX32, reduce=scl.SCL_R_SUM))
            outs.append(None)
        elif s.kind == synth.KIND_POLY3:
            p = scl.scl_load_partition(c.handle, d[0], scl.SCL_F32, stream=st)
            tasks.append(dict(part=p, kernel=scl.SCL_K_POLY3, reduce=scl.SCL_R_SUM_MIN_MAX))
            outs.append(None)
        else:
            p = scl.scl_load_partition_kv(c.handle, d[0], d[1], stream=st)
            o = torch.zeros(4096 * 4, dtype=torch.int32, device="cuda")
            outs.append(o)
            tasks.append(dict(part=p, kernel=scl.SCL_K_IDENT, reduce=scl.SCL_R_KEYED_COUNT_SUM,
                              num_keys=4096, counts_out=o.data_ptr(),
                              sums_out=o.data_ptr() + 16384, sums64_out=o.data_ptr() + 32768))
    torch.cuda.synchronize()
    arr = scl.make_tasks(tasks)
    # results of each task alone
    alone = []
    for i, t in enumerate(tasks):
        if t["reduce"] == scl.SCL_R_KEYED_COUNT_SUM:
            alone.append(None)
        else:
            alone.append(scl.scl_map_reduce(c.handle, t["part"], t["kernel"], t["reduce"],
                                            stream=st))
    yield c, scl, st, torch, specs, data, tasks, outs, arr, alone
    c.close()


def check_served(scl, specs, data, outs, alone, i, r):
    s = specs[i]
    assert r.status == 0 and r.n == s.n, (i, r.status)
    if s.kind == synth.KIND_KEYED:
        o = outs[i].cpu().numpy()
        assert check_keyed(o[:4096].view(np.uint32), o[4096:8192].view(np.float32),
                           o[8192:].view(np.float64), data[i][0], data[i][1], 4096) == 0
        assert r.u64_sum == s.n
        return
    a = alone[i]
    assert r.u64_sum == a.u64_sum and r.f64_sum == a.f64_sum, i
    assert r.f32_min == a.f32_min and r.f32_max == a.f32_max, i
    if s.kind == synth.KIND_MIX32:
        assert r.u64_sum == oracle.sum_u32(data[i][0], mix=True)
    else:
        check_f32_result(r, data[i][0], True)


@pytest.mark.parametrize("inflight,batch", [(4, 4096), (2, 8), (1, 1)])
def test_served_equals_alone(env, inflight, batch):
    c, scl, st, torch, specs, data, tasks, outs, arr, alone = env
    scl.scl_server_start(c.handle, inflight_batches=inflight, max_batch_tasks=batch)
    try:
        tickets = [scl.scl_server_submit(c.handle, arr, i) for i in range(len(tasks))]
        for i, tk in enumerate(tickets):
            check_served(scl, specs, data, outs, alone, i, scl.scl_server_wait(c.handle, tk))
        stats = scl.scl_server_get_stats(c.handle)
        assert stats["completed"] == len(tasks) and stats["max_batch"] <= batch
        if batch == 1:
            assert stats["batches"] == len(tasks)
    finally:
        scl.scl_server_stop(c.handle)


def test_budget_admission(env):
    c, scl, st, torch, specs, data, tasks, outs, arr, alone = env
    resident = scl.scl_arena_stats(c.handle)
    scl.scl_server_start(c.handle, inflight_batches=4)
    base = scl.scl_server_get_stats(c.handle)["resident_bytes"]
    scl.scl_server_stop(c.handle)
    # room for one 4 MiB input at a time on top of what is resident
    budget = base + (6 << 20)
    rng = np.random.default_rng(703)
    hosts = [rng.standard_normal(1 << 20, dtype=np.float32) for _ in range(4)]
    tf = scl.make_tasks([dict(part=0, kernel=scl.SCL_K_POLY3, reduce=scl.SCL_R_SUM_MIN_MAX)])
    scl.scl_server_start(c.handle, inflight_batches=4, hbm_budget_bytes=budget)
    try:
        lt = [scl.scl_server_submit_load(c.handle, h, None, scl.SCL_F32, h.size, tf)
              for h in hosts]
        tickets = [scl.scl_server_submit(c.handle, arr, i) for i in range(len(tasks))]
        for h, t in zip(hosts, lt):
            check_f32_result(scl.scl_server_wait(c.handle, t), h, True)
        for i, tk in enumerate(tickets):
            check_served(scl, specs, data, outs, alone, i, scl.scl_server_wait(c.handle, tk))
        stats = scl.scl_server_get_stats(c.handle)
        assert stats["peak_bytes_in_use"] <= budget
        assert stats["admission_waits"] >= 3
        # a task that can never fit is refused at submit
        big = np.zeros(2 << 20, np.float32)
        with pytest.raises(scl.SclError) as e:
            scl.scl_server_submit_load(c.handle, big, None, scl.SCL_F32, big.size, tf)
        assert e.value.status == scl.SCL_E_BUDGET
    finally:
        scl.scl_server_stop(c.handle)
    assert scl.scl_arena_stats(c.handle) == resident


def test_tasks_with_new_data(env):
    c, scl, st, torch, *_ = env
    rng = np.random.default_rng(701)
    free0 = scl.scl_arena_stats(c.handle)[0]
    hosts = [rng.standard_normal(int(n), dtype=np.float32) for n in (5, 70_000, 1 << 20)]
    hu = [rng.integers(0, 1 << 32, size=int(n), dtype=np.uint32) for n in (3, 4096 * 5 + 1)]
    kk = rng.integers(0, 4096, size=300_001, dtype=np.int32)
    kv = rng.random(300_001, dtype=np.float32)
    ko = torch.zeros(4096 * 4, dtype=torch.int32, device="cuda")
    tf = scl.make_tasks([dict(part=0, kernel=scl.SCL_K_POLY3, reduce=scl.SCL_R_SUM_MIN_MAX)])
    tu = scl.make_tasks([dict(part=0, kernel=scl.SCL_K_MIX32, reduce=scl.SCL_R_SUM)])
    tk = scl.make_tasks([dict(part=0, kernel=scl.SCL_K_IDENT, reduce=scl.SCL_R_KEYED_COUNT_SUM,
                              num_keys=4096, counts_out=ko.data_ptr(),
                              sums_out=ko.data_ptr() + 16384, sums64_out=ko.data_ptr() + 32768)])
    scl.scl_server_start(c.handle)
    try:
        tf_t = [scl.scl_server_submit_load(c.handle, h, None, scl.SCL_F32, h.size, tf)
                for h in hosts]
        tu_t = [scl.scl_server_submit_load(c.handle, h, None, scl.SCL_U32, h.size, tu)
                for h in hu]
        tk_t = scl.scl_server_submit_load(c.handle, kk, kv, scl.SCL_KV_I32_F32, kk.size, tk)
        for h, t in zip(hosts, tf_t):
            check_f32_result(scl.scl_server_wait(c.handle, t), h, True)
        for h, t in zip(hu, tu_t):
            assert scl.scl_server_wait(c.handle, t).u64_sum == oracle.sum_u32(h)
        scl.scl_server_wait(c.handle, tk_t)
        o = ko.cpu().numpy()
        assert check_keyed(o[:4096].view(np.uint32), o[4096:8192].view(np.float32),
                           o[8192:].view(np.float64), kk, kv, 4096) == 0
    finally:
        scl.scl_server_stop(c.handle)
    assert scl.scl_arena_stats(c.handle)[0] == free0


def test_open_loop_replay(env):
    c, scl, st, torch, specs, data, tasks, outs, arr, alone = env
    rng = np.random.default_rng(702)
    n = 3000
    pick = rng.integers(0, len(tasks), size=n)
    rep = scl.make_tasks([tasks[i] for i in pick])
    arrivals = synth.poisson_arrivals(20_000.0, n, rng)
    scl.scl_server_start(c.handle, inflight_batches=4)
    try:
        lat, res = scl.scl_server_replay(c.handle, rep, arrivals, n)
        stats = scl.scl_server_get_stats(c.handle)
    finally:
        scl.scl_server_stop(c.handle)
    assert np.all(lat > 0)
    assert stats["completed"] == n and stats["batches"] < n
    for j in range(0, n, 97):
        i = int(pick[j])
        if specs[i].kind != synth.KIND_KEYED:
            assert int(res[j]["u64_sum"]) == alone[i].u64_sum
            assert float(res[j]["f64_sum"]) == alone[i].f64_sum


def test_poll_and_errors(env):
    c, scl, st, torch, specs, data, tasks, outs, arr, alone = env
    with pytest.raises(scl.SclError) as e:
        scl.scl_server_submit(c.handle, arr, 0)
    assert e.value.status == scl.SCL_E_STATE
    scl.scl_server_start(c.handle)
    try:
        with pytest.raises(scl.SclError):
            scl.scl_server_start(c.handle)
        tk = scl.scl_server_submit(c.handle, arr, 5)
        r = None
        for _ in range(200_000):
            r = scl.scl_server_poll(c.handle, tk)
            if r is not None:
                break
        assert r is not None and r.status == 0
        with pytest.raises(scl.SclError) as e:
            scl.scl_server_poll(c.handle, 10 ** 9)
        assert e.value.status == scl.SCL_E_INVALID
    finally:
        scl.scl_server_stop(c.handle)
