"""The device-polling server (k_doorbell resident kernel).

* Every job's result equals the task run alone by scl_map_reduce, bitwise for
  uint32 and fp32 tasks (the same segment code and geometry), and matches the
  oracle; keyed jobs (one piece and many) give exact counts and sums within
  1e-5 of the oracle; a bad key gives SCL_E_KEY_RANGE.
* The open-loop replay and concurrent submitters finish every job.
* The host ends the kernel after its idle period and launches it again with
  the next job.
* The bounded device wait: with the host's idle stop switched off, a kernel
  left without work gives up after its wait limit, reports it in host memory,
  and the server recovers and keeps serving.
"""
from __future__ import annotations

import threading
import time

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
    rng = np.random.default_rng(900)
    sizes = np.concatenate([[0, 1, 255, 4096, 65537, 1 << 20, (1 << 22) + 3],
                            synth.lognormal_sizes(60, 1 << 14, 1.5, 1024, 1 << 22, rng)])
    kinds = np.concatenate([[0, 1, 2, 2, 2, 2, 1], rng.integers(0, 3, size=60)])
    specs = [synth.TaskSpec(int(k), int(n), 9000 + i)
             for i, (n, k) in enumerate(zip(sizes, kinds))]
    data, tasks, outs = [], [], []
    for i, s in enumerate(specs):
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
    alone = [None if t["reduce"] == scl.SCL_R_KEYED_COUNT_SUM else
             scl.scl_map_reduce(c.handle, t["part"], t["kernel"], t["reduce"], stream=st)
             for t in tasks]
    yield c, scl, st, torch, specs, data, tasks, outs, arr, alone
    scl.scl_devserver_stop(c.handle)
    c.close()


def check_job(scl, specs, data, outs, alone, i, r):
    s = specs[i]
    assert r.status == 0 and r.n == s.n, (i, r.status, r.n, s.n)
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


def clear_outputs(outs):
    for o in outs:
        if o is not None:
            o.zero_()


def test_jobs_match_alone_and_oracle(env):
    c, scl, st, torch, specs, data, tasks, outs, arr, alone = env
    clear_outputs(outs)
    torch.cuda.synchronize()
    scl.scl_devserver_start(c.handle)
    try:
        tickets = [scl.scl_devserver_submit(c.handle, arr, i) for i in range(len(tasks))]
        res = [scl.scl_devserver_wait(c.handle, t, 30_000) for t in tickets]
        stats = scl.scl_devserver_get_stats(c.handle)
    finally:
        scl.scl_devserver_stop(c.handle)
    for i, r in enumerate(res):
        check_job(scl, specs, data, outs, alone, i, r)
    assert stats["completed"] == len(tasks) and stats["failed"] == 0
    assert stats["device_errors"] == 0 and stats["kernel_launches"] >= 1
    assert stats["grid"] > 0 and stats["block"] in (256, 512)


def test_unaligned_partition_and_bad_key(env):
    c, scl, st, torch, *_ = env
    rng = np.random.default_rng(901)
    x = rng.standard_normal(100_003, dtype=np.float32)
    buf = torch.from_numpy(np.concatenate([[0.0], x]).astype(np.float32)).cuda()
    p = scl.scl_wrap_device(c.handle, buf.data_ptr() + 4, None, scl.SCL_F32, x.size)
    alone = scl.scl_map_reduce(c.handle, p, scl.SCL_K_POLY3, scl.SCL_R_SUM_MIN_MAX, stream=st)
    keys = rng.integers(0, 4096, size=300_000, dtype=np.int32)
    keys[12345] = 5000
    vals = rng.random(300_000, dtype=np.float32)
    pk = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
    o = torch.zeros(4096 * 3, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    arr = scl.make_tasks([
        dict(part=p, kernel=scl.SCL_K_POLY3, reduce=scl.SCL_R_SUM_MIN_MAX),
        dict(part=pk, kernel=scl.SCL_K_IDENT, reduce=scl.SCL_R_KEYED_COUNT_SUM, num_keys=4096,
             counts_out=o.data_ptr(), sums_out=o.data_ptr() + 16384),
        dict(part=pk, kernel=scl.SCL_K_MIX32, reduce=scl.SCL_R_KEYED_COUNT_SUM, num_keys=1000,
             counts_out=o.data_ptr() + 32768, sums_out=o.data_ptr() + 36768)])
    scl.scl_devserver_start(c.handle)
    try:
        r0 = scl.scl_devserver_wait(c.handle, scl.scl_devserver_submit(c.handle, arr, 0))
        r1 = scl.scl_devserver_wait(c.handle, scl.scl_devserver_submit(c.handle, arr, 1))
        r2 = scl.scl_devserver_wait(c.handle, scl.scl_devserver_submit(c.handle, arr, 2))
        with pytest.raises(scl.SclError):
            scl.scl_devserver_start(c.handle)   # already running
    finally:
        scl.scl_devserver_stop(c.handle)
    assert r0.u64_sum == alone.u64_sum and r0.f64_sum == alone.f64_sum
    assert r0.f32_min == alone.f32_min and r0.f32_max == alone.f32_max
    check_f32_result(r0, x, True)
    h = o.cpu().numpy()
    assert r1.status == scl.SCL_E_KEY_RANGE
    good = keys != 5000
    assert np.array_equal(h[:4096].view(np.uint32),
                          np.bincount(keys[good], minlength=4096).astype(np.uint32))
    assert r1.u64_sum == good.sum()
    # hashed buckets: every key is valid, the oracle defines the bucket
    ocnt, osum = oracle.keyed_hashed_count_sum(keys, vals, 1000)
    assert r2.status == 0
    assert np.array_equal(h[8192:9192].view(np.uint32), ocnt)
    s = h[9192:10192].view(np.float32).astype(np.float64)
    assert np.all(np.abs(s - osum) <= 1e-5 * np.abs(osum))
    scl.scl_free_partition(c.handle, p)
    scl.scl_free_partition(c.handle, pk)


def test_replay_open_loop_and_concurrent_submitters(env):
    c, scl, st, torch, specs, data, tasks, outs, arr, alone = env
    clear_outputs(outs)
    torch.cuda.synchronize()
    scl.scl_devserver_start(c.handle)
    try:
        t = synth.poisson_arrivals(20_000.0, len(tasks), np.random.default_rng(902))
        lat, res = scl.scl_devserver_replay(c.handle, arr, t, len(tasks))
        assert np.all(lat > 0)
        for i in range(len(tasks)):
            r = scl.scl_result.from_buffer_copy(res[i].tobytes())
            check_job(scl, specs, data, outs, alone, i, r)
        # four threads submitting the streaming tasks at once
        idx = [i for i, s in enumerate(specs) if s.kind != synth.KIND_KEYED]
        got = {}

        def worker(k):
            for i in idx[k::4]:
                tk = scl.scl_devserver_submit(c.handle, arr, i)
                got[i] = scl.scl_devserver_wait(c.handle, tk)

        th = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        assert sorted(got) == idx
        for i in idx:
            check_job(scl, specs, data, outs, alone, i, got[i])
    finally:
        scl.scl_devserver_stop(c.handle)


def test_idle_stop_and_relaunch(env):
    c, scl, st, torch, specs, data, tasks, outs, arr, alone = env
    i = next(k for k, s in enumerate(specs) if s.kind == synth.KIND_POLY3 and s.n > 1000)
    scl.scl_devserver_start(c.handle, idle_stop_ns=1_000_000)
    try:
        r = scl.scl_devserver_wait(c.handle, scl.scl_devserver_submit(c.handle, arr, i))
        check_job(scl, specs, data, outs, alone, i, r)
        time.sleep(0.1)
        s0 = scl.scl_devserver_get_stats(c.handle)
        assert s0["idle_stops"] >= 1
        r = scl.scl_devserver_wait(c.handle, scl.scl_devserver_submit(c.handle, arr, i))
        check_job(scl, specs, data, outs, alone, i, r)
        s1 = scl.scl_devserver_get_stats(c.handle)
        assert s1["kernel_launches"] == s0["kernel_launches"] + 1
        assert s1["device_errors"] == 0
    finally:
        scl.scl_devserver_stop(c.handle)
    # the SMs are free again: an ordinary launch runs
    r = scl.scl_map_reduce(c.handle, tasks[i]["part"], tasks[i]["kernel"], tasks[i]["reduce"],
                           stream=st)
    assert r.f64_sum == alone[i].f64_sum


def test_device_wait_limit_is_reported_and_recovered(env):
    c, scl, st, torch, specs, data, tasks, outs, arr, alone = env
    i = next(k for k, s in enumerate(specs) if s.kind == synth.KIND_MIX32 and s.n > 1000)
    scl.scl_devserver_start(c.handle, idle_stop_ns=scl.IDLE_STOP_NEVER, wait_limit_ns=50_000_000)
    try:
        r = scl.scl_devserver_wait(c.handle, scl.scl_devserver_submit(c.handle, arr, i))
        check_job(scl, specs, data, outs, alone, i, r)
        # no work: every CTA's wait for the doorbell runs out after 50 ms
        deadline = time.time() + 5.0
        while scl.scl_devserver_get_stats(c.handle)["device_errors"] == 0:
            assert time.time() < deadline, "the device wait limit was not reported"
            time.sleep(0.02)
        s0 = scl.scl_devserver_get_stats(c.handle)
        assert s0["failed"] == 0 and s0["idle_stops"] == 0
        # the context stays usable: the next job relaunches the kernel
        r = scl.scl_devserver_wait(c.handle, scl.scl_devserver_submit(c.handle, arr, i))
        check_job(scl, specs, data, outs, alone, i, r)
        assert scl.scl_devserver_get_stats(c.handle)["kernel_launches"] == \
            s0["kernel_launches"] + 1
    finally:
        scl.scl_devserver_stop(c.handle)


def test_submit_errors(env):
    c, scl, st, torch, specs, data, tasks, outs, arr, alone = env
    bad = scl.make_tasks([dict(part=987654321, kernel=scl.SCL_K_MIX32, reduce=scl.SCL_R_SUM)])
    with pytest.raises(scl.SclError):
        scl.scl_devserver_submit(c.handle, bad, 0)   # not running
    scl.scl_devserver_start(c.handle)
    try:
        with pytest.raises(scl.SclError):
            scl.scl_devserver_submit(c.handle, bad, 0)   # unknown partition
        with pytest.raises(scl.SclError):
            scl.scl_devserver_wait(c.handle, 10**9)      # unknown ticket
    finally:
        scl.scl_devserver_stop(c.handle)
    scl.scl_devserver_stop(c.handle)   # no-op when not running


def test_small_rings_wrap_around(env):
    """Rings far smaller than the work: 8 job slots, 64 work units (and partial
    slots), 2 keyed accumulators.  Jobs wait for ring space, slots and unit-map
    entries are reused many times over, and every result must still match."""
    c, scl, st, torch, specs, data, tasks, outs, arr, alone = env
    clear_outputs(outs)
    torch.cuda.synchronize()
    # jobs that fit the 64-unit ring: streaming tasks up to 64 segments, keyed
    # tasks up to 64 pieces (the 4 Mi-element ones have 256 segments)
    fit = [i for i, s in enumerate(specs)
           if (s.kind == synth.KIND_KEYED and s.n <= 64 * 65536)
           or (s.kind != synth.KIND_KEYED and s.n <= 64 * 32768 and s.n <= 1 << 21)]
    assert len(fit) > 30
    scl.scl_devserver_start(c.handle, job_ring=8, unit_ring=64, keyed_slots=2)
    try:
        for rep in range(3):
            tickets = [(i, scl.scl_devserver_submit(c.handle, arr, i)) for i in fit]
            for i, t in tickets:
                check_job(scl, specs, data, outs, alone, i, scl.scl_devserver_wait(c.handle, t))
        s = scl.scl_devserver_get_stats(c.handle)
        assert s["ring_waits"] > 0 and s["max_inflight"] <= 8
        assert s["completed"] == 3 * len(fit) and s["failed"] == 0 and s["device_errors"] == 0
        # a job with more units than the ring holds is refused at once
        big = next(i for i, sp in enumerate(specs) if sp.kind == synth.KIND_POLY3 and sp.n > 1 << 21)
        with pytest.raises(scl.SclError):
            scl.scl_devserver_submit(c.handle, arr, big)
    finally:
        scl.scl_devserver_stop(c.handle)
