"""Batched launch: many uneven partitions in one persistent launch.

Each task's result in a batch must match the oracle, and must equal the same
task run alone: bitwise for integer sums, fp32/fp64 sums and min/max (fp32
tasks see the same segment geometry and the same fixed-order fold in both),
counts bitwise and sums within tolerance for keyed tasks.  Graph replays must
give the same results launch after launch.  Batches that mix families run
both ways: split into concurrent per-family launches (the default) and as one
mixed-kernel launch; the two agree bitwise on the streaming tasks.
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
    c = Context(6 << 30, device=0)
    yield c, scl, current_stream(0), torch
    c.close()


def make_batch(c, scl, st, torch, specs, seed=0):
    """Load each spec's data, build task dicts with device output tables."""
    parts, data, outs, tasks = [], [], [], []
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
            o = (torch.zeros(4096, dtype=torch.int32, device="cuda"),
                 torch.zeros(4096, dtype=torch.float32, device="cuda"),
                 torch.zeros(4096, dtype=torch.float64, device="cuda"))
            outs.append(o)
            tasks.append(dict(part=p, kernel=scl.SCL_K_IDENT, reduce=scl.SCL_R_KEYED_COUNT_SUM,
                              num_keys=4096, counts_out=o[0], sums_out=o[1], sums64_out=o[2]))
        parts.append(p)
    return parts, data, outs, tasks


def check_batch(scl, specs, data, outs, res):
    for i, s in enumerate(specs):
        r = res[i]
        if s.kind == synth.KIND_MIX32:
            assert int(r["u64_sum"]) == oracle.sum_u32(data[i][0], mix=True), i
        elif s.kind == synth.KIND_POLY3:
            rr = scl.scl_result()
            for k in ("u64_sum", "f64_sum", "f32_min", "f32_max", "status", "n"):
                setattr(rr, k, r[k].item())
            check_f32_result(rr, data[i][0], True)
        else:
            cnt = outs[i][0].cpu().numpy().view(np.uint32)
            sums = outs[i][1].cpu().numpy()
            s64 = outs[i][2].cpu().numpy()
            assert check_keyed(cnt, sums, s64, data[i][0], data[i][1], 4096) == 0
            assert int(r["u64_sum"]) == s.n and int(r["status"]) == 0


@pytest.mark.parametrize("split", [True, False])
def test_mixed_batch_matches_oracle_and_alone(env, split):
    c, scl, st, torch = env
    scl.scl_set_batch_split(c.handle, split)
    rng = np.random.default_rng(200)
    sizes = [0, 1, 255, 256, 4097, 65_536, 1_000_003, 3_000_000, 17, 123_456, 8_388_608, 999]
    specs = [synth.TaskSpec(int(k), n, 1000 + i)
             for i, (n, k) in enumerate(zip(sizes * 3, rng.integers(0, 3, size=36)))]
    parts, data, outs, tasks = make_batch(c, scl, st, torch, specs)
    arr = scl.make_tasks(tasks)
    res = scl.scl_batch_run(c.handle, arr, len(tasks), stream=st)
    torch.cuda.synchronize()
    check_batch(scl, specs, data, outs, res)
    # alone: same bits for the streaming kinds
    for i, s in enumerate(specs):
        if s.kind == synth.KIND_KEYED:
            continue
        t = tasks[i]
        r = scl.scl_map_reduce(c.handle, t["part"], t["kernel"], t["reduce"], stream=st)
        assert r.u64_sum == int(res[i]["u64_sum"]), i
        assert r.f64_sum == float(res[i]["f64_sum"]) or (np.isnan(r.f64_sum)), i
        assert np.float32(r.f32_min) == res[i]["f32_min"] and \
            np.float32(r.f32_max) == res[i]["f32_max"], i
    scl.scl_set_batch_split(c.handle, True)


@pytest.mark.parametrize("kind", [synth.KIND_MIX32, synth.KIND_POLY3, synth.KIND_KEYED])
def test_homogeneous_batches(env, kind):
    c, scl, st, torch = env
    specs = [synth.TaskSpec(kind, n, 300 + i) for i, n in
             enumerate([5, 70_000, 2_500_000, 0, 4096, 1 << 20, 333_333])]
    parts, data, outs, tasks = make_batch(c, scl, st, torch, specs)
    res = scl.scl_batch_run(c.handle, scl.make_tasks(tasks), len(tasks), stream=st)
    check_batch(scl, specs, data, outs, res)


@pytest.mark.parametrize("split", [True, False])
def test_graph_replays_are_identical(env, split):
    c, scl, st, torch = env
    specs = synth.batch_tasks(count=300, seed=9)
    parts, data, outs, tasks = make_batch(c, scl, st, torch, specs)
    arr = scl.make_tasks(tasks)
    scl.scl_set_batch_split(c.handle, split)
    b = scl.scl_batch_create(c.handle, arr, len(tasks))
    scl.scl_set_batch_split(c.handle, True)
    s2 = torch.cuda.Stream()
    scl.scl_batch_capture(b, s2.cuda_stream)
    first = None
    for _ in range(4):
        scl.scl_batch_launch(b, s2.cuda_stream)
        res = scl.scl_batch_results(b, len(tasks), stream=s2.cuda_stream)
        if first is None:
            first = res.copy()
            check_batch(scl, specs, data, outs, res)
        else:
            streaming = np.array([s.kind != synth.KIND_KEYED for s in specs])
            assert np.array_equal(res[streaming], first[streaming])
            assert np.array_equal(res["u64_sum"], first["u64_sum"])
    # split: a kernel per family (3) and the keyed fold; mixed: one and the fold
    assert scl.scl_batch_kernel_launches(b) in ((3, 4) if split else (1, 2))
    scl.scl_batch_destroy(b)


def test_split_and_mixed_launches_agree(env):
    c, scl, st, torch = env
    specs = synth.batch_tasks(count=500, seed=21)
    parts, data, outs, tasks = make_batch(c, scl, st, torch, specs)
    arr = scl.make_tasks(tasks)
    got = {}
    for split in (True, False):
        scl.scl_set_batch_split(c.handle, split)
        got[split] = scl.scl_batch_run(c.handle, arr, len(tasks), stream=st)
        check_batch(scl, specs, data, outs, got[split])
    scl.scl_set_batch_split(c.handle, True)
    streaming = np.array([s.kind != synth.KIND_KEYED for s in specs])
    assert np.array_equal(got[True][streaming], got[False][streaming])
    assert np.array_equal(got[True]["u64_sum"], got[False]["u64_sum"])
    assert scl.lib.scl_set_batch_split(c.handle, 2) == scl.SCL_E_INVALID


def test_single_task_and_empty_batches(env):
    c, scl, st, torch = env
    specs = [synth.TaskSpec(synth.KIND_POLY3, 5_000_000, 77)]
    parts, data, outs, tasks = make_batch(c, scl, st, torch, specs)
    res = scl.scl_batch_run(c.handle, scl.make_tasks(tasks), 1, stream=st)
    check_batch(scl, specs, data, outs, res)
    res = scl.scl_batch_run(c.handle, scl.make_tasks([]), 0, stream=st)
    assert res.size == 0


def test_one_big_and_many_tiny(env):
    c, scl, st, torch = env
    specs = [synth.TaskSpec(synth.KIND_MIX32, 8_388_608, 5)] + \
            [synth.TaskSpec(i % 3, 256 + (i % 7), 10 + i) for i in range(2000)]
    parts, data, outs, tasks = make_batch(c, scl, st, torch, specs)
    res = scl.scl_batch_run(c.handle, scl.make_tasks(tasks), len(tasks), stream=st)
    check_batch(scl, specs, data, outs, res)


@pytest.mark.parametrize("kinds", [(synth.KIND_MIX32, synth.KIND_KEYED),
                                   (synth.KIND_POLY3, synth.KIND_KEYED),
                                   (synth.KIND_MIX32, synth.KIND_POLY3)])
def test_two_family_batches(env, kinds):
    # split into two concurrent launch groups (the keyed one, if any, on the
    # 48-register kernel)
    c, scl, st, torch = env
    sizes = [3_000_000, 200_000, 20_000, 4097, 0, 1_000_003]
    specs = [synth.TaskSpec(kinds[i % 2], n, 700 + i) for i, n in enumerate(sizes)]
    parts, data, outs, tasks = make_batch(c, scl, st, torch, specs)
    arr = scl.make_tasks(tasks)
    b = scl.scl_batch_create(c.handle, arr, len(tasks))
    assert scl.scl_batch_kernel_launches(b) in (2, 3)
    s2 = torch.cuda.Stream()   # capture needs a stream other than the legacy default
    scl.scl_batch_capture(b, s2.cuda_stream)
    scl.scl_batch_launch(b, s2.cuda_stream)
    res = scl.scl_batch_results(b, len(tasks), stream=s2.cuda_stream)
    scl.scl_batch_destroy(b)
    check_batch(scl, specs, data, outs, res)


@pytest.mark.parametrize("n", [20_000, 200_000, 3_000_000])
def test_split_batch_key_out_of_range(env, n):
    # one keyed piece (20 K pairs), a few pieces folded by the last writer
    # (200 K), many pieces folded by k_keyed_fold (3 M): a bad key is reported,
    # and the next launch of a clean batch is not affected
    c, scl, st, torch = env
    rng = np.random.default_rng(800 + n % 97)
    keys = rng.integers(0, 4096, size=n, dtype=np.int32)
    keys[[1, n - 1]] = [-5, 4096]
    vals = rng.random(n, dtype=np.float32)
    pk = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
    o = (torch.zeros(4096, dtype=torch.int32, device="cuda"),
         torch.zeros(4096, dtype=torch.float32, device="cuda"))
    specs = [synth.TaskSpec(synth.KIND_MIX32, 100_000, 901), synth.TaskSpec(synth.KIND_POLY3, 70_000, 902)]
    parts, data, outs, tasks = make_batch(c, scl, st, torch, specs)
    bad = dict(part=pk, kernel=scl.SCL_K_IDENT, reduce=scl.SCL_R_KEYED_COUNT_SUM, num_keys=4096,
               counts_out=o[0], sums_out=o[1])
    with pytest.raises(scl.SclError) as e:
        scl.scl_batch_run(c.handle, scl.make_tasks(tasks + [bad]), 3, stream=st)
    assert e.value.status == scl.SCL_E_KEY_RANGE
    res = scl.scl_batch_run(c.handle, scl.make_tasks(tasks + [bad]), 3, stream=st,
                            allow_key_range=True)
    assert int(res[2]["status"]) == scl.SCL_E_KEY_RANGE and int(res[2]["u64_sum"]) == n - 2
    assert int(res[0]["status"]) == 0 and int(res[1]["status"]) == 0
    check_batch(scl, specs, data, outs, res[:2])
    cnt = o[0].cpu().numpy().view(np.uint32)
    ocnt, _, _ = oracle.keyed_count_sum(keys, vals, 4096)
    assert np.array_equal(cnt, ocnt)   # the bad keys are dropped, the rest counted
    res = scl.scl_batch_run(c.handle, scl.make_tasks(tasks), 2, stream=st)
    check_batch(scl, specs, data, outs, res)
