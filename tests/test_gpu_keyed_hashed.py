"""Keyed reduce with keys hashed into buckets, (mix32(key) * num_keys) >> 32:
counts bit-exact and sums within 1e-5 of the fp64 oracle, alone, in batches
mixed with the plain keyed reduce, and through the server."""
from __future__ import annotations

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _check(cnt, sums, s64, keys, vals, nk):
    ocnt, osum = oracle.keyed_hashed_count_sum(keys, vals, nk)
    assert np.array_equal(cnt, ocnt)
    nz = ocnt > 0
    assert np.all(sums[~nz] == 0)
    assert np.all(np.abs(s64[nz] - osum[nz]) <= 1e-5 * np.abs(osum[nz]))
    assert np.all(np.abs(sums[nz].astype(np.float64) - osum[nz]) <= 1e-5 * np.abs(osum[nz]))


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1505_01120_gb300 import scl
    from paper_1505_01120_gb300.context import Context, current_stream
    torch.cuda.set_device(0)
    c = Context(2 << 30, device=0)
    yield c, scl, current_stream(0), torch
    c.close()


@pytest.mark.parametrize("nk", [1, 7, 1000, 4096])
def test_hashed_single(env, nk):
    c, scl, st, _ = env
    rng = np.random.default_rng(1400 + nk)
    for n in (0, 1, 63, 65, 4099, 300_001, 3_000_000):
        keys = rng.integers(-2**31, 2**31, size=n, dtype=np.int32)
        vals = rng.random(n, dtype=np.float32)
        p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
        cnt, sums, s64, r = scl.scl_keyed_reduce_hashed(c.handle, p, nk, stream=st)
        _check(cnt, sums, s64, keys, vals, nk)
        assert r.status == 0 and r.u64_sum == n     # no key is out of range
        scl.scl_free_partition(c.handle, p)


def test_hashed_in_batch_and_server(env):
    c, scl, st, torch = env
    rng = np.random.default_rng(1500)
    data, tasks, outs = [], [], []
    for i, n in enumerate([5, 70_000, 2_000_000, 0, 123_457, 1 << 20]):
        keys = rng.integers(-2**31, 2**31, size=n, dtype=np.int32)
        if i % 2:
            keys = keys & np.int32(4095)     # plain keyed tasks need keys in range
        vals = rng.random(n, dtype=np.float32)
        p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
        o = torch.zeros(4096 * 4, dtype=torch.int32, device="cuda")
        outs.append(o)
        data.append((keys, vals, i % 2 == 0))
        tasks.append(dict(part=p, kernel=scl.SCL_K_MIX32 if i % 2 == 0 else scl.SCL_K_IDENT,
                          reduce=scl.SCL_R_KEYED_COUNT_SUM, num_keys=4096,
                          counts_out=o.data_ptr(), sums_out=o.data_ptr() + 16384,
                          sums64_out=o.data_ptr() + 32768))
    arr = scl.make_tasks(tasks)

    def verify():
        for (keys, vals, hashed), o in zip(data, outs):
            t = o.cpu().numpy()
            cnt, sums, s64 = t[:4096].view(np.uint32), t[4096:8192].view(np.float32), \
                t[8192:].view(np.float64)
            if hashed:
                _check(cnt, sums, s64, keys, vals, 4096)
            else:
                ocnt, osum, bad = oracle.keyed_count_sum(keys, vals, 4096)
                assert bad == 0 and np.array_equal(cnt, ocnt)
            o.zero_()

    res = scl.scl_batch_run(c.handle, arr, len(tasks), stream=st)
    assert np.all(res["status"] == 0)
    verify()
    scl.scl_server_start(c.handle)
    try:
        tickets = [scl.scl_server_submit(c.handle, arr, i) for i in range(len(tasks))]
        for t in tickets:
            assert scl.scl_server_wait(c.handle, t).status == 0
    finally:
        scl.scl_server_stop(c.handle)
    verify()
