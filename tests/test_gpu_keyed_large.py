"""Keyed reduce over large key spaces (up to 2^24 keys): counts bit-exact and
sums within 1e-5 of the fp64 oracle, for uniform keys and for Zipf-skewed keys
whose frequent ids are small (the shared-memory hot table); out-of-range keys
are skipped and reported."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_common import check_keyed
from paper_1505_01120_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1505_01120_gb300 import scl
    from paper_1505_01120_gb300.context import Context, current_stream
    torch.cuda.set_device(0)
    c = Context(2 << 30, device=0)
    yield c, scl, current_stream(0), torch
    c.close()


@pytest.mark.parametrize("nk", [1, 4096, 4097, 65_536, 1 << 20, 1 << 24])
def test_large_uniform(env, nk):
    c, scl, st, _ = env
    rng = np.random.default_rng(1600 + nk % 9973)
    for n in (0, 1, 1000, 300_001, 5_000_000):
        keys = rng.integers(0, nk, size=n, dtype=np.int32)
        vals = rng.random(n, dtype=np.float32)
        p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
        cnt, sums, s64, r = scl.scl_keyed_reduce_large(c.handle, p, nk, stream=st)
        assert check_keyed(cnt, sums, s64, keys, vals, nk) == 0
        assert r.status == 0 and r.u64_sum == n and r.n == n
        total = float(vals.astype(np.float64).sum())
        assert abs(r.f64_sum - total) <= 1e-5 * max(total, 1.0)
        scl.scl_free_partition(c.handle, p)


def test_large_zipf(env):
    c, scl, st, _ = env
    rng = np.random.default_rng(1700)
    nk, n = 1 << 20, 20_000_000
    keys = synth.zipf_keys_i32(n, rng, nk)
    vals = rng.random(n, dtype=np.float32)
    p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
    cnt, sums, s64, r = scl.scl_keyed_reduce_large(c.handle, p, nk, stream=st)
    assert check_keyed(cnt, sums, s64, keys, vals, nk) == 0
    assert cnt[0] == cnt.max()      # the frequent id is 0


def test_large_out_of_range_and_async(env):
    c, scl, st, torch = env
    rng = np.random.default_rng(1800)
    nk, n = 100_000, 2_000_000
    keys = rng.integers(0, nk, size=n, dtype=np.int32)
    keys[[5, n - 1]] = [nk, -3]
    vals = rng.random(n, dtype=np.float32)
    p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
    with pytest.raises(scl.SclError) as e:
        scl.scl_keyed_reduce_large(c.handle, p, nk, stream=st)
    assert e.value.status == scl.SCL_E_KEY_RANGE
    cnt, sums, s64, r = e.value.tables
    assert check_keyed(cnt, sums, s64, keys, vals, nk) == 2
    # device tables, twice in a row (the tables are zeroed on the stream)
    dc = torch.empty(nk, dtype=torch.int32, device="cuda")
    ds = torch.empty(nk, dtype=torch.float32, device="cuda")
    d64 = torch.empty(nk, dtype=torch.float64, device="cuda")
    dr = torch.empty(48, dtype=torch.uint8, device="cuda")
    ok = keys.copy()
    ok[[5, n - 1]] = [0, 1]
    q = scl.scl_load_partition_kv(c.handle, ok, vals, stream=st)
    for _ in range(2):
        scl.scl_keyed_reduce_large_async(c.handle, q, nk, dc, ds, d64, dr, stream=st)
        torch.cuda.synchronize()
        assert check_keyed(dc.cpu().numpy().view(np.uint32), ds.cpu().numpy(),
                           d64.cpu().numpy(), ok, vals, nk) == 0
        res = dr.cpu().numpy().view(scl.RESULT_DTYPE)[0]
        assert int(res["status"]) == 0 and int(res["u64_sum"]) == n


def test_large_errors(env):
    c, scl, st, _ = env
    p = scl.scl_load_partition(c.handle, np.zeros(4, np.float32), scl.SCL_F32, stream=st)
    with pytest.raises(scl.SclError) as e:
        scl.scl_keyed_reduce_large(c.handle, p, 10, stream=st)
    assert e.value.status == scl.SCL_E_UNSUPPORTED
    q = scl.scl_load_partition_kv(c.handle, np.zeros(4, np.int32), np.zeros(4, np.float32),
                                  stream=st)
    for nk in (0, (1 << 24) + 1):
        with pytest.raises(scl.SclError) as e:
            scl.scl_keyed_reduce_large(c.handle, q, nk, stream=st)
        assert e.value.status == scl.SCL_E_INVALID


def test_large_async_on_four_streams(env):
    """Async large-key reduces on four streams at once (per-stream scratch):
    every table exact in counts."""
    c, scl, st, torch = env
    rng = np.random.default_rng(1800)
    nk, n = 1 << 18, 3_000_001
    data, parts = [], []
    for _ in range(4):
        keys = rng.integers(0, nk, size=n, dtype=np.int32)
        vals = rng.random(n, dtype=np.float32)
        data.append((keys, vals))
        parts.append(scl.scl_load_partition_kv(c.handle, keys, vals, stream=st))
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(4)]
    outs = [(torch.empty(nk, dtype=torch.int32, device="cuda"),
             torch.empty(nk, dtype=torch.float32, device="cuda"),
             torch.empty(nk, dtype=torch.float64, device="cuda"),
             torch.empty(48, dtype=torch.uint8, device="cuda")) for _ in range(4)]
    for rep in range(2):
        for p, s, o in zip(parts, streams, outs):
            scl.scl_keyed_reduce_large_async(c.handle, p, nk, o[0], o[1], o[2], o[3],
                                             stream=s.cuda_stream)
        torch.cuda.synchronize()
        for (keys, vals), o in zip(data, outs):
            cnt = o[0].cpu().numpy().view(np.uint32)
            assert check_keyed(cnt, o[1].cpu().numpy(), o[2].cpu().numpy(), keys, vals, nk) == 0
            r = o[3].cpu().numpy().view(scl.RESULT_DTYPE)[0]
            assert int(r["status"]) == 0 and int(r["u64_sum"]) == n
    for p in parts:
        scl.scl_free_partition(c.handle, p)
