"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Sizes span several segments and chunks plus ragged tails; unaligned
partitions are wrapped at odd element offsets of a device buffer; edge cases
are empty partitions, single elements, NaN/inf, all-equal keys, out-of-range
keys and the maximum key count.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1505_01120_gb300 import synth
from gpu_common import check_f32_result, check_keyed

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 3, 4, 5, 31, 32, 33, 127, 128, 129, 1023, 1024, 4095, 4096, 4097,
         16_383, 16_384, 16_385, 65_536 + 17, 262_144 - 3, 1_000_003]


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1505_01120_gb300 import scl
    from paper_1505_01120_gb300.context import Context, current_stream
    torch.cuda.set_device(0)
    c = Context(4 << 30, device=0)
    yield c, scl, current_stream(0), torch
    c.close()


def test_mix32_sum_bit_exact(env):
    c, scl, st, _ = env
    rng = np.random.default_rng(100)
    for n in SIZES:
        a = rng.integers(0, 1 << 32, size=n, dtype=np.uint32)
        p = scl.scl_load_partition(c.handle, a, scl.SCL_U32, stream=st)
        r = scl.scl_map_reduce(c.handle, p, scl.SCL_K_MIX32, scl.SCL_R_SUM, stream=st)
        assert r.u64_sum == oracle.sum_u32(a, mix=True), n
        assert r.n == n and r.status == 0
        r = scl.scl_map_reduce(c.handle, p, scl.SCL_K_IDENT, scl.SCL_R_SUM, stream=st)
        assert r.u64_sum == oracle.sum_u32(a, mix=False), n
        scl.scl_free_partition(c.handle, p)


def test_int32_partition_is_mixed_as_bits(env):
    c, scl, st, _ = env
    a = np.random.default_rng(101).integers(-2**31, 2**31, size=77_777, dtype=np.int32)
    p = scl.scl_load_partition(c.handle, a, scl.SCL_I32, stream=st)
    r = scl.scl_map_reduce(c.handle, p, scl.SCL_K_MIX32, scl.SCL_R_SUM, stream=st)
    assert r.u64_sum == oracle.sum_u32(a.view(np.uint32), mix=True)


def test_poly3_sum_min_max(env):
    c, scl, st, _ = env
    rng = np.random.default_rng(102)
    for n in SIZES:
        x = rng.standard_normal(n, dtype=np.float32)
        p = scl.scl_load_partition(c.handle, x, scl.SCL_F32, stream=st)
        r = scl.scl_map_reduce(c.handle, p, scl.SCL_K_POLY3, scl.SCL_R_SUM_MIN_MAX, stream=st)
        check_f32_result(r, x, True)
        r = scl.scl_map_reduce(c.handle, p, scl.SCL_K_IDENT, scl.SCL_R_SUM_MIN_MAX, stream=st)
        check_f32_result(r, x, False)
        scl.scl_free_partition(c.handle, p)


def test_poly3_other_coefficients(env):
    c, scl, st, _ = env
    x = np.random.default_rng(103).standard_normal(300_001, dtype=np.float32)
    coef = (-3.0, 0.75, 1e-3)
    p = scl.scl_load_partition(c.handle, x, scl.SCL_F32, stream=st)
    r = scl.scl_map_reduce(c.handle, p, scl.SCL_K_POLY3, scl.SCL_R_SUM, coef=coef, stream=st)
    check_f32_result(r, x, True, coef)


def test_empty_partition_results(env):
    c, scl, st, _ = env
    p = scl.scl_load_partition(c.handle, np.zeros(0, np.float32), scl.SCL_F32, stream=st)
    r = scl.scl_map_reduce(c.handle, p, scl.SCL_K_POLY3, scl.SCL_R_SUM_MIN_MAX, stream=st)
    assert r.n == 0 and r.f64_sum == 0.0 and r.f32_min == np.inf and r.f32_max == -np.inf
    p = scl.scl_load_partition(c.handle, np.zeros(0, np.uint32), scl.SCL_U32, stream=st)
    r = scl.scl_map_reduce(c.handle, p, scl.SCL_K_MIX32, scl.SCL_R_SUM, stream=st)
    assert r.n == 0 and r.u64_sum == 0


def test_nan_and_inf_handling(env):
    c, scl, st, _ = env
    x = np.random.default_rng(104).standard_normal(50_000, dtype=np.float32)
    x[[7, 4096, 33_333]] = np.nan
    p = scl.scl_load_partition(c.handle, x, scl.SCL_F32, stream=st)
    r = scl.scl_map_reduce(c.handle, p, scl.SCL_K_IDENT, scl.SCL_R_SUM_MIN_MAX, stream=st)
    check_f32_result(r, x, False)          # NaN sum, NaN-ignoring min/max
    x = np.random.default_rng(105).standard_normal(50_000, dtype=np.float32)
    x[123], x[40_000] = np.inf, -np.inf
    p = scl.scl_load_partition(c.handle, x, scl.SCL_F32, stream=st)
    r = scl.scl_map_reduce(c.handle, p, scl.SCL_K_IDENT, scl.SCL_R_SUM_MIN_MAX, stream=st)
    assert r.f32_min == -np.inf and r.f32_max == np.inf


def test_unaligned_wrapped_partitions(env):
    c, scl, st, torch = env
    rng = np.random.default_rng(106)
    a = rng.integers(0, 1 << 32, size=200_003, dtype=np.uint32)
    x = rng.standard_normal(200_003, dtype=np.float32)
    da = torch.from_numpy(a.view(np.int32)).cuda()
    dx = torch.from_numpy(x).cuda()
    torch.cuda.synchronize()
    for off in (1, 2, 3, 5):
        n = a.size - off - 7
        p = scl.scl_wrap_device(c.handle, da.data_ptr() + 4 * off, None, scl.SCL_U32, n)
        r = scl.scl_map_reduce(c.handle, p, scl.SCL_K_MIX32, scl.SCL_R_SUM, stream=st)
        assert r.u64_sum == oracle.sum_u32(a[off:off + n], mix=True), off
        q = scl.scl_wrap_device(c.handle, dx.data_ptr() + 4 * off, None, scl.SCL_F32, n)
        r = scl.scl_map_reduce(c.handle, q, scl.SCL_K_POLY3, scl.SCL_R_SUM_MIN_MAX, stream=st)
        check_f32_result(r, x[off:off + n], True)
        scl.scl_free_partition(c.handle, p)
        scl.scl_free_partition(c.handle, q)


def test_f32_results_bitwise_reproducible(env):
    c, scl, st, _ = env
    x = np.random.default_rng(107).standard_normal(3_000_017, dtype=np.float32)
    p = scl.scl_load_partition(c.handle, x, scl.SCL_F32, stream=st)
    rs = [scl.scl_map_reduce(c.handle, p, scl.SCL_K_POLY3, scl.SCL_R_SUM_MIN_MAX, stream=st)
          for _ in range(4)]
    for r in rs[1:]:
        assert r.f64_sum == rs[0].f64_sum and r.f32_min == rs[0].f32_min


@pytest.mark.parametrize("nk", [1, 17, 4096])
def test_keyed_count_sum(env, nk):
    c, scl, st, _ = env
    rng = np.random.default_rng(108 + nk)
    for n in [0, 1, 5, 63, 64, 65, 4097, 100_003, 2_000_001]:
        keys = rng.integers(0, nk, size=n, dtype=np.int32)
        vals = rng.random(n, dtype=np.float32)
        p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
        cnt, sums, s64, r = scl.scl_keyed_reduce(c.handle, p, nk, stream=st)
        assert check_keyed(cnt, sums, s64, keys, vals, nk) == 0
        assert r.n == n and r.u64_sum == n and r.status == 0
        scl.scl_free_partition(c.handle, p)


def test_keyed_ones_give_exact_counts_as_sums(env):
    c, scl, st, _ = env
    n = 4096 * 999
    keys = (np.arange(n) % 4096).astype(np.int32)
    p = scl.scl_load_partition_kv(c.handle, keys, np.ones(n, np.float32), stream=st)
    cnt, sums, s64, _ = scl.scl_keyed_reduce(c.handle, p, 4096, stream=st)
    assert np.all(cnt == 999) and np.all(sums == 999.0) and np.all(s64 == 999.0)


@pytest.mark.parametrize("nk", [1, 32, 33, 4096])
def test_keyed_zipf_keys(env, nk):
    """Zipf(1.2) keys, id 0 the most frequent: the sums of ids below 32 go
    through per-warp copies folded into the table.  Counts exact, sums within
    the fp32 tolerance; one CTA and many pieces alike."""
    c, scl, st, _ = env
    rng = np.random.default_rng(111 + nk)
    for n in (1000, 3_000_001):
        keys = synth.zipf_keys_i32(n, rng, nk)
        vals = rng.random(n, dtype=np.float32)
        p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
        cnt, sums, s64, r = scl.scl_keyed_reduce(c.handle, p, nk, stream=st)
        assert check_keyed(cnt, sums, s64, keys, vals, nk) == 0
        assert r.u64_sum == n and r.status == 0
        scl.scl_free_partition(c.handle, p)


def test_keyed_out_of_range_keys(env):
    c, scl, st, _ = env
    rng = np.random.default_rng(109)
    for n in (1000, 3_000_000):
        keys = rng.integers(0, 4096, size=n, dtype=np.int32)
        keys[[0, n // 2]] = [-1, 4096]
        vals = rng.random(n, dtype=np.float32)
        p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
        with pytest.raises(scl.SclError) as e:
            scl.scl_keyed_reduce(c.handle, p, 4096, stream=st)
        assert e.value.status == scl.SCL_E_KEY_RANGE
        cnt, sums, s64, r = e.value.tables
        assert check_keyed(cnt, sums, s64, keys, vals, 4096) == 2
        assert r.status == scl.SCL_E_KEY_RANGE and r.u64_sum == n - 2
        # the flag does not leak into the next call
        ok = scl.scl_load_partition_kv(c.handle, keys[1:n // 2], vals[1:n // 2], stream=st)
        scl.scl_keyed_reduce(c.handle, ok, 4096, stream=st)


def test_map_materialised_bit_exact(env):
    c, scl, st, torch = env
    rng = np.random.default_rng(110)
    for n in (0, 1, 7, 4096, 4099, 1_000_003):
        a = rng.integers(0, 1 << 32, size=n, dtype=np.uint32)
        p = scl.scl_load_partition(c.handle, a, scl.SCL_U32, stream=st)
        q = scl.scl_map(c.handle, p, scl.SCL_K_MIX32, stream=st)
        out = np.empty(n, np.uint32)
        scl.scl_read_partition(c.handle, q, out, stream=st)
        assert np.array_equal(out, oracle.map_mix32(a)), n
        x = rng.standard_normal(n, dtype=np.float32)
        p = scl.scl_load_partition(c.handle, x, scl.SCL_F32, stream=st)
        q = scl.scl_map(c.handle, p, scl.SCL_K_POLY3, stream=st)
        y = np.empty(n, np.float32)
        scl.scl_read_partition(c.handle, q, y, stream=st)
        assert np.array_equal(y.view(np.uint32), oracle.map_poly3(x).view(np.uint32)), n
    # unaligned source
    d = torch.from_numpy(a.view(np.int32)).cuda()
    torch.cuda.synchronize()
    p = scl.scl_wrap_device(c.handle, d.data_ptr() + 4, None, scl.SCL_U32, a.size - 1)
    q = scl.scl_map(c.handle, p, scl.SCL_K_MIX32, stream=st)
    out = np.empty(a.size - 1, np.uint32)
    scl.scl_read_partition(c.handle, q, out, stream=st)
    assert np.array_equal(out, oracle.map_mix32(a[1:]))


def test_map_into_existing_and_in_place(env):
    c, scl, st, torch = env
    rng = np.random.default_rng(112)
    x = rng.standard_normal(70_003, dtype=np.float32)
    p = scl.scl_load_partition(c.handle, x, scl.SCL_F32, stream=st)
    q = scl.scl_load_partition(c.handle, np.zeros_like(x), scl.SCL_F32, stream=st)
    free0 = scl.scl_arena_stats(c.handle)[0]
    scl.scl_map_into(c.handle, p, scl.SCL_K_POLY3, q, stream=st)
    assert scl.scl_arena_stats(c.handle)[0] == free0
    y = np.empty_like(x)
    scl.scl_read_partition(c.handle, q, y, stream=st)
    assert np.array_equal(y.view(np.uint32), oracle.map_poly3(x).view(np.uint32))
    scl.scl_map_into(c.handle, p, scl.SCL_K_POLY3, p, stream=st)      # in place
    scl.scl_read_partition(c.handle, p, y, stream=st)
    assert np.array_equal(y.view(np.uint32), oracle.map_poly3(x).view(np.uint32))
    r = scl.scl_load_partition(c.handle, np.zeros(5, np.float32), scl.SCL_F32, stream=st)
    with pytest.raises(scl.SclError) as e:
        scl.scl_map_into(c.handle, p, scl.SCL_K_POLY3, r, stream=st)
    assert e.value.status == scl.SCL_E_INVALID


def test_async_result_in_device_memory(env):
    c, scl, st, torch = env
    a = np.random.default_rng(111).integers(0, 1 << 32, size=123_457, dtype=np.uint32)
    p = scl.scl_load_partition(c.handle, a, scl.SCL_U32, stream=st)
    dev = torch.zeros(48 * 3, dtype=torch.uint8, device="cuda")
    for i in range(3):
        scl.scl_map_reduce_async(c.handle, p, scl.SCL_K_MIX32, scl.SCL_R_SUM,
                                 dev.data_ptr() + 48 * i, stream=st)
    torch.cuda.synchronize()
    res = dev.cpu().numpy().view(scl.RESULT_DTYPE)
    assert all(int(r["u64_sum"]) == oracle.sum_u32(a) for r in res)


def test_async_calls_on_many_streams_overlap_safely(env):
    """Async single-partition calls on 8 streams at once: each stream has its
    own scratch, so overlapping launches give the same results as one at a time."""
    c, scl, st, torch = env
    rng = np.random.default_rng(112)
    n = 3_000_017
    xs = [rng.standard_normal(n, dtype=np.float32) for _ in range(8)]
    parts = [scl.scl_load_partition(c.handle, x, scl.SCL_F32, stream=st) for x in xs]
    alone = [scl.scl_map_reduce(c.handle, p, scl.SCL_K_POLY3, scl.SCL_R_SUM_MIN_MAX, stream=st)
             for p in parts]
    streams = [torch.cuda.Stream() for _ in range(8)]
    dev = torch.zeros(48 * 8 * 4, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    for rep in range(4):
        for i, (p, s) in enumerate(zip(parts, streams)):
            scl.scl_map_reduce_async(c.handle, p, scl.SCL_K_POLY3, scl.SCL_R_SUM_MIN_MAX,
                                     dev.data_ptr() + 48 * (rep * 8 + i), stream=s.cuda_stream)
    torch.cuda.synchronize()
    res = dev.cpu().numpy().view(scl.RESULT_DTYPE).reshape(4, 8)
    for rep in range(4):
        for i in range(8):
            r = res[rep, i]
            assert float(r["f64_sum"]) == alone[i].f64_sum and int(r["n"]) == n, (rep, i)
            assert float(r["f32_min"]) == alone[i].f32_min
    for i, x in enumerate(xs):
        check_f32_result(alone[i], x, True)
    for p in parts:
        scl.scl_free_partition(c.handle, p)


def test_invalid_calls_raise(env):
    c, scl, st, _ = env
    with pytest.raises(scl.SclError) as e:
        scl.scl_map_reduce(c.handle, 987654, scl.SCL_K_MIX32, scl.SCL_R_SUM, stream=st)
    assert e.value.status == scl.SCL_E_INVALID
    p = scl.scl_load_partition(c.handle, np.zeros(10, np.float32), scl.SCL_F32, stream=st)
    with pytest.raises(scl.SclError) as e:
        scl.scl_map_reduce(c.handle, p, scl.SCL_K_MIX32, scl.SCL_R_SUM, stream=st)
    assert e.value.status == scl.SCL_E_UNSUPPORTED
    with pytest.raises(scl.SclError) as e:
        scl.scl_keyed_reduce(c.handle, p, 4096, stream=st)
    assert e.value.status == scl.SCL_E_UNSUPPORTED
