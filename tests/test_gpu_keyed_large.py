"""Keyed reduce over large key spaces (up to 2^24 keys): counts bit-exact and
sums within 1e-5 of the fp64 oracle, for uniform keys and for Zipf-skewed keys
whose frequent ids are small (the shared-memory hot table); out-of-range keys
are skipped and reported."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_common import check_keyed, check_keyed_nonfinite
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


def _launches(scl, fn):
    before = scl.scl_kernel_launches_total()
    out = fn()
    return out, scl.scl_kernel_launches_total() - before


class _path:
    """The context's large-key path for one test, back to automatic after."""

    def __init__(self, scl, ctx, path):
        self.scl, self.ctx, self.path = scl, ctx, path

    def __enter__(self):
        self.scl.scl_set_large_path(self.ctx, self.path)

    def __exit__(self, *exc):
        self.scl.scl_set_large_path(self.ctx, self.scl.SCL_LARGE_AUTO)


# Bucket-partitioned path (chosen with SCL_LARGE_PARTITIONED; taken for
# partitions of at least 2^20 aligned pairs over more than 4096 keys):
# histogram, scan, the two scatter forms (one of them returns at once), the
# per-bucket reduce, then the finishing pass -- 6 launches; the direct path
# makes 2.
RADIX_CASES = {
    # every pair on an id below 1024: counted in the scatter's hot tables, the
    # partition stays empty
    "all_hot": lambda rng: (1 << 20, rng.integers(0, 1024, (1 << 20) + 9, dtype=np.int32)),
    # ids on both sides of the hot limit (1022 .. 1026): hot ids bypass
    "hot_edge": lambda rng: (5000, rng.integers(1022, 1027, (1 << 20) + 2, dtype=np.int32)),
    # hot ids just under 1/8 of the pairs: no bypass, they go through bucket 0
    "few_hot": lambda rng: (1 << 20, np.where(rng.random((1 << 20) + 3) < 0.12,
                                              rng.integers(0, 1024, (1 << 20) + 3),
                                              rng.integers(1024, 1 << 20, (1 << 20) + 3)
                                              ).astype(np.int32)),
    # one key for every pair: a single bucket split over the whole grid
    "one_key": lambda rng: (1 << 20, np.full((1 << 20) + 3, 777_777, np.int32)),
    # only the last, partial bucket (3 keys) is used
    "last_bucket": lambda rng: (4096 * 5 + 3,
                                rng.integers(4096 * 5, 4096 * 5 + 3, (1 << 20) + 1,
                                             dtype=np.int32)),
    # odd length: ragged tails in every pass
    "odd_length": lambda rng: (1 << 20, rng.integers(0, 1 << 20, (1 << 20) + 12_345,
                                                    dtype=np.int32)),
    # 2^24 keys: 1024 buckets of 16384 ids, a few pairs per id
    "max_keys": lambda rng: (1 << 24, rng.integers(0, 1 << 24, 1 << 21, dtype=np.int32)),
    # 2^24 keys, Zipf: the hot ids in bucket 0 of the widest table
    "max_keys_zipf": lambda rng: (1 << 24, synth.zipf_keys_i32(1 << 21, rng, 1 << 24)),
    # 2^23 + 1 keys: 513 buckets of 16384 ids, the last holding one id (two
    # buckets per thread in the tile scan)
    "wide_buckets": lambda rng: ((1 << 23) + 1,
                                 rng.integers(0, (1 << 23) + 1, (1 << 20) + 5, dtype=np.int32)),
    # 2^19 + 3 keys: 65 buckets of 8192 ids, the last holding 3
    "buckets_8192": lambda rng: ((1 << 19) + 3,
                                 rng.integers(0, (1 << 19) + 3, (1 << 20) + 11, dtype=np.int32)),
    # 2^22 keys: 256 buckets of 16384 ids
    "mid_buckets": lambda rng: (1 << 22, rng.integers(0, 1 << 22, 3 << 20, dtype=np.int32)),
    # 2^21 + 7 keys: 129 buckets of 16384 ids, the last holding 7
    "buckets_16384": lambda rng: ((1 << 21) + 7,
                                 rng.integers(0, (1 << 21) + 7, (1 << 21) + 3, dtype=np.int32)),
    # sorted keys: CTAs that hold whole buckets store them without atomics
    "sorted": lambda rng: (1 << 22, np.sort(rng.integers(0, 1 << 22, 1 << 21,
                                                         dtype=np.int32))),
    # Zipf(1.2): most pairs in bucket 0, one hot key per warp
    "zipf": lambda rng: (1 << 20, synth.zipf_keys_i32(3_000_000, rng, 1 << 20)),
    # two keys in different buckets, alternating
    "two_buckets": lambda rng: (8192 + 10, np.tile(np.array([3, 8195], np.int32),
                                                   (1 << 20) // 2 + 7)),
}


@pytest.mark.parametrize("case", sorted(RADIX_CASES))
def test_large_radix_cases(env, case):
    c, scl, st, _ = env
    rng = np.random.default_rng(1900 + len(case))
    nk, keys = RADIX_CASES[case](rng)
    vals = rng.random(keys.size, dtype=np.float32)
    p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
    with _path(scl, c.handle, scl.SCL_LARGE_PARTITIONED):
        (cnt, sums, s64, r), nl = _launches(
            scl, lambda: scl.scl_keyed_reduce_large(c.handle, p, nk, stream=st))
    assert nl == 6
    assert check_keyed(cnt, sums, s64, keys, vals, nk) == 0
    assert r.status == 0 and r.u64_sum == keys.size and r.n == keys.size
    scl.scl_free_partition(c.handle, p)


def test_large_radix_out_of_range(env):
    """Out-of-range keys are dropped by the histogram and the scatter alike;
    the tables of the valid pairs stay exact."""
    c, scl, st, _ = env
    rng = np.random.default_rng(2000)
    nk, n = 300_000, (1 << 20) + 77
    keys = rng.integers(0, nk, size=n, dtype=np.int32)
    keys[[0, 1, 4096, n // 2, n - 1]] = [nk, -1, 1 << 30, nk + 4096, -(1 << 31)]
    vals = rng.random(n, dtype=np.float32)
    p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
    with _path(scl, c.handle, scl.SCL_LARGE_PARTITIONED), pytest.raises(scl.SclError) as e:
        scl.scl_keyed_reduce_large(c.handle, p, nk, stream=st)
    assert e.value.status == scl.SCL_E_KEY_RANGE
    cnt, sums, s64, r = e.value.tables
    assert check_keyed(cnt, sums, s64, keys, vals, nk) == 5
    assert r.u64_sum == n - 5
    scl.scl_free_partition(c.handle, p)


def test_large_radix_and_direct_agree(env):
    """The same pairs through the partitioned path (aligned) and the direct
    kernel (a view one pair in, so 4-byte aligned only): counts identical,
    sums within the fp32 tolerance of the oracle on both."""
    c, scl, st, torch = env
    rng = np.random.default_rng(2100)
    nk, n = 1 << 19, (1 << 21) + 1
    keys = rng.integers(0, nk, size=n, dtype=np.int32)
    vals = rng.random(n, dtype=np.float32)
    dk = torch.from_numpy(keys).cuda()
    dv = torch.from_numpy(vals).cuda()
    torch.cuda.synchronize()
    whole = scl.scl_wrap_device(c.handle, dk.data_ptr(), dv.data_ptr(), scl.SCL_KV_I32_F32, n)
    tail = scl.scl_wrap_device(c.handle, dk.data_ptr() + 4, dv.data_ptr() + 4,
                               scl.SCL_KV_I32_F32, n - 1)
    with _path(scl, c.handle, scl.SCL_LARGE_PARTITIONED):
        (a, _, _, _), na = _launches(scl, lambda: scl.scl_keyed_reduce_large(c.handle, whole, nk,
                                                                            stream=st))
        (b, bs, b64, _), nb_ = _launches(scl, lambda: scl.scl_keyed_reduce_large(
            c.handle, tail, nk, stream=st))
    assert (na, nb_) == (6, 2)
    ref = np.bincount(keys, minlength=nk).astype(np.uint32)
    assert np.array_equal(a, ref)
    ref[keys[0]] -= 1
    assert np.array_equal(b, ref)
    assert check_keyed(b, bs, b64, keys[1:], vals[1:], nk) == 0
    scl.scl_free_partition(c.handle, whole)
    scl.scl_free_partition(c.handle, tail)


def test_large_radix_falls_back_when_arena_is_short():
    """With no arena room for the bucket tables (8 B per pair) the direct
    kernel runs; the result is the same."""
    import torch
    from paper_1505_01120_gb300 import scl
    from paper_1505_01120_gb300.context import Context, current_stream
    rng = np.random.default_rng(2200)
    nk, n = 1 << 18, 1 << 21
    keys = rng.integers(0, nk, size=n, dtype=np.int32)
    vals = rng.random(n, dtype=np.float32)
    # partition 16 MiB + tables 4 MiB fit; another 16 MiB for the buckets does not
    with Context(24 << 20, device=0) as c:
        st = current_stream(0)
        scl.scl_set_large_path(c.handle, scl.SCL_LARGE_PARTITIONED)
        p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
        (cnt, sums, s64, r), nl = _launches(
            scl, lambda: scl.scl_keyed_reduce_large(c.handle, p, nk, stream=st))
        assert nl == 2
        assert check_keyed(cnt, sums, s64, keys, vals, nk) == 0
        scl.scl_free_partition(c.handle, p)
    torch.cuda.synchronize()


def test_large_async_buffer_grows_and_is_reused(env):
    """The async form keeps its bucket copy per stream: a larger partition
    grows it (after the device drains), a smaller one reuses it; every table
    exact in counts."""
    c, scl, st, torch = env
    rng = np.random.default_rng(2300)
    nk = 1 << 18
    s2 = torch.cuda.Stream()
    dc = torch.empty(nk, dtype=torch.int32, device="cuda")
    ds = torch.empty(nk, dtype=torch.float32, device="cuda")
    d64 = torch.empty(nk, dtype=torch.float64, device="cuda")
    dr = torch.empty(48, dtype=torch.uint8, device="cuda")
    for n in ((1 << 20) + 5, 3 << 20, (1 << 20) + 77):
        keys = rng.integers(0, nk, size=n, dtype=np.int32)
        vals = rng.random(n, dtype=np.float32)
        p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
        torch.cuda.synchronize()
        before = scl.scl_kernel_launches_total()
        with _path(scl, c.handle, scl.SCL_LARGE_PARTITIONED):
            scl.scl_keyed_reduce_large_async(c.handle, p, nk, dc, ds, d64, dr,
                                             stream=s2.cuda_stream)
        nl = scl.scl_kernel_launches_total() - before
        torch.cuda.synchronize()
        assert nl == 6
        assert check_keyed(dc.cpu().numpy().view(np.uint32), ds.cpu().numpy(),
                           d64.cpu().numpy(), keys, vals, nk) == 0
        scl.scl_free_partition(c.handle, p)


# Packed direct path (the default for 2^17 to 2^22 keys): the scale pass, the direct
# kernel with packed L2 words, the finishing pass, then the three guarded
# kernels of the repair chain -- 6 launches whether or not the repair runs.

def test_packed_values_on_both_sides_of_the_window(env):
    """Values below the window, above it, negative, zeros, NaN and inf, on ids
    above and below 4096: exact counts, sums within the fp32 tolerance,
    non-finite sums as the oracle's."""
    c, scl, st, _ = env
    rng = np.random.default_rng(2400)
    nk, n = 1 << 20, 3_000_017
    keys = rng.integers(0, nk, size=n, dtype=np.int32)
    vals = rng.random(n, dtype=np.float32)
    idx = rng.choice(n, size=n // 40, replace=False)
    q = len(idx) // 5
    vals[idx[:q]] = rng.random(q, dtype=np.float32) * np.float32(1e-4)
    vals[idx[q:2 * q]] = np.float32(2.0) + rng.random(q, dtype=np.float32) * 1000
    vals[idx[2 * q:3 * q]] = 0.0
    vals[idx[3 * q:4 * q]] = -0.0
    vals[idx[4 * q:]] = -rng.random(len(idx) - 4 * q, dtype=np.float32) * np.float32(1e-3)
    vals[[7, 1000, 2_000_000]] = [np.nan, np.inf, -np.inf]
    keys[[7, 1000, 2_000_000]] = [5000, 100, 700_000]
    p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
    (cnt, sums, s64, r), nl = _launches(
        scl, lambda: scl.scl_keyed_reduce_large(c.handle, p, nk, stream=st))
    assert nl == 6 and r.status == 0 and r.u64_sum == n
    check_keyed_nonfinite(cnt, sums, s64, keys, vals, nk)
    scl.scl_free_partition(c.handle, p)


@pytest.mark.parametrize("hot", [40_000, 17_000_000])
def test_packed_overflow_is_repaired(env, hot):
    """One id far above 4096 takes more packed pairs than its word holds:
    40,000 values near 1 overflow the 40-bit sum (limit 32,768 at 2^25 each);
    17 M pairs also wrap the 24-bit count.  The finishing pass sees the
    decoded counts fall short of the packed adds and the repair chain redoes
    the call without packing: the same tables."""
    c, scl, st, _ = env
    rng = np.random.default_rng(2500 + hot % 97)
    nk = 1 << 20
    n = hot + 1_000_003
    keys = rng.integers(0, nk, size=n, dtype=np.int32)
    keys[rng.permutation(n)[:hot]] = 654_321
    vals = (np.float32(0.5) + np.float32(0.5) * rng.random(n, dtype=np.float32)).astype(np.float32)
    p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
    (cnt, sums, s64, r), nl = _launches(
        scl, lambda: scl.scl_keyed_reduce_large(c.handle, p, nk, stream=st))
    assert nl == 6 and r.status == 0 and r.u64_sum == n
    assert check_keyed(cnt, sums, s64, keys, vals, nk) == 0
    assert cnt[654_321] >= hot
    scl.scl_free_partition(c.handle, p)


@pytest.mark.parametrize("kind", ["negative", "zeros", "huge"])
def test_packed_without_a_window(env, kind):
    """No window (no non-negative finite value, only zeros, or values beyond
    2^90): every pair takes the count / fp64 adds; same tables."""
    c, scl, st, _ = env
    rng = np.random.default_rng(2600)
    nk, n = 100_000, 1_500_000
    keys = rng.integers(0, nk, size=n, dtype=np.int32)
    if kind == "negative":
        vals = -rng.random(n, dtype=np.float32)
    elif kind == "zeros":
        vals = np.zeros(n, np.float32)
    else:
        vals = (rng.random(n, dtype=np.float32) * np.float32(1e30)).astype(np.float32)
    p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
    with _path(scl, c.handle, scl.SCL_LARGE_PACKED):
        cnt, sums, s64, r = scl.scl_keyed_reduce_large(c.handle, p, nk, stream=st)
    assert r.status == 0 and r.u64_sum == n
    if kind == "zeros":
        ocnt, _, _ = oracle.keyed_count_sum(keys, vals, nk)
        assert np.array_equal(cnt, ocnt) and np.all(s64 == 0) and np.all(sums == 0)
    else:
        assert check_keyed(cnt, sums, s64, keys, vals, nk) == 0
    scl.scl_free_partition(c.handle, p)


def test_packed_unaligned_async_and_paths_agree(env):
    """An unaligned view (the direct kernel's scalar loads) through the
    packed path, twice in a row on device tables; the direct path without
    packing and the partitioned path give the same counts and sums within
    the tolerance; an unknown path is rejected."""
    c, scl, st, torch = env
    rng = np.random.default_rng(2700)
    nk, n = 1 << 21, (1 << 21) + 3
    keys = rng.integers(0, nk, size=n, dtype=np.int32)
    vals = rng.random(n, dtype=np.float32)
    dk = torch.from_numpy(keys).cuda()
    dv = torch.from_numpy(vals).cuda()
    torch.cuda.synchronize()
    tail = scl.scl_wrap_device(c.handle, dk.data_ptr() + 4, dv.data_ptr() + 4,
                               scl.SCL_KV_I32_F32, n - 1)
    whole = scl.scl_wrap_device(c.handle, dk.data_ptr(), dv.data_ptr(), scl.SCL_KV_I32_F32, n)
    dc = torch.empty(nk, dtype=torch.int32, device="cuda")
    ds = torch.empty(nk, dtype=torch.float32, device="cuda")
    d64 = torch.empty(nk, dtype=torch.float64, device="cuda")
    dr = torch.empty(48, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        scl.scl_keyed_reduce_large_async(c.handle, tail, nk, dc, ds, d64, dr, stream=st)
        torch.cuda.synchronize()
        assert check_keyed(dc.cpu().numpy().view(np.uint32), ds.cpu().numpy(),
                           d64.cpu().numpy(), keys[1:], vals[1:], nk) == 0
        res = dr.cpu().numpy().view(scl.RESULT_DTYPE)[0]
        assert int(res["status"]) == 0 and int(res["u64_sum"]) == n - 1
    tables = {}
    for path, want in ((scl.SCL_LARGE_PACKED, 6), (scl.SCL_LARGE_DIRECT, 2),
                       (scl.SCL_LARGE_PARTITIONED, 6)):
        with _path(scl, c.handle, path):
            (cnt, sums, s64, r), nl = _launches(
                scl, lambda: scl.scl_keyed_reduce_large(c.handle, whole, nk, stream=st))
        assert nl == want
        assert check_keyed(cnt, sums, s64, keys, vals, nk) == 0
        tables[path] = cnt
    assert np.array_equal(tables[scl.SCL_LARGE_PACKED], tables[scl.SCL_LARGE_DIRECT])
    assert np.array_equal(tables[scl.SCL_LARGE_PACKED], tables[scl.SCL_LARGE_PARTITIONED])
    with pytest.raises(scl.SclError) as e:
        scl.scl_set_large_path(c.handle, 9)
    assert e.value.status == scl.SCL_E_INVALID
    scl.scl_free_partition(c.handle, tail)
    scl.scl_free_partition(c.handle, whole)

