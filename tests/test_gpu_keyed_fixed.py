"""The keyed reduce's fixed-point window against the oracle.

Long pieces over key spaces of 1024 keys or more add the values inside the
window [B/32, B) as int32 multiples of 2^-F; B is the power of two just above
the largest value of the piece's first chunk.  Other values take fp32 adds.
A window in which one key takes 512 pairs or more makes the piece run again
on the fp32 table.  These cases cover values on both sides of the window,
zeros of both signs, negative values, NaN and inf, a first chunk much smaller
than the rest, a key that overflows a window, Zipf keys (most pairs on the
head ids below 32), and hashed keys.  Counts must
be exact and sums within 1e-5 of the fp64 oracle.  Non-finite sums must match
the oracle's (NaN where it has NaN, the same infinity).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_common import REL, check_keyed, check_keyed_nonfinite

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1505_01120_gb300 import scl
    from paper_1505_01120_gb300.context import Context, current_stream
    torch.cuda.set_device(0)
    c = Context(2 << 30, device=0)
    yield c, scl, current_stream(0)
    c.close()


def _run(env, keys, vals, nk):
    c, scl, st = env
    p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
    try:
        cnt, sums, s64, r = scl.scl_keyed_reduce(c.handle, p, nk, stream=st)
    finally:
        scl.scl_free_partition(c.handle, p)
    assert r.status == 0 and r.u64_sum == keys.size
    return cnt, sums, s64


@pytest.mark.parametrize("n", [16_384, 65_536 * 3 + 4097, 2_000_003])
def test_uniform_values_in_and_out_of_window(env, n):
    rng = np.random.default_rng(500 + n % 97)
    keys = rng.integers(0, 4096, size=n, dtype=np.int32)
    vals = rng.random(n, dtype=np.float32)
    # values below the window, above it, zeros of both signs, a few negatives
    idx = rng.choice(n, size=n // 50, replace=False)
    q = len(idx) // 5
    vals[idx[:q]] = rng.random(q, dtype=np.float32) * np.float32(1e-3)
    vals[idx[q:2 * q]] = np.float32(3.0) + rng.random(q, dtype=np.float32) * 100
    vals[idx[2 * q:3 * q]] = 0.0
    vals[idx[3 * q:4 * q]] = -0.0
    vals[idx[4 * q:]] = -rng.random(len(idx) - 4 * q, dtype=np.float32) * np.float32(0.01)
    cnt, sums, s64 = _run(env, keys, vals, 4096)
    assert check_keyed(cnt, sums, s64, keys, vals, 4096) == 0


def test_first_chunk_smaller_than_the_rest(env):
    n = 1_500_000
    rng = np.random.default_rng(501)
    keys = rng.integers(0, 4096, size=n, dtype=np.int32)
    vals = rng.random(n, dtype=np.float32)
    vals[:40_000] *= np.float32(0.01)    # window chosen on values below 0.01
    cnt, sums, s64 = _run(env, keys, vals, 4096)
    assert check_keyed(cnt, sums, s64, keys, vals, 4096) == 0


@pytest.mark.parametrize("scale", [1e-20, 1e-3, 7.5, 1e12, 1e25])
def test_magnitudes(env, scale):
    n = 600_000
    rng = np.random.default_rng(502)
    keys = rng.integers(0, 2048, size=n, dtype=np.int32)
    vals = (rng.random(n, dtype=np.float32) * np.float32(scale)).astype(np.float32)
    cnt, sums, s64 = _run(env, keys, vals, 2048)
    assert check_keyed(cnt, sums, s64, keys, vals, 2048) == 0


def test_nan_and_inf(env):
    n = 800_000
    rng = np.random.default_rng(503)
    keys = rng.integers(0, 4096, size=n, dtype=np.int32)
    vals = rng.random(n, dtype=np.float32)
    vals[[10, 200_000, 700_001]] = [np.nan, np.inf, -np.inf]
    keys[[10, 200_000, 700_001]] = [100, 200, 300]
    vals[5] = np.inf            # inside the first chunk
    keys[5] = 400
    cnt, sums, s64 = _run(env, keys, vals, 4096)
    check_keyed_nonfinite(cnt, sums, s64, keys, vals, 4096)


def test_window_overflow_reruns_on_the_fp32_table(env):
    n = 1_000_000
    rng = np.random.default_rng(504)
    keys = rng.integers(0, 4096, size=n, dtype=np.int32)
    keys[rng.random(n) < 0.3] = 1000        # far more than 512 pairs per window
    vals = rng.random(n, dtype=np.float32)
    cnt, sums, s64 = _run(env, keys, vals, 4096)
    assert check_keyed(cnt, sums, s64, keys, vals, 4096) == 0


def test_small_key_spaces_and_short_pieces(env):
    rng = np.random.default_rng(505)
    for nk, n in ((1023, 2_000_000), (1024, 2_000_000), (4096, 16_383), (4096, 16_385)):
        keys = rng.integers(0, nk, size=n, dtype=np.int32)
        vals = rng.random(n, dtype=np.float32)
        cnt, sums, s64 = _run(env, keys, vals, nk)
        assert check_keyed(cnt, sums, s64, keys, vals, nk) == 0


def test_hashed_keys(env):
    c, scl, st = env
    n = 3_000_000
    rng = np.random.default_rng(506)
    keys = rng.integers(-2**31, 2**31, size=n, dtype=np.int64).astype(np.int32)
    vals = rng.random(n, dtype=np.float32)
    p = scl.scl_load_partition_kv(c.handle, keys, vals, stream=st)
    cnt, sums, s64, r = scl.scl_keyed_reduce_hashed(c.handle, p, 4096, stream=st)
    scl.scl_free_partition(c.handle, p)
    ocnt, osum = oracle.keyed_hashed_count_sum(keys, vals, 4096)
    assert np.array_equal(cnt, ocnt)
    nz = ocnt > 0
    assert np.all(np.abs(s64[nz] - osum[nz]) <= REL * np.abs(osum[nz]))


@pytest.mark.parametrize("n", [1_000_003, 16_777_216])
def test_zipf_head_ids(env, n):
    # Zipf(1.2) keys put ~2/3 of the pairs on ids below 32, which take the
    # fp32 head copies while the other ids' in-window values take the int32
    # table.  Some head values are moved below and above the window, some
    # negated.
    from paper_1505_01120_gb300 import synth
    rng = np.random.default_rng(508)
    keys = synth.zipf_keys_i32(n, rng, 4096)
    vals = rng.random(n, dtype=np.float32)
    hot = np.nonzero(keys < 32)[0]
    sel = rng.choice(hot, size=len(hot) // 50, replace=False)
    q = len(sel) // 3
    vals[sel[:q]] *= np.float32(1e-4)
    vals[sel[q:2 * q]] = -vals[sel[q:2 * q]]
    vals[sel[2 * q:]] += np.float32(3.0)
    cnt, sums, s64 = _run(env, keys, vals, 4096)
    assert check_keyed(cnt, sums, s64, keys, vals, 4096) == 0


def test_repeat_calls_agree(env):
    n = 4_000_000
    rng = np.random.default_rng(507)
    keys = rng.integers(0, 4096, size=n, dtype=np.int32)
    vals = rng.random(n, dtype=np.float32)
    a = _run(env, keys, vals, 4096)
    b = _run(env, keys, vals, 4096)
    assert np.array_equal(a[0], b[0])
    assert np.all(np.abs(a[2] - b[2]) <= 2 * REL * np.abs(a[2]))
