"""ReduceCL over partition arrays with the Fig. 3 vector-add kernel, on the GPU.

Each output element is the same fixed sequence of fp32 adds (the
binary-counter tree) on both sides, so results must match the oracle bit for
bit, for every k, length, alignment and dtype.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1505_01120_gb300 import scl
    from paper_1505_01120_gb300.context import Context, current_stream
    torch.cuda.set_device(0)
    c = Context(3 << 30, device=0)
    yield c, scl, current_stream(0), torch
    c.close()


def _load(c, scl, st, arrays, dtype):
    return [scl.scl_load_partition(c.handle, a, dtype, stream=st) for a in arrays]


def _read(c, scl, st, part, n, dt):
    out = np.empty(n, dt)
    scl.scl_read_partition(c.handle, part, out, stream=st)
    return out


@pytest.mark.parametrize("k", [1, 2, 3, 4, 7, 8, 13, 64, 100, 127, 128, 200])
def test_reduce_arrays_f32_bit_exact(env, k):
    c, scl, st, _ = env
    rng = np.random.default_rng(1000 + k)
    n = 40_961 if k <= 64 else 4099
    xs = [rng.standard_normal(n, dtype=np.float32) * np.float32(j % 5 + 1) for j in range(k)]
    parts = _load(c, scl, st, xs, scl.SCL_F32)
    out = scl.scl_reduce_arrays(c.handle, parts, stream=st)
    got = _read(c, scl, st, out, n, np.float32)
    assert np.array_equal(got.view(np.uint32), oracle.add_arrays(xs).view(np.uint32)), k
    for p in parts + [out]:
        scl.scl_free_partition(c.handle, p)


def test_vector_add_and_sizes(env):
    c, scl, st, _ = env
    rng = np.random.default_rng(1100)
    for n in (0, 1, 3, 4, 5, 1023, 1024, 1025, 1_000_003):
        a = rng.standard_normal(n, dtype=np.float32)
        b = rng.standard_normal(n, dtype=np.float32)
        pa, pb = _load(c, scl, st, [a, b], scl.SCL_F32)
        pc = scl.scl_vector_add(c.handle, pa, pb, stream=st)
        got = _read(c, scl, st, pc, n, np.float32)
        assert np.array_equal(got.view(np.uint32), np.add(a, b).view(np.uint32)), n
        for p in (pa, pb, pc):
            scl.scl_free_partition(c.handle, p)


def test_reduce_arrays_u32_wraps(env):
    c, scl, st, _ = env
    rng = np.random.default_rng(1200)
    xs = [rng.integers(0, 1 << 32, size=77_777, dtype=np.uint32) for _ in range(9)]
    parts = _load(c, scl, st, xs, scl.SCL_U32)
    out = scl.scl_reduce_arrays(c.handle, parts, stream=st)
    assert np.array_equal(_read(c, scl, st, out, xs[0].size, np.uint32), oracle.add_arrays(xs))


def test_tree_shape_rounding_cases(env):
    c, scl, st, _ = env
    big, one, zero = np.float32(2.0 ** 24), np.float32(1.0), np.float32(0.0)
    for vals, want in (((big, one, one), big),
                       ((one, one, one, one, big, one), big + np.float32(4.0)),
                       ((big, zero, zero, zero, one, zero, one), big + np.float32(2.0))):
        xs = [np.full(4101, v, np.float32) for v in vals]
        parts = _load(c, scl, st, xs, scl.SCL_F32)
        out = scl.scl_reduce_arrays(c.handle, parts, stream=st)
        got = _read(c, scl, st, out, 4101, np.float32)
        assert np.all(got == want), (vals, got[:3])


def test_unaligned_inputs_and_into(env):
    c, scl, st, torch = env
    rng = np.random.default_rng(1300)
    n, k = 100_003, 6
    xs = [rng.standard_normal(n + 1, dtype=np.float32) for _ in range(k)]
    ds = [torch.from_numpy(x).cuda() for x in xs]
    torch.cuda.synchronize()
    parts = [scl.scl_wrap_device(c.handle, d.data_ptr() + 4, None, scl.SCL_F32, n) for d in ds]
    want = oracle.add_arrays([x[1:] for x in xs])
    out = scl.scl_reduce_arrays(c.handle, parts, stream=st)
    assert np.array_equal(_read(c, scl, st, out, n, np.float32).view(np.uint32),
                          want.view(np.uint32))
    # into an existing (aligned) partition: nothing allocated, same bits
    free0 = scl.scl_arena_stats(c.handle)[0]
    scl.scl_reduce_arrays_into(c.handle, parts, out, stream=st)
    assert scl.scl_arena_stats(c.handle)[0] == free0
    assert np.array_equal(_read(c, scl, st, out, n, np.float32).view(np.uint32),
                          want.view(np.uint32))


def test_reduce_arrays_errors(env):
    c, scl, st, _ = env
    a = scl.scl_load_partition(c.handle, np.zeros(10, np.float32), scl.SCL_F32, stream=st)
    b = scl.scl_load_partition(c.handle, np.zeros(11, np.float32), scl.SCL_F32, stream=st)
    u = scl.scl_load_partition(c.handle, np.zeros(10, np.uint32), scl.SCL_U32, stream=st)
    kv = scl.scl_load_partition_kv(c.handle, np.zeros(10, np.int32), np.zeros(10, np.float32),
                                   stream=st)
    for parts, status in (([a, b], scl.SCL_E_INVALID), ([a, u], scl.SCL_E_INVALID),
                          ([a, kv], scl.SCL_E_UNSUPPORTED), ([], scl.SCL_E_INVALID),
                          ([a] * 1025, scl.SCL_E_INVALID)):
        with pytest.raises(scl.SclError) as e:
            scl.scl_reduce_arrays(c.handle, parts, stream=st)
        assert e.value.status == status
