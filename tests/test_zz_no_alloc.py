"""The allocation-free map+reduce entry point against the regular one.

scl_map_reduce_noalloc is for callers that cannot allocate device memory when
they need a result (an open stream capture, a host application whose pool
owns all GPU memory, paths that cannot take cudaMalloc's synchronisation).
It keeps its scratch in a fixed device array inside the library.  This file
is collected last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process, where its
first call does the per-device set-up.
"""
from __future__ import annotations

import numpy as np
import pytest

from gpu_common import sum_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1505_01120_gb300 import scl
    from paper_1505_01120_gb300.context import Context, current_stream
    torch.cuda.set_device(0)
    c = Context(1 << 30, device=0)
    yield c, scl, current_stream(0), torch
    c.close()


CASES = [
    ("u32", 1, 0), ("u32", 1, 1_000_003), ("u32", 0, 4097),
    ("f32", 2, 3), ("f32", 2, 2_500_001), ("f32", 0, 65_537),
    ("u32", 1, 67_108_864), ("f32", 2, 67_108_864 - 5),
]


@pytest.mark.parametrize("kind,kernel,n", CASES)
def test_noalloc_matches_map_reduce_twice(env, kind, kernel, n):
    c, scl, st, torch = env
    rng = np.random.default_rng(n + kernel)
    if kind == "u32":
        host = rng.integers(0, 1 << 32, size=n, dtype=np.uint32)
        dtype, reduce = scl.SCL_U32, scl.SCL_R_SUM
        dev = torch.from_numpy(host.view(np.int32)).cuda()
    else:
        host = rng.standard_normal(n, dtype=np.float32)
        dtype, reduce = scl.SCL_F32, scl.SCL_R_SUM_MIN_MAX
        dev = torch.from_numpy(host).cuda()
    torch.cuda.synchronize()
    part = scl.scl_wrap_device(c.handle, dev.data_ptr(), None, dtype, n)
    ref = scl.scl_map_reduce(c.handle, part, kernel, reduce, stream=st)
    out = torch.zeros(2 * 48, dtype=torch.uint8, device="cuda")
    for i in range(2):   # two calls in a row share the fixed scratch
        scl.scl_map_reduce_noalloc(dev.data_ptr(), dtype, n, kernel, reduce,
                                   out.data_ptr() + 48 * i, stream=st)
    torch.cuda.synchronize()
    res = out.cpu().numpy().view(scl.RESULT_DTYPE)
    for r in res:
        assert int(r["n"]) == n and int(r["status"]) == 0
        if kind == "u32":
            assert int(r["u64_sum"]) == ref.u64_sum
        else:
            assert abs(float(r["f64_sum"]) - ref.f64_sum) <= sum_tol(ref.f64_sum, 0.0) + 1e-9
            assert r["f32_min"] == np.float32(ref.f32_min)
            assert r["f32_max"] == np.float32(ref.f32_max)
    scl.scl_free_partition(c.handle, part)


def test_noalloc_rejects_oversized_partitions(env):
    c, scl, st, torch = env
    out = torch.zeros(48, dtype=torch.uint8, device="cuda")
    with pytest.raises(scl.SclError) as e:
        scl.scl_map_reduce_noalloc(out.data_ptr(), scl.SCL_U32, scl.SCL_NOALLOC_MAX_ELEMENTS + 1,
                                   scl.SCL_K_MIX32, scl.SCL_R_SUM, out.data_ptr(), stream=st)
    assert e.value.status == scl.SCL_E_INVALID
    assert "at most" in str(e.value)
