"""The allocation-free map+reduce entry point against the oracle.

scl_map_reduce_noalloc is for callers that cannot allocate device memory when
they need a result: plug-ins inside a host application whose own pool holds
all of the GPU's memory, and paths that cannot take the device
synchronisation of cudaMalloc/cudaFree.  It keeps its scratch in a fixed
device array inside the library.  Every result is checked against the CPU
oracle (integer sums bit-exact, fp32 sums within the fp32 tolerance with the
real sum of |y|, min/max exact), on two calls in a row that share that array.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process, where
its first call does the per-device set-up.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_common import check_f32_result

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1505_01120_gb300 import scl
    from paper_1505_01120_gb300.context import current_stream
    torch.cuda.set_device(0)
    yield scl, current_stream(0), torch


CASES = [
    ("u32", 1, 0), ("u32", 1, 1_000_003), ("u32", 0, 4097),
    ("f32", 2, 3), ("f32", 2, 2_500_001), ("f32", 0, 65_537),
    ("u32", 1, 67_108_864), ("f32", 2, 67_108_864 - 5),
]


class _R:
    """Field access for check_f32_result."""
    def __init__(self, rec):
        for k in ("u64_sum", "f64_sum", "f32_min", "f32_max", "n", "status"):
            setattr(self, k, rec[k].item())


@pytest.mark.parametrize("kind,kernel,n", CASES)
def test_noalloc_matches_oracle_twice(env, kind, kernel, n):
    scl, st, torch = env
    rng = np.random.default_rng(n + kernel)
    if kind == "u32":
        host = rng.integers(0, 1 << 32, size=n, dtype=np.uint32)
        dtype, reduce = scl.SCL_U32, scl.SCL_R_SUM
        dev = torch.from_numpy(host.view(np.int32)).cuda()
        want = oracle.sum_u32(host, mix=kernel == scl.SCL_K_MIX32)
    else:
        host = rng.standard_normal(n, dtype=np.float32)
        dtype, reduce = scl.SCL_F32, scl.SCL_R_SUM_MIN_MAX
        dev = torch.from_numpy(host).cuda()
    out = torch.zeros(3 * 48, dtype=torch.uint8, device="cuda")
    # a first call (per-device set-up on a fresh process), then two calls in a
    # row during which the device's free memory must not change
    scl.scl_map_reduce_noalloc(dev.data_ptr(), dtype, n, kernel, reduce, out.data_ptr(), stream=st)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for i in (1, 2):
        scl.scl_map_reduce_noalloc(dev.data_ptr(), dtype, n, kernel, reduce,
                                   out.data_ptr() + 48 * i, stream=st)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    res = out.cpu().numpy().view(scl.RESULT_DTYPE)
    for rec in res:
        r = _R(rec)
        if kind == "u32":
            assert r.n == n and r.status == 0
            assert r.u64_sum == want
        else:
            check_f32_result(r, host, poly=kernel == scl.SCL_K_POLY3)


def test_noalloc_rejects_oversized_partitions(env):
    scl, st, torch = env
    out = torch.zeros(48, dtype=torch.uint8, device="cuda")
    with pytest.raises(scl.SclError) as e:
        scl.scl_map_reduce_noalloc(out.data_ptr(), scl.SCL_U32, scl.SCL_NOALLOC_MAX_ELEMENTS + 1,
                                   scl.SCL_K_MIX32, scl.SCL_R_SUM, out.data_ptr(), stream=st)
    assert e.value.status == scl.SCL_E_INVALID
    assert "at most" in str(e.value)
