"""Large-size checks of the CUDA path.

* Closed form, no oracle in the loop: mix32 is a bijection of uint32, so the
  GPU's mix32 + uint64 sum over all 2^32 inputs (four device-built iota
  partitions, folded by the library's ReduceCL combine) is 2^31 (2^32 - 1).
* A single fp32 partition of 2^31 + 7 elements (beyond 32-bit indexing)
  against the oracle.
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
    from paper_1505_01120_gb300.context import Context, current_stream
    torch.cuda.set_device(0)
    c = Context(1 << 30, device=0)
    yield c, scl, current_stream(0), torch
    c.close()


def test_mix32_full_domain_closed_form_on_gpu(env):
    c, scl, st, torch = env
    chunk = 1 << 30
    results = []
    for q in range(4):
        # the 32-bit patterns q*2^30 .. (q+1)*2^30 - 1, built on the device
        lo = q * chunk - (1 << 31)
        iota = torch.arange(lo, lo + chunk, dtype=torch.int64, device="cuda").to(torch.int32)
        p = scl.scl_wrap_device(c.handle, iota.data_ptr(), None, scl.SCL_U32, chunk)
        results.append(scl.scl_map_reduce(c.handle, p, scl.SCL_K_MIX32, scl.SCL_R_SUM, stream=st))
        scl.scl_free_partition(c.handle, p)
        del iota
        torch.cuda.empty_cache()
    total = scl.scl_combine(results)
    assert total.n == 1 << 32
    assert total.u64_sum == (1 << 31) * ((1 << 32) - 1)


def test_partition_beyond_32_bit_indexing(env):
    c, scl, st, torch = env
    n = (1 << 31) + 7
    g = torch.Generator(device="cuda")
    g.manual_seed(9)
    x = torch.randn(n, device="cuda", generator=g)
    p = scl.scl_wrap_device(c.handle, x.data_ptr(), None, scl.SCL_F32, n)
    r = scl.scl_map_reduce(c.handle, p, scl.SCL_K_POLY3, scl.SCL_R_SUM_MIN_MAX, stream=st)
    scl.scl_free_partition(c.handle, p)
    host = x.cpu().numpy()
    del x
    torch.cuda.empty_cache()
    assert r.n == n
    check_f32_result(r, host, True)
