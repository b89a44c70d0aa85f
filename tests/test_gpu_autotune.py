"""The launch-shape autotuner: it times candidates, keeps a valid shape per
family, writes and reloads its cache, and results stay oracle-exact after."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_common import check_f32_result, check_keyed

pytestmark = pytest.mark.gpu


def test_autotune_chooses_valid_shapes_and_persists(tmp_path):
    import torch
    from paper_1505_01120_gb300 import scl
    from paper_1505_01120_gb300.context import Context, current_stream
    torch.cuda.set_device(0)
    cache = str(tmp_path / "tune.txt")
    st = current_stream(0)
    with Context(2 << 30, tune_cache_path=cache) as c:
        rep = scl.scl_autotune(c.handle, st, probe_bytes=64 << 20, reps=3)
        for fam in range(4):
            assert rep[fam]["candidates"] > 0 and rep[fam]["best_ms"] > 0
            got = scl.scl_get_shape(c.handle, fam)
            for k in ("block", "items_per_thread", "ctas_per_sm", "path"):
                assert got[k] == rep[fam][k], (fam, k)
        assert rep[3]["block"] == rep[1]["block"]
        assert rep[3]["items_per_thread"] == rep[1]["items_per_thread"]
        lines = [l for l in open(cache) if not l.startswith("#")]
        assert len(lines) == 4
        # results after tuning
        rng = np.random.default_rng(600)
        a = rng.integers(0, 1 << 32, size=1_234_567, dtype=np.uint32)
        x = rng.standard_normal(3_333_333, dtype=np.float32)
        k = rng.integers(0, 4096, size=2_000_001, dtype=np.int32)
        v = rng.random(2_000_001, dtype=np.float32)
        pa = scl.scl_load_partition(c.handle, a, scl.SCL_U32, stream=st)
        px = scl.scl_load_partition(c.handle, x, scl.SCL_F32, stream=st)
        pk = scl.scl_load_partition_kv(c.handle, k, v, stream=st)
        r = scl.scl_map_reduce(c.handle, pa, scl.SCL_K_MIX32, scl.SCL_R_SUM, stream=st)
        assert r.u64_sum == oracle.sum_u32(a)
        r = scl.scl_map_reduce(c.handle, px, scl.SCL_K_POLY3, scl.SCL_R_SUM_MIN_MAX, stream=st)
        check_f32_result(r, x, True)
        cnt, sums, s64, _ = scl.scl_keyed_reduce(c.handle, pk, 4096, stream=st)
        assert check_keyed(cnt, sums, s64, k, v, 4096) == 0
        shapes = [scl.scl_get_shape(c.handle, f) for f in range(4)]
    with Context(1 << 30, tune_cache_path=cache) as c2:
        assert [scl.scl_get_shape(c2.handle, f) for f in range(4)] == shapes
