"""Every compiled launch shape and path against the oracle and each other.

The TMA bulk-copy pipeline (path 1) must give results bit-identical to the
vector-load kernel (path 0) of the same (block, items_per_thread): same
segment geometry, same per-thread element mapping, same reduction order.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_common import check_f32_result
from paper_1505_01120_gb300 import synth

pytestmark = pytest.mark.gpu

LDG_SHAPES = [(256, 2), (256, 4), (256, 8), (512, 2), (512, 4), (512, 8)]
TMA_SHAPES = [(256, 2, 12), (256, 4, 6), (256, 4, 4), (256, 8, 3), (512, 2, 6), (512, 4, 3)]
SIZES = [0, 1, 5, 1023, 4096, 4097, 16_384 * 3 + 5, 262_147, 2_000_003, 9_000_001]


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1505_01120_gb300 import scl
    from paper_1505_01120_gb300.context import Context, current_stream
    torch.cuda.set_device(0)
    c = Context(2 << 30, device=0)
    rng = np.random.default_rng(500)
    data = {n: (rng.integers(0, 1 << 32, size=n, dtype=np.uint32),
                rng.standard_normal(n, dtype=np.float32)) for n in SIZES}
    parts = {n: (scl.scl_load_partition(c.handle, a, scl.SCL_U32, stream=current_stream(0)),
                 scl.scl_load_partition(c.handle, x, scl.SCL_F32, stream=current_stream(0)))
             for n, (a, x) in data.items()}
    yield c, scl, current_stream(0), torch, data, parts
    c.close()


def run_all(c, scl, st, data, parts):
    out = {}
    for n in SIZES:
        pu, pf = parts[n]
        ru = scl.scl_map_reduce(c.handle, pu, scl.SCL_K_MIX32, scl.SCL_R_SUM, stream=st)
        rf = scl.scl_map_reduce(c.handle, pf, scl.SCL_K_POLY3, scl.SCL_R_SUM_MIN_MAX, stream=st)
        out[n] = (ru.u64_sum, rf.f64_sum, rf.f32_min, rf.f32_max)
        assert ru.u64_sum == oracle.sum_u32(data[n][0], mix=True), n
        check_f32_result(rf, data[n][1], True)
    return out


@pytest.mark.parametrize("block,ipt", LDG_SHAPES)
def test_ldg_shapes(env, block, ipt):
    c, scl, st, torch, data, parts = env
    for fam in (scl.SCL_FAMILY_U32, scl.SCL_FAMILY_F32):
        scl.scl_set_shape(c.handle, fam, block, ipt, path=0)
    run_all(c, scl, st, data, parts)


@pytest.mark.parametrize("block,ipt,stages", TMA_SHAPES)
def test_tma_shapes_match_ldg_bitwise(env, block, ipt, stages):
    c, scl, st, torch, data, parts = env
    for fam in (scl.SCL_FAMILY_U32, scl.SCL_FAMILY_F32):
        scl.scl_set_shape(c.handle, fam, block, ipt, path=0)
    ref = run_all(c, scl, st, data, parts)
    for fam in (scl.SCL_FAMILY_U32, scl.SCL_FAMILY_F32):
        scl.scl_set_shape(c.handle, fam, block, ipt, path=1, stages=stages)
        assert scl.scl_get_shape(c.handle, fam)["path"] == 1
    got = run_all(c, scl, st, data, parts)
    for n in SIZES:
        assert got[n][0] == ref[n][0]
        assert np.float64(got[n][1]).tobytes() == np.float64(ref[n][1]).tobytes(), n
        assert got[n][2] == ref[n][2] and got[n][3] == ref[n][3]


def test_tma_unaligned_and_batches(env):
    c, scl, st, torch, data, parts = env
    for fam in (scl.SCL_FAMILY_U32, scl.SCL_FAMILY_F32):
        scl.scl_set_shape(c.handle, fam, 256, 4, path=1, stages=6)
    a, x = data[2_000_003]
    dx = torch.from_numpy(x).cuda()
    torch.cuda.synchronize()
    for off in (1, 3):
        q = scl.scl_wrap_device(c.handle, dx.data_ptr() + 4 * off, None, scl.SCL_F32,
                                x.size - off)
        r = scl.scl_map_reduce(c.handle, q, scl.SCL_K_POLY3, scl.SCL_R_SUM_MIN_MAX, stream=st)
        check_f32_result(r, x[off:], True)
    # homogeneous fp32 and uint32 batches on the TMA path, replayed from a graph
    for kind in (synth.KIND_POLY3, synth.KIND_MIX32):
        specs = [synth.TaskSpec(kind, n, 900 + i)
                 for i, n in enumerate([0, 3, 4096, 70_001, 1_000_000, 4_194_304])]
        ds, tasks = [], []
        for s in specs:
            d = synth.task_data(s)[0]
            ds.append(d)
            dt = scl.SCL_F32 if kind == synth.KIND_POLY3 else scl.SCL_U32
            p = scl.scl_load_partition(c.handle, d, dt, stream=st)
            tasks.append(dict(part=p, kernel=scl.SCL_K_POLY3 if kind == synth.KIND_POLY3
                              else scl.SCL_K_MIX32,
                              reduce=scl.SCL_R_SUM_MIN_MAX if kind == synth.KIND_POLY3
                              else scl.SCL_R_SUM))
        b = scl.scl_batch_create(c.handle, scl.make_tasks(tasks), len(tasks))
        s2 = torch.cuda.Stream()
        scl.scl_batch_capture(b, s2.cuda_stream)
        for _ in range(3):
            scl.scl_batch_launch(b, s2.cuda_stream)
            res = scl.scl_batch_results(b, len(tasks), stream=s2.cuda_stream)
            for i, d in enumerate(ds):
                if kind == synth.KIND_MIX32:
                    assert int(res[i]["u64_sum"]) == oracle.sum_u32(d, mix=True)
                else:
                    rr = scl.scl_result()
                    for k in ("u64_sum", "f64_sum", "f32_min", "f32_max", "status", "n"):
                        setattr(rr, k, res[i][k].item())
                    check_f32_result(rr, d, True)
        scl.scl_batch_destroy(b)
    for fam in (scl.SCL_FAMILY_U32, scl.SCL_FAMILY_F32):
        scl.scl_set_shape(c.handle, fam, 256, 4, path=0)


def test_unsupported_shapes_rejected(env):
    c, scl, *_ = env
    with pytest.raises(scl.SclError) as e:
        scl.scl_set_shape(c.handle, scl.SCL_FAMILY_F32, 384, 4)
    assert e.value.status == scl.SCL_E_UNSUPPORTED
    with pytest.raises(scl.SclError) as e:
        scl.scl_set_shape(c.handle, scl.SCL_FAMILY_KEYED, 256, 4, path=1)
    assert e.value.status == scl.SCL_E_UNSUPPORTED
