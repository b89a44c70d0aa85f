"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/scl.h declares, its structs have the declared layout, and its host-only
calls (status text, the ReduceCL combine across partitions) agree with the
oracle.  No GPU compute is called here."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions() -> set[str]:
    names = set()
    for h in os.listdir(HEADER_DIR):
        if h.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(scl_\w+)\s*\(", text, re.M))
    return names


@pytest.fixture(scope="module")
def scl():
    from paper_1505_01120_gb300 import build
    build.build()
    from paper_1505_01120_gb300 import scl as mod
    return mod


def test_library_exports_every_declared_symbol(scl):
    decl = declared_functions()
    assert len(decl) >= 25
    out = subprocess.run(["nm", "-D", "--defined-only", scl._LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(scl_\w+)", out))
    missing = decl - exported
    assert not missing, "declared in include/*.h but not exported: %s" % sorted(missing)
    for name in decl:
        assert hasattr(scl.lib, name)
    # the binding wraps every declared function
    assert decl <= set(scl.exported_symbols()) | {"scl_server_stop"} | \
        {n for n in decl if n.startswith("scl_server") or n.startswith("scl_tune")}


def test_struct_layouts_match_header(scl):
    assert ctypes.sizeof(scl.scl_result) == 48
    assert ctypes.sizeof(scl.scl_task) == 64
    assert scl.scl_result.f64_sum.offset == 8 and scl.scl_result.n.offset == 32
    assert scl.scl_task.coef.offset == 20 and scl.scl_task.counts_out.offset == 32
    assert scl.scl_abi_version() == 1
    assert ctypes.sizeof(scl.scl_devserver_config) == 48
    assert ctypes.sizeof(scl.scl_devserver_stats) == 112
    assert scl.scl_devserver_stats.grid.offset == 72


def test_status_text(scl):
    assert scl._strerror(scl.SCL_OK) == "ok"
    assert "key" in scl._strerror(scl.SCL_E_KEY_RANGE)
    assert scl._strerror(12345) == "unknown status"


def _res(scl, u=0, f=0.0, mn=np.inf, mx=-np.inf, n=0, status=0):
    r = scl.scl_result()
    r.u64_sum, r.f64_sum, r.f32_min, r.f32_max, r.n, r.status = u, f, mn, mx, n, status
    return r


def test_combine_matches_oracle_fold(scl):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(100_000, dtype=np.float32)
    u = rng.integers(0, 1 << 32, size=100_000, dtype=np.uint32)
    cuts = np.sort(rng.integers(0, x.size, size=40))
    parts, us = [], []
    for xs, uu in zip(np.split(x, cuts), np.split(u, cuts)):
        s, mn, mx = oracle.reduce_f32(xs, True)
        us.append(oracle.sum_u32(uu))
        parts.append(_res(scl, us[-1], s, mn, mx, xs.size))
    r = scl.scl_combine(parts)
    uo, fo, mno, mxo = oracle.combine(us, [p.f64_sum for p in parts],
                                      [p.f32_min for p in parts], [p.f32_max for p in parts])
    assert r.u64_sum == uo and r.n == x.size
    assert r.f32_min == mno and r.f32_max == mxo
    assert abs(r.f64_sum - fo) <= 1e-12 * float(np.abs(oracle.map_poly3(x)).sum())


def test_combine_empty_and_status(scl):
    r = scl.scl_combine([])
    assert r.u64_sum == 0 and r.f64_sum == 0.0 and r.f32_min == np.inf and r.f32_max == -np.inf
    r = scl.scl_combine([_res(scl, 1), _res(scl, 2, status=scl.SCL_E_KEY_RANGE), _res(scl, 3)])
    assert r.u64_sum == 6 and r.status == scl.SCL_E_KEY_RANGE
    r = scl.scl_combine([_res(scl, mn=np.nan, mx=np.nan), _res(scl, mn=-1.0, mx=2.0)])
    assert r.f32_min == -1.0 and r.f32_max == 2.0


def test_combine_keyed_matches_oracle(scl):
    rng = np.random.default_rng(4)
    counts = rng.integers(0, 1000, size=(13, 4096)).astype(np.uint32)
    sums = rng.random((13, 4096))
    co, so = scl.scl_combine_keyed(counts, sums)
    oc, os_ = oracle.combine_keyed(counts, sums)
    assert np.array_equal(co, oc)
    assert np.allclose(so, os_, rtol=1e-13, atol=0)


def test_create_without_device_fails_cleanly(scl):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(scl.SclError) as e:
        scl.scl_create(0, 1 << 20, 1 << 20)
    assert e.value.status in (scl.SCL_E_CUDA, scl.SCL_E_INVALID)
