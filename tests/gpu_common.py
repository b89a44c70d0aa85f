"""Shared helpers of the GPU tests: one context per test module, tolerances.

Tolerances (fixed by the workload definitions):
  * integer maps, counts and integer sums: bit-exact;
  * fp32 sums: |gpu - oracle| <= 1e-5 * |oracle| against the fp64 oracle, with
    an absolute floor of 1e-6 * sum|y| for tiny partitions whose sum cancels
    (the kernel's own error bound is a few 1e-7 * sum|y|: fp32 within a
    thread's 4*IPT-element chunk, float-float pairs of about 44 bits after);
  * min / max: exact (same fp32 map in the same rounding on both sides).
"""
from __future__ import annotations

import numpy as np

import oracle

REL = 1e-5
ABS_FLOOR = 1e-6


def sum_tol(ref: float, sum_abs: float) -> float:
    return max(REL * abs(ref), ABS_FLOOR * sum_abs)


def check_f32_result(r, x: np.ndarray, poly: bool, coef=oracle.F32_DEFAULT_COEF):
    s, mn, mx = oracle.reduce_f32(x, poly, coef)
    y = oracle.map_poly3(x, coef) if poly else x
    sa = float(np.abs(y.astype(np.float64)).sum()) if y.size else 0.0
    if np.isnan(s):
        assert np.isnan(r.f64_sum)
    else:
        assert abs(r.f64_sum - s) <= sum_tol(s, sa), (r.f64_sum, s, x.size)
    assert np.float32(r.f32_min).tobytes() == np.float32(mn).tobytes() or r.f32_min == mn, \
        (r.f32_min, mn)
    assert np.float32(r.f32_max).tobytes() == np.float32(mx).tobytes() or r.f32_max == mx, \
        (r.f32_max, mx)
    assert r.n == x.size and r.status == 0


def check_keyed(cnt, sums, s64, keys, vals, nk):
    ocnt, osum, bad = oracle.keyed_count_sum(keys, vals, nk)
    assert np.array_equal(cnt, ocnt)
    zero = ocnt == 0
    assert np.all(sums[zero] == 0) and (s64 is None or np.all(s64[zero] == 0))
    nz = ~zero
    if s64 is not None:
        assert np.all(np.abs(s64[nz] - osum[nz]) <= REL * np.abs(osum[nz])), \
            float(np.max(np.abs(s64[nz] - osum[nz]) / np.abs(osum[nz])))
    assert np.all(np.abs(sums[nz].astype(np.float64) - osum[nz]) <= REL * np.abs(osum[nz]))
    return bad


def check_keyed_nonfinite(cnt, sums, s64, keys, vals, nk):
    """check_keyed where some sums are inf or NaN: those must match the
    oracle's (NaN where it has NaN, the same infinity); the finite ones are
    within the fp32 tolerance."""
    ocnt, osum, _ = oracle.keyed_count_sum(keys, vals, nk)
    assert np.array_equal(cnt, ocnt)
    fin = np.isfinite(osum)
    assert np.array_equal(np.isnan(s64), np.isnan(osum))
    assert np.array_equal(np.isinf(s64), np.isinf(osum))
    assert np.array_equal(np.sign(s64[np.isinf(osum)]), np.sign(osum[np.isinf(osum)]))
    nz = fin & (ocnt > 0)
    assert np.all(np.abs(s64[nz] - osum[nz]) <= REL * np.abs(osum[nz]))
    assert np.all(np.abs(sums[nz].astype(np.float64) - osum[nz]) <= REL * np.abs(osum[nz]))

