"""Pins of the CPU oracle to facts other than itself (no GPU needed).

Each ``pin_*`` function checks the oracle build ``lib`` against something the
SparkCL workloads and the mathematics fix: an inverse built by inverting each
mix32 step, the closed-form sum of a bijection over its whole domain, exact
rational evaluation with IEEE round-to-nearest-even, moments of N(0,1),
numpy's bincount / min / max / fsum, odd symmetry, constant partitions and
brute force on tiny inputs.  ``test_oracle_mutations.py`` runs the same pins
against deliberately broken copies of ``oracle.c`` to show each pin catches
the mistake it is meant to catch.
"""
from __future__ import annotations

import math
import threading
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1505_01120_gb300 import synth

U32 = (1 << 32) - 1


# ------------------------------------------------------------------ helpers

def unmix32(y: np.ndarray) -> np.ndarray:
    """Inverse of mix32 built from its steps: each xorshift-right is undone by
    iterating x = y ^ (x >> k) to its fixed point, each multiply by an odd
    constant by the multiplicative inverse mod 2^32."""
    c1_inv = pow(0x7feb352d, -1, 1 << 32)
    c2_inv = pow(0x846ca68b, -1, 1 << 32)

    def unxorshift(v, k):
        x = v.copy()
        for _ in range(32 // k + 1):
            x = v ^ (x >> np.uint64(k))
        return x & np.uint64(U32)

    x = y.astype(np.uint64)
    x = unxorshift(x, 16)
    x = (x * np.uint64(c2_inv)) & np.uint64(U32)
    x = unxorshift(x, 15)
    x = (x * np.uint64(c1_inv)) & np.uint64(U32)
    x = unxorshift(x, 16)
    return x.astype(np.uint32)


def round_f32(q: Fraction) -> np.float32:
    """Round an exact rational to binary32, nearest with ties to even."""
    if q == 0:
        return np.float32(0.0)
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    # now 2^e <= a < 2^(e+1)
    e = max(e, -126)                      # subnormals share the 2^-149 grid
    ulp = Fraction(2) ** (e - 23)
    m = a / ulp
    fl = math.floor(m)
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    v = fl * ulp
    if v >= Fraction(2) ** 128:
        return np.float32(sign * np.inf)
    return np.float32(sign * float(v))    # exact: v is a binary32 value


def poly3_exact(x: np.float32, a, b, c) -> np.float32:
    """poly3 with the three roundings of the Horner reading done exactly:
    R(R(a * R(x*x) + b) * x + c), each R a single binary32 rounding."""
    X, A, B, C = (Fraction(float(np.float32(v))) for v in (x, a, b, c))
    x2 = Fraction(float(round_f32(X * X)))
    t = Fraction(float(round_f32(A * x2 + B)))
    return round_f32(t * X + C)


def f32_bits(v) -> int:
    return int(np.asarray(v, dtype=np.float32).view(np.uint32))


# -------------------------------------------------------------------- pins

def pin_mix32_left_inverse(lib):
    rng = np.random.default_rng(11)
    x = np.concatenate([
        np.array([0, 1, 2, 3, 0x7FFFFFFF, 0x80000000, U32, 0x12345678], np.uint32),
        rng.integers(0, 1 << 32, size=200_000, dtype=np.uint32)])
    y = oracle.map_mix32(x, lib=lib)
    assert np.array_equal(unmix32(y), x), "oracle mix32 is not inverted by its stated steps"
    assert oracle.mix32(0, lib=lib) == 0


def pin_mix32_full_domain_sum(lib, threads: int = 8):
    """mix32 is a bijection of uint32, so its sum over all 2^32 inputs is
    sum_{v=0}^{2^32-1} v = 2^31 (2^32 - 1)."""
    step = (1 << 32) // threads
    parts = [0] * threads

    def run(i):
        parts[i] = oracle.mix32_sum_range(i * step, (i + 1) * step, lib=lib)

    ts = [threading.Thread(target=run, args=(i,)) for i in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert sum(parts) % (1 << 64) == (1 << 31) * ((1 << 32) - 1)


def pin_sum_u32_brute_force(lib):
    rng = np.random.default_rng(12)
    for n in (0, 1, 3, 4, 5, 31, 32, 33, 127, 128, 129, 255, 256, 257, 1023, 100_003):
        a = rng.integers(0, 1 << 32, size=n, dtype=np.uint32)
        exact_mix = sum(int(v) for v in oracle.map_mix32(a, lib=lib)) % (1 << 64)
        exact_raw = sum(int(v) for v in a) % (1 << 64)
        assert oracle.sum_u32(a, mix=True, lib=lib) == exact_mix, n
        assert oracle.sum_u32(a, mix=False, lib=lib) == exact_raw, n


def pin_poly3_exact_rounding(lib):
    rng = np.random.default_rng(13)
    coef = (np.float32(0.5), np.float32(-1.25), np.float32(0.1))
    xs = np.concatenate([
        np.array([0.0, 1.0, -1.0, 2.0, -2.0, 0.5, 1e-20, -3e-39, 1e13, -7.25],
                 np.float32),
        rng.standard_normal(3000, dtype=np.float32),
        (rng.standard_normal(1000) * 100).astype(np.float32)])
    got = oracle.map_poly3(xs, coef, lib=lib)
    for x, g in zip(xs, got):
        want = poly3_exact(x, *coef)
        assert f32_bits(g) == f32_bits(want), (float(x), float(g), float(want))
    # a non-default coefficient set goes through the same three roundings
    coef2 = (np.float32(-3.0), np.float32(0.75), np.float32(1e-3))
    got2 = oracle.map_poly3(xs[:500], coef2, lib=lib)
    for x, g in zip(xs[:500], got2):
        assert f32_bits(g) == f32_bits(poly3_exact(x, *coef2)), float(x)


def pin_poly3_moments(lib):
    """Under x ~ N(0,1): E[y] = 0.1, Var[y] = 0.25*15 - 2*0.5*1.25*3 + 1.25^2
    = 1.5625 and E[x (y - 0.1)] = 0.5*3 - 1.25 = 0.25 (E x^2=1, x^4=3, x^6=15).
    Bounds are 5 standard errors (E[(y-0.1)^4] = 253.89, Var[x(y-0.1)] = 12.125)."""
    n = 2_000_000
    x = synth.normal_f32(n, np.random.default_rng(14))
    y = oracle.map_poly3(x, lib=lib).astype(np.float64)
    z = y - 0.1
    assert abs(y.mean() - 0.1) < 5 * 1.25 / math.sqrt(n)
    assert abs(z.var() - 1.5625) < 5 * math.sqrt((253.89 - 1.5625 ** 2) / n)
    assert abs((x.astype(np.float64) * z).mean() - 0.25) < 5 * math.sqrt(12.125 / n)


def pin_poly3_odd_symmetry(lib):
    rng = np.random.default_rng(15)
    x = rng.standard_normal(50_000, dtype=np.float32)
    coef = (0.5, -1.25, 0.0)
    yp = oracle.map_poly3(x, coef, lib=lib)
    yn = oracle.map_poly3(-x, coef, lib=lib)
    assert np.array_equal(yp.view(np.uint32), (-yn).view(np.uint32))
    s, mn, mx = oracle.reduce_f32(np.concatenate([x, -x]), True, coef, lib=lib)
    assert mn == -mx
    # pairs cancel exactly only if summed pairwise; a sequential fp64 sum of
    # 1e5 terms of size ~1 stays within 1e5 * 2^-53 * sum|y|
    bound = 1e5 * 2.0 ** -53 * float(np.abs(yp).astype(np.float64).sum()) * 2
    assert abs(s) <= bound


def pin_reduce_constant_partitions(lib):
    n = 1_000_003
    s, mn, mx = oracle.reduce_f32(np.zeros(n, np.float32), True, lib=lib)
    c = np.float32(0.1)
    assert s == n * float(c)           # k * 0.1f is exact in fp64 for k < 2^29
    assert mn == c and mx == c
    y1 = poly3_exact(np.float32(1.0), 0.5, -1.25, 0.1)
    s, mn, mx = oracle.reduce_f32(np.ones(n, np.float32), True, lib=lib)
    assert f32_bits(mn) == f32_bits(y1) and f32_bits(mx) == f32_bits(y1)
    assert s == n * float(y1)


def pin_reduce_f32_against_numpy(lib):
    rng = np.random.default_rng(16)
    for n in (1, 2, 3, 5, 31, 33, 255, 257, 4099, 300_001):
        x = rng.standard_normal(n, dtype=np.float32)
        for poly in (True, False):
            y = oracle.map_poly3(x, lib=lib) if poly else x
            s, mn, mx = oracle.reduce_f32(x, poly, lib=lib)
            exact = math.fsum(y.astype(np.float64))
            scale = float(np.abs(y).astype(np.float64).sum())
            assert abs(s - exact) <= n * 2.0 ** -52 * scale + 1e-300, (n, poly)
            assert mn == y.min() and mx == y.max(), (n, poly)


def pin_reduce_edge_cases(lib):
    s, mn, mx = oracle.reduce_f32(np.zeros(0, np.float32), True, lib=lib)
    assert s == 0.0 and mn == np.inf and mx == -np.inf
    x = np.array([1.0, np.nan, -2.0, np.nan, 0.5], np.float32)
    s, mn, mx = oracle.reduce_f32(x, False, lib=lib)
    assert math.isnan(s) and mn == -2.0 and mx == 1.0
    assert oracle.sum_u32(np.zeros(0, np.uint32), lib=lib) == 0


def pin_keyed_against_bincount(lib):
    rng = np.random.default_rng(17)
    for n, nk in ((0, 4096), (1, 4096), (257, 17), (100_000, 4096), (33_333, 1)):
        keys = rng.integers(0, nk, size=n, dtype=np.int32)
        vals = rng.random(n, dtype=np.float32)
        cnt, s, bad = oracle.keyed_count_sum(keys, vals, nk, lib=lib)
        assert bad == 0
        assert np.array_equal(cnt, np.bincount(keys, minlength=nk).astype(np.uint32))
        ref = np.bincount(keys, weights=vals.astype(np.float64), minlength=nk)
        assert np.allclose(s, ref, rtol=1e-12, atol=0.0)
        assert int(cnt.sum()) == n
        assert abs(s.sum() - math.fsum(vals.astype(np.float64))) <= 1e-9 * max(1.0, n)


def pin_keyed_special_cases(lib):
    n, nk = 4096 * 37, 4096
    keys = (np.arange(n) % nk).astype(np.int32)
    ones = np.ones(n, np.float32)
    cnt, s, bad = oracle.keyed_count_sum(keys, ones, nk, lib=lib)
    assert bad == 0 and np.all(cnt == 37) and np.array_equal(s, cnt.astype(np.float64))
    # out-of-range keys are skipped and counted; the rest is the histogram of the valid pairs
    rng = np.random.default_rng(18)
    keys = rng.integers(-5, nk + 5, size=20_000, dtype=np.int32)
    vals = rng.random(20_000, dtype=np.float32)
    cnt, s, bad = oracle.keyed_count_sum(keys, vals, nk, lib=lib)
    ok = (keys >= 0) & (keys < nk)
    assert bad == int((~ok).sum())
    assert np.array_equal(cnt, np.bincount(keys[ok], minlength=nk).astype(np.uint32))
    assert np.allclose(s, np.bincount(keys[ok], weights=vals[ok].astype(np.float64),
                                      minlength=nk), rtol=1e-12, atol=0)


def pin_combine_equals_whole(lib):
    rng = np.random.default_rng(19)
    x = rng.standard_normal(200_000, dtype=np.float32)
    u = rng.integers(0, 1 << 32, size=200_000, dtype=np.uint32)
    cuts = np.sort(rng.integers(0, x.size, size=15))
    xs, us = np.split(x, cuts), np.split(u, cuts)
    parts = [oracle.reduce_f32(p, True, lib=lib) for p in xs]
    usum = [oracle.sum_u32(p, lib=lib) for p in us]
    uo, fo, mno, mxo = oracle.combine(usum, [p[0] for p in parts], [p[1] for p in parts],
                                      [p[2] for p in parts], lib=lib)
    s, mn, mx = oracle.reduce_f32(x, True, lib=lib)
    assert uo == oracle.sum_u32(u, lib=lib)
    assert mno == mn and mxo == mx
    assert abs(fo - s) <= 1e-12 * float(np.abs(oracle.map_poly3(x, lib=lib)).sum())
    keys = rng.integers(0, 64, size=x.size, dtype=np.int32)
    tabs = [oracle.keyed_count_sum(k, v, 64, lib=lib) for k, v in
            zip(np.split(keys, cuts), np.split(x, cuts))]
    co, so = oracle.combine_keyed(np.stack([t[0] for t in tabs]),
                                  np.stack([t[1] for t in tabs]), lib=lib)
    cw, sw, _ = oracle.keyed_count_sum(keys, x, 64, lib=lib)
    assert np.array_equal(co, cw)
    assert np.allclose(so, sw, rtol=1e-9, atol=1e-9)


def pin_keyed_hashed(lib):
    """Hashed buckets: for num_keys = 2^m the bucket is the top m bits of mix32
    (multiply-high by a power of two is a shift), with mix32 itself pinned by its
    inverse; for any num_keys, bucket counts/sums equal numpy bincount over the
    buckets computed with Python integers, and every pair is counted."""
    rng = np.random.default_rng(22)
    keys = rng.integers(-2**31, 2**31, size=60_000, dtype=np.int32)
    vals = rng.random(60_000, dtype=np.float32)
    mixed = oracle.map_mix32(keys.view(np.uint32), lib=lib)
    assert np.array_equal(unmix32(mixed), keys.view(np.uint32))
    for m in (0, 1, 6, 12):
        nk = 1 << m
        cnt, s = oracle.keyed_hashed_count_sum(keys, vals, nk, lib=lib)
        b = (mixed >> np.uint32(32 - m)).astype(np.int64) if m else np.zeros(keys.size, np.int64)
        assert np.array_equal(cnt, np.bincount(b, minlength=nk).astype(np.uint32)), m
        assert np.allclose(s, np.bincount(b, weights=vals.astype(np.float64), minlength=nk),
                           rtol=1e-12, atol=0)
    for nk in (3, 1000, 4095):
        cnt, s = oracle.keyed_hashed_count_sum(keys, vals, nk, lib=lib)
        b = np.array([(int(h) * nk) >> 32 for h in mixed], np.int64)
        assert np.array_equal(cnt, np.bincount(b, minlength=nk).astype(np.uint32)), nk
        assert int(cnt.sum()) == keys.size


def pin_add_arrays(lib):
    """The tree reduce of k arrays: k = 1 is the identity; k = 2 is one fp32
    add (numpy's np.add rounds once); k a power of two is the balanced pairwise
    tree, computed level by level by numpy; for any k, arrays of small integers
    (exact in fp32) sum to numpy's exact total; uint32 wraps mod 2^32."""
    rng = np.random.default_rng(21)
    n = 1000
    xs = [rng.standard_normal(n, dtype=np.float32) * (j + 1) for j in range(33)]
    assert np.array_equal(oracle.add_arrays(xs[:1], lib=lib), xs[0])
    assert np.array_equal(oracle.add_arrays(xs[:2], lib=lib).view(np.uint32),
                          np.add(xs[0], xs[1]).view(np.uint32))
    for k in (4, 8, 16, 32):
        lev = np.stack(xs[:k])
        while lev.shape[0] > 1:
            lev = lev[0::2] + lev[1::2]          # fp32 adds, adjacent pairs
        assert np.array_equal(oracle.add_arrays(xs[:k], lib=lib).view(np.uint32),
                              lev[0].view(np.uint32)), k
    for k in (3, 5, 7, 13, 33):
        ints = [rng.integers(-1000, 1000, size=n).astype(np.float32) for _ in range(k)]
        assert np.array_equal(oracle.add_arrays(ints, lib=lib),
                              np.sum(np.stack(ints), axis=0, dtype=np.float64).astype(np.float32))
        got = oracle.add_arrays(xs[:k], lib=lib).astype(np.float64)
        exact = np.array([math.fsum(float(x[i]) for x in xs[:k]) for i in range(n)])
        scale = np.sum(np.abs(np.stack(xs[:k]).astype(np.float64)), axis=0)
        assert np.all(np.abs(got - exact) <= k * 2.0 ** -24 * scale)
    us = [rng.integers(0, 1 << 32, size=n, dtype=np.uint32) for _ in range(9)]
    want = np.array([sum(int(u[i]) for u in us) % (1 << 32) for i in range(n)], np.uint32)
    assert np.array_equal(oracle.add_arrays(us, lib=lib), want)


def pin_add_arrays_tree_shape(lib):
    """Non-power-of-two k: the binary-counter tree for k = 3 is x0 + ... taken
    as (x0 + x1) + x2, and for k = 6 as ((x0+x1)+(x2+x3)) + (x4+x5).  Values are
    chosen so a different association rounds differently."""
    big, one = np.float32(2.0 ** 24), np.float32(1.0)
    a = [np.array([v], np.float32) for v in (big, one, one)]
    # (2^24 + 1) rounds to 2^24, then + 1 rounds to 2^24 again
    assert oracle.add_arrays(a, lib=lib)[0] == big
    b = [np.array([v], np.float32) for v in (one, one, one, one, big, one)]
    # ((1+1)+(1+1)) + (2^24+1) = 4 + 2^24 -> 2^24 + 4
    assert oracle.add_arrays(b, lib=lib)[0] == big + np.float32(4.0)
    zero = np.float32(0.0)
    c = [np.array([v], np.float32) for v in (big, zero, zero, zero, one, zero, one)]
    # k = 7 leaves three subtrees of 4, 2 and 1 leaves: 2^24 + ((1+0) + 1) is
    # 2^24 + 2, while (2^24 + 1) + 1 would round to 2^24 twice
    assert oracle.add_arrays(c, lib=lib)[0] == big + np.float32(2.0)


PINS = {
    "mix32_left_inverse": pin_mix32_left_inverse,
    "mix32_full_domain_sum": pin_mix32_full_domain_sum,
    "sum_u32_brute_force": pin_sum_u32_brute_force,
    "poly3_exact_rounding": pin_poly3_exact_rounding,
    "poly3_moments": pin_poly3_moments,
    "poly3_odd_symmetry": pin_poly3_odd_symmetry,
    "reduce_constant_partitions": pin_reduce_constant_partitions,
    "reduce_f32_against_numpy": pin_reduce_f32_against_numpy,
    "reduce_edge_cases": pin_reduce_edge_cases,
    "keyed_against_bincount": pin_keyed_against_bincount,
    "keyed_special_cases": pin_keyed_special_cases,
    "combine_equals_whole": pin_combine_equals_whole,
    "keyed_hashed": pin_keyed_hashed,
    "add_arrays": pin_add_arrays,
    "add_arrays_tree_shape": pin_add_arrays_tree_shape,
}


@pytest.mark.parametrize("name", sorted(PINS))
def test_oracle_pin(name):
    PINS[name](oracle.load())


def test_round_f32_helper_agrees_with_numpy_on_doubles():
    """The exact rounding helper must agree with numpy's float64->float32 cast
    wherever that cast is a single rounding (inputs that are doubles)."""
    rng = np.random.default_rng(20)
    for v in np.concatenate([rng.standard_normal(2000) * 1e3,
                             rng.standard_normal(200) * 1e-40,
                             [0.1, -0.65, 1.5, 3.4e38, 1e-45]]):
        assert f32_bits(round_f32(Fraction(float(v)))) == f32_bits(np.float32(v)), v


def test_golden_fixtures():
    """Regression vectors written by tests/golden/make_golden.py (oracle only)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_vectors.txt")
    lib = oracle.load()
    seen = 0
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, *fields = line.split()
            if kind == "mix32":
                assert oracle.mix32(int(fields[0], 16), lib=lib) == int(fields[1], 16)
            elif kind == "poly3":
                x = np.uint32(int(fields[0], 16)).view(np.float32)
                assert f32_bits(oracle.poly3(x, lib=lib)) == int(fields[1], 16)
            elif kind == "mix32_sum_range":
                assert oracle.mix32_sum_range(int(fields[0]), int(fields[1]), lib=lib) \
                    == int(fields[2])
            else:
                raise AssertionError("unknown golden record " + kind)
            seen += 1
    assert seen >= 10
