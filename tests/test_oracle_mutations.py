"""Each plausible mistake planted in a copy of oracle.c must fail a pin.

The copies are compiled into a temporary directory and loaded beside the real
oracle; the real ``oracle.c`` is never modified.  This shows the pins in
``test_oracle_pins.py`` are sensitive to dropped terms, wrong signs, wrong
constants or shifts, wrong indices and a separately rounded product where the
reading fixes a fused multiply-add.
"""
from __future__ import annotations

import os

import pytest

import oracle
from test_oracle_pins import PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# (name, text in oracle.c, replacement, pins of which at least one must fail)
MUTATIONS = [
    ("wrong_mix_constant", "x *= 0x846ca68bu;", "x *= 0x846ca68du;",
     ["mix32_left_inverse"]),
    ("wrong_mix_shift", "x ^= x >> 15;", "x ^= x >> 14;",
     ["mix32_left_inverse"]),
    ("mix_steps_swapped", "x *= 0x7feb352du;\n    x ^= x >> 15;",
     "x ^= x >> 15;\n    x *= 0x7feb352du;", ["mix32_left_inverse"]),
    ("even_mix_constant", "x *= 0x7feb352du;", "x *= 0x7feb352eu;",
     ["mix32_full_domain_sum", "mix32_left_inverse"]),
    ("u32_sum_truncated", "s += (uint64_t)v;", "s = (uint32_t)(s + v);",
     ["sum_u32_brute_force", "mix32_full_domain_sum"]),
    ("sum_drops_last", "for (uint64_t i = 0; i < n; ++i) {\n        uint32_t v",
     "for (uint64_t i = 0; i + 1 < n; ++i) {\n        uint32_t v",
     ["sum_u32_brute_force"]),
    ("unfused_first_fma", "float t = fmaf(a, x2, b);", "float t = a * x2 + b;",
     ["poly3_exact_rounding"]),
    ("unfused_second_fma", "return fmaf(t, x, c);", "return t * x + c;",
     ["poly3_exact_rounding"]),
    ("poly_sign_flip", "float t = fmaf(a, x2, b);", "float t = fmaf(a, x2, -b);",
     ["poly3_moments", "poly3_exact_rounding"]),
    ("poly_drops_constant", "return fmaf(t, x, c);", "return t * x;",
     ["poly3_moments", "reduce_constant_partitions"]),
    ("poly_wrong_power", "float x2 = x * x;", "float x2 = x;",
     ["poly3_moments", "poly3_odd_symmetry", "poly3_exact_rounding"]),
    ("f32_sum_in_float", "double s = 0.0;\n    float lo", "float s = 0.0f;\n    float lo",
     ["reduce_f32_against_numpy", "reduce_constant_partitions"]),
    ("max_compares_wrong_way", "if (y > hi) hi = y;", "if (y < hi) hi = y;",
     ["reduce_f32_against_numpy", "reduce_constant_partitions"]),
    ("min_propagates_nan", "if (y == y) {             /* NaN never becomes the min or the max */\n            if (y < lo) lo = y;",
     "if (1) {\n            if (!(y >= lo)) lo = y;",
     ["reduce_edge_cases"]),
    ("keyed_value_off_by_one", "sum[k] += (double)vals[i];",
     "sum[k] += (double)vals[i ? i - 1 : 0];", ["keyed_against_bincount"]),
    ("keyed_accepts_last_bad_key", "(uint32_t)k >= num_keys", "(uint32_t)k > num_keys",
     ["keyed_special_cases"]),
    ("hash_bucket_by_low_bits", "uint32_t b = (uint32_t)(((uint64_t)h * num_keys) >> 32);",
     "uint32_t b = h % num_keys;", ["keyed_hashed"]),
    ("hash_bucket_unmixed", "uint32_t h = orc_mix32((uint32_t)keys[i]);",
     "uint32_t h = (uint32_t)keys[i];", ["keyed_hashed"]),
    ("tree_as_left_fold", "while (top >= 2 && size[top - 2] == size[top - 1]) {",
     "while (top >= 2) {", ["add_arrays", "add_arrays_tree_shape"]),
    ("tree_final_fold_oldest_first",
     "float acc = stack[top - 1];\n    for (uint32_t i = top - 1; i-- > 0;)\n        acc = stack[i] + acc;",
     "float acc = stack[0];\n    for (uint32_t i = 1; i < top; ++i)\n        acc = acc + stack[i];",
     ["add_arrays_tree_shape"]),
    ("add_drops_last_array", "for (uint32_t j = 0; j < k; ++j)\n            col[j] = arrays[j][i];\n        out[i] = tree_sum_f32(col, k);",
     "for (uint32_t j = 0; j < k; ++j)\n            col[j] = arrays[j][i];\n        out[i] = tree_sum_f32(col, k - 1);",
     ["add_arrays"]),
    ("u32_add_drops_array", "for (uint32_t j = 0; j < k; ++j)\n            s += arrays[j][i];",
     "for (uint32_t j = 1; j < k; ++j)\n            s += arrays[j][i];", ["add_arrays"]),
    ("combine_first_only", "us += u64_sums[i];", "us += u64_sums[0];",
     ["combine_equals_whole"]),
    ("combine_keyed_transposed", "c += counts[(uint64_t)i * num_keys + j];",
     "c += counts[(uint64_t)j * k + i];", ["combine_equals_whole"]),
]


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new, pins):
    text = open(SRC).read()
    assert text.count(old) == 1, "mutation anchor must occur exactly once: " + old
    src = tmp_path / "oracle_mut.c"
    src.write_text(text.replace(old, new))
    lib = oracle.load(oracle.build(str(src), str(tmp_path / "liboracle_mut.so")))
    caught = []
    for p in pins:
        try:
            PINS[p](lib)
        except (AssertionError, ValueError, OverflowError):
            caught.append(p)
    assert caught, "planted mistake %s passed every pin %s" % (name, pins)
