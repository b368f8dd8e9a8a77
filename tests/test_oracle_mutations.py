"""The oracle's pins catch plausible mistakes planted in the oracle.

Each case copies the oracle's C source, plants one mistake (a flipped
tie-break, a transposed operand, a dropped term), compiles the copy on the
CPU and checks that at least one pin from test_oracle_pins fails on it.
Mistakes are chosen so that the mutated code still stays inside its arrays.
"""
import os

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins
import test_oracle_setops as setpins
import test_oracle_wide as widepins

# (name, text in mp_oracle.c, replacement)
MUTATIONS = [
    ("merge ties take B",
     "else take_b = gt_##SFX(a[i], b[j]);",
     "else take_b = !gt_##SFX(b[j], a[i]);"),
    ("merge compares the wrong way round",
     "else take_b = gt_##SFX(a[i], b[j]);",
     "else take_b = gt_##SFX(b[j], a[i]);"),
    ("float order drops the sign of zero",
     "if (x == y && x == 0.0f) return !signbit(x) && signbit(y);",
     "if (x == y && x == 0.0f) return 0;"),
    ("float order flips the sign of zero",
     "if (x == y && x == 0.0f) return !signbit(x) && signbit(y);",
     "if (x == y && x == 0.0f) return signbit(x) && !signbit(y);"),
    ("split accepts with a strict lower test",
     "int lower_ok = (a_i <= 0) || (b_i >= nb) || !gt_##SFX(a[a_i - 1], b[b_i]);",
     "int lower_ok = (a_i <= 0) || (b_i >= nb) || gt_##SFX(b[b_i], a[a_i - 1]);"),
    ("split drops the upper test",
     "int upper_ok = (a_i >= na) || (b_i <= 0) || gt_##SFX(a[a_i], b[b_i - 1]);",
     "int upper_ok = 1;"),
    ("sort merges the right run as A",
     """oracle_merge_##SFX(src + lo, srcv ? srcv + lo : NULL, mid - lo,          \\
                               src + mid, srcv ? srcv + mid : NULL, hi - mid,        \\""",
     """oracle_merge_##SFX(src + mid, srcv ? srcv + mid : NULL, hi - mid,        \\
                               src + lo, srcv ? srcv + lo : NULL, mid - lo,        \\"""),
    ("batched writes segments at the A offset only",
     "int64_t c = a_off[s] + b_off[s];",
     "int64_t c = a_off[s] + b_off[s] - (s > 0 && b_off[s] > 0 ? 1 : 0);"),
    ("set op: symmetric difference keeps matched pairs",
     "const int keep_pair = (op == 0 || op == 1);",
     "const int keep_pair = (op == 0 || op == 1 || op == 3);"),
    ("set op: equal heads treated as B smaller",
     "if (gt_##SFX(a[i], b[j])) {          /* B's head is smaller */",
     "if (!gt_##SFX(b[j], a[i])) {          /* B's head is smaller */"),
    ("set op: a matched pair advances A only",
     """            i++;                                                                     \\
            j++;                                                                     \\
        }                                                                            \\
    }                                                                                \\
    for (; i < na; i++)""",
     """            i++;                                                                     \\
        }                                                                            \\
    }                                                                                \\
    for (; i < na; i++)"""),
    ("128-bit keys compared on the low word only",
     "static int gt_u128(unsigned __int128 x, unsigned __int128 y) { return x > y; }",
     "static int gt_u128(unsigned __int128 x, unsigned __int128 y) { return (uint64_t)x > (uint64_t)y; }"),
    ("signed 128-bit keys compared without their sign",
     "static int gt_i128(__int128 x, __int128 y) { return x > y; }",
     "static int gt_i128(__int128 x, __int128 y) { return (unsigned __int128)x > (unsigned __int128)y; }"),
    ("set op: difference keeps B's leftovers",
     "const int keep_b_alone = (op == 0 || op == 3);",
     "const int keep_b_alone = (op == 0 || op == 2 || op == 3);"),
    ("merge stops when either side runs out",
     "while (i < na || j < nb) {",
     "while (i < na && j < nb) {"),
    ("sort stops one round early",
     "for (int64_t w = 1; w < n; w *= 2) {",
     "for (int64_t w = 1; 2 * w < n; w *= 2) {"),
    ("sort drops the second run of a ragged tail",
     "int64_t hi = lo + 2 * w < n ? lo + 2 * w : n;",
     "int64_t hi = lo + 2 * w < n ? lo + 2 * w : mid;"),
]

PINS = [
    pins.test_golden_alg2_bounds,
    pins.test_golden_adversarial_all_a_greater_than_b,
    pins.test_golden_f32_total_order,
    pins.test_merge_and_split_exhaustive_tiny,
    pins.test_closed_form_distinct16_groups,
    pins.test_sort_special_orders,
    pins.test_merge_batched_vs_brute_force,
    setpins.test_set_ops_hand_example,
    setpins.test_set_ops_cardinality_identities,
    setpins.test_set_ops_exhaustive_tiny_vs_counting,
    lambda: widepins.test_wide_merge_split_exhaustive_tiny("u128"),
    lambda: widepins.test_wide_merge_split_exhaustive_tiny("i128"),
]
PINS_DTYPE = [
    pins.test_closed_form_all_equal,
    pins.test_closed_form_all_a_greater,
    pins.test_merge_random_vs_library_stable_sort,
    pins.test_split_invariants,
    pins.test_sort_vs_brute_force,
]


def _caught(lib, monkeypatch):
    """Name of the first pin that fails on ``lib`` (an assertion, or the
    oracle reporting a failed search), else None."""
    monkeypatch.setattr(oracle, "_lib", lib)
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError):
            return pin.__name__
    for pin in PINS_DTYPE:
        for dt in pins.DTYPES:
            try:
                pin(dt)
            except (AssertionError, ValueError):
                return f"{pin.__name__}[{np.dtype(dt).name}]"
    return None


def test_source_has_every_mutation_site():
    with open(oracle._SRC) as f:
        src = f.read()
    for name, old, _ in MUTATIONS:
        assert src.count(old) == 1, name


@pytest.mark.parametrize("idx", range(len(MUTATIONS)), ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(idx, tmp_path, monkeypatch):
    name, old, new = MUTATIONS[idx]
    with open(oracle._SRC) as f:
        src = f.read()
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.load_library(oracle.compile_source(str(mutated), str(tmp_path / "mutant.so")))
    assert _caught(lib, monkeypatch) is not None, f"no pin caught: {name}"
