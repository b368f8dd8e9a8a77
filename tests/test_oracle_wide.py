"""Pins of the oracle's 128-bit (multi-word) keys.

Keys are uint64 arrays of shape (n, 2), low word first.  The pins convert
every key to a Python integer (arbitrary precision; two's complement for
i128) and check the oracle's merge, split, sort and set operations against
Python's stable sort and per-key counting, so a dropped word, a swapped word
order or a lost sign fails them.
"""
import itertools

import numpy as np
import pytest

import oracle
from test_oracle_setops import counting_expect

M64 = (1 << 64) - 1


def to_int(row, kind):
    u = int(row[0]) | (int(row[1]) << 64)
    if kind == "i128" and u >= 1 << 127:
        u -= 1 << 128
    return u


def from_ints(xs):
    out = np.empty((len(xs), 2), dtype=np.uint64)
    for i, x in enumerate(xs):
        u = x % (1 << 128)
        out[i, 0] = u & M64
        out[i, 1] = u >> 64
    return out


# Values that differ only in the high word, only in the low word, and (for
# i128) in sign.
ALPHABET = {
    "u128": [0, 1, 1 << 64, (1 << 64) + 1, (1 << 127), (1 << 128) - 1],
    "i128": [-(1 << 127), -(1 << 64), -1, 0, 1, 1 << 64, (1 << 127) - 1],
}


def _ints(keys, kind):
    return [to_int(r, kind) for r in keys]


@pytest.mark.parametrize("kind", ["u128", "i128"])
def test_wide_merge_split_exhaustive_tiny(kind):
    alpha = ALPHABET[kind][:4]
    seqs = [list(c) for n in range(4) for c in itertools.combinations_with_replacement(alpha, n)]
    for xa in seqs:
        for xb in seqs:
            a, b = from_ints(xa), from_ints(xb)
            av = np.arange(len(xa), dtype=np.uint32)
            bv = np.arange(100, 100 + len(xb), dtype=np.uint32)
            k, v = oracle.merge(a, b, av, bv, kind=kind)
            tagged = sorted([(x, int(t)) for x, t in zip(xa, av)] + [(x, int(t)) for x, t in zip(xb, bv)],
                            key=lambda p: p[0])
            assert _ints(k, kind) == [p[0] for p in tagged] and v.tolist() == [p[1] for p in tagged]
            for d in range(len(xa) + len(xb) + 1):
                got, _ = oracle.split(a, b, d, kind=kind)
                assert got == sum(1 for p in tagged[:d] if p[1] < 100), (xa, xb, d)


@pytest.mark.parametrize("kind", ["u128", "i128"])
def test_wide_sort_and_merge_random(kind):
    rng = np.random.default_rng(71)
    alpha = ALPHABET[kind]
    for n in [0, 1, 7, 300, 2000]:
        # keys: alphabet entries plus random offsets in both words
        xs = [int(alpha[rng.integers(len(alpha))]) + int(rng.integers(-3, 4)) * (1 << int(rng.integers(0, 2)) * 64)
              for _ in range(n)]
        lo = -(1 << 127) if kind == "i128" else 0
        xs = [min(max(x, lo), lo + (1 << 128) - 1) for x in xs]
        keys = from_ints(xs)
        vals = np.arange(n, dtype=np.uint32)
        k, v = oracle.sort(keys, vals, kind=kind)
        expect = sorted(zip(xs, range(n)), key=lambda p: p[0])
        assert _ints(k, kind) == [p[0] for p in expect] and v.tolist() == [p[1] for p in expect]
        half = n // 2
        a = from_ints(sorted(xs[:half]))
        b = from_ints(sorted(xs[half:]))
        mk, _ = oracle.merge(a, b, kind=kind)
        assert _ints(mk, kind) == sorted(xs)


@pytest.mark.parametrize("kind", ["u128", "i128"])
def test_wide_set_ops_vs_counting(kind):
    rng = np.random.default_rng(72)
    alpha = ALPHABET[kind]
    for na, nb in [(0, 5), (5, 0), (30, 40), (200, 150)]:
        xa = sorted(int(alpha[i]) for i in rng.integers(0, len(alpha), na))
        xb = sorted(int(alpha[i]) for i in rng.integers(0, len(alpha), nb))
        a, b = from_ints(xa), from_ints(xb)
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        for op in oracle.SET_OPS:
            k, v = oracle.set_op(op, a, b, av, bv, kind=kind)
            ek, ev = counting_expect(op, np.array(xa, dtype=object), np.array(xb, dtype=object), av, bv)
            assert _ints(k, kind) == ek and v.tolist() == ev, (op, na, nb)
