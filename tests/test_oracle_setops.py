"""Pins of the oracle's merge-based set operations (multiset semantics).

The oracle walks both inputs with two pointers; these pins check it against
things fixed independently of that walk:
  * a brute force by counting: for every distinct key, its m copies in A
    and n copies in B give the expected copies directly (union: A's m, then
    B's copies after the m-th; intersection: A's first min(m, n); difference:
    A's copies after the n-th; symmetric difference: both of the latter);
  * numpy's set routines on duplicate-free inputs (the textbook special case);
  * the cardinality identities |U| + |I| = |A| + |B|, |D| = |A| - |I|,
    |S| = |U| - |I| on multisets;
  * a small example worked by hand.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from _util import random_sorted

DTYPES = [np.int32, np.uint32, np.float32, np.uint64, np.int64]
OPS = list(oracle.SET_OPS)


def counting_expect(op, a, b, av, bv):
    """Expected (keys, values) of set operation op by per-key counting."""
    # Keys as (value, sign) so that -0.0 and +0.0 stay distinct and ordered.
    def key(x):
        return (x, math.copysign(1.0, x)) if isinstance(x, float) else (x, 0)
    ka, kb = [key(x) for x in a.tolist()], [key(x) for x in b.tolist()]
    keys = sorted(set(ka) | set(kb))
    out_k, out_v = [], []
    for v in keys:
        la = [int(av[i]) for i, x in enumerate(ka) if x == v]
        lb = [int(bv[j]) for j, x in enumerate(kb) if x == v]
        m, n = len(la), len(lb)
        if op == "union":
            pick = la + lb[m:]
        elif op == "intersection":
            pick = la[:min(m, n)]
        elif op == "difference":
            pick = la[n:]
        else:
            pick = la[n:] + lb[m:]
        out_k += [v[0]] * len(pick)
        out_v += pick
    return out_k, out_v


def _sorted_multisets(alphabet, max_len):
    for n in range(max_len + 1):
        for combo in itertools.combinations_with_replacement(alphabet, n):
            yield np.array(combo, dtype=np.int32)


def test_set_ops_exhaustive_tiny_vs_counting():
    seqs = list(_sorted_multisets([0, 1, 2], 4))
    for a in seqs:
        for b in seqs:
            av = np.arange(a.size, dtype=np.uint32)
            bv = np.arange(100, 100 + b.size, dtype=np.uint32)
            for op in OPS:
                k, v = oracle.set_op(op, a, b, av, bv)
                ek, ev = counting_expect(op, a, b, av, bv)
                assert k.tolist() == ek and v.tolist() == ev, (op, a, b)


@pytest.mark.parametrize("dtype", DTYPES, ids=lambda d: np.dtype(d).name)
def test_set_ops_random_vs_counting(dtype):
    rng = np.random.default_rng(61)
    for na, nb in [(0, 9), (9, 0), (40, 55), (300, 200)]:
        a = random_sorted(rng, dtype, na, "ties")
        b = random_sorted(rng, dtype, nb, "ties")
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        for op in OPS:
            k, v = oracle.set_op(op, a, b, av, bv)
            ek, ev = counting_expect(op, a, b, av, bv)
            assert v.tolist() == ev, (op, na, nb)  # values identify each element exactly
            assert np.array_equal(k, np.array(ek, dtype=dtype)), (op, na, nb)


@pytest.mark.parametrize("dtype", [np.int32, np.uint32, np.uint64, np.int64, np.float32],
                         ids=lambda d: np.dtype(d).name)
def test_set_ops_sets_vs_numpy(dtype):
    """Duplicate-free inputs: the ordinary set operations (numpy treats -0.0
    and +0.0 as one value, so float inputs avoid zeros)."""
    rng = np.random.default_rng(62)
    lib = {"union": np.union1d, "intersection": np.intersect1d,
           "difference": np.setdiff1d, "symmetric_difference": np.setxor1d}
    for na, nb in [(0, 50), (50, 0), (1000, 1500), (20_000, 7_000)]:
        pool = np.unique(random_sorted(rng, dtype, 4 * (na + nb) + 10, "ties"))
        if dtype == np.float32:
            pool = pool[pool != 0]
        a = np.sort(rng.choice(pool, min(na, pool.size), replace=False)).astype(dtype)
        b = np.sort(rng.choice(pool, min(nb, pool.size), replace=False)).astype(dtype)
        for op in OPS:
            k, _ = oracle.set_op(op, a, b)
            assert np.array_equal(k, lib[op](a, b)), (op, na, nb)


def test_set_ops_cardinality_identities():
    rng = np.random.default_rng(63)
    for _ in range(30):
        na, nb = int(rng.integers(0, 400)), int(rng.integers(0, 400))
        a = np.sort(rng.integers(0, 40, na)).astype(np.int64)
        b = np.sort(rng.integers(0, 40, nb)).astype(np.int64)
        u, i, d, s = (oracle.set_op(op, a, b)[0].size for op in OPS)
        assert u + i == na + nb
        assert d == na - i
        assert s == u - i
        assert oracle.set_op("difference", b, a)[0].size == nb - i


def test_set_ops_hand_example():
    """A = {1, 2, 2, 2, 5, 7}, B = {2, 2, 3, 5, 5, 8} worked by hand: key 2 is
    in A three times and in B twice, key 5 once and twice."""
    a = np.array([1, 2, 2, 2, 5, 7], np.int32)
    b = np.array([2, 2, 3, 5, 5, 8], np.int32)
    av = np.arange(6, dtype=np.uint32)
    bv = np.arange(10, 16, dtype=np.uint32)
    expect = {
        "union": ([1, 2, 2, 2, 3, 5, 5, 7, 8], [0, 1, 2, 3, 12, 4, 14, 5, 15]),
        "intersection": ([2, 2, 5], [1, 2, 4]),
        "difference": ([1, 2, 7], [0, 3, 5]),
        "symmetric_difference": ([1, 2, 3, 5, 7, 8], [0, 3, 12, 14, 5, 15]),
    }
    for op, (ek, ev) in expect.items():
        k, v = oracle.set_op(op, a, b, av, bv)
        assert k.tolist() == ek and v.tolist() == ev, op
