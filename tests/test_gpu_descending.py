"""Descending order (MP_DESCENDING).  The paper assumes ascending order
without loss of generality; the stable descending merge of A and B (ties
keep A first) equals the reversed ascending stable merge of reversed B with
reversed A, and the stable descending sort of x equals the reversed stable
ascending sort of reversed x.  The first test pins those identities against
a brute force on the CPU; the GPU tests use them with the oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1406_2628_gb300 as mp
from _util import first_mismatch, random_sorted, to_dev, to_host, vals_to_dev

DTYPES = [np.int32, np.uint32, np.float32, np.uint64, np.int64]


def desc_merge_expect(a, b, av, bv):
    k, v = oracle.merge(b[::-1].copy(), a[::-1].copy(), bv[::-1].copy(), av[::-1].copy())
    return k[::-1].copy(), v[::-1].copy()


def desc_sort_expect(x, v):
    k, w = oracle.sort(x[::-1].copy(), v[::-1].copy())
    return k[::-1].copy(), w[::-1].copy()


def _order_key(x):
    return (x, math.copysign(1.0, x)) if isinstance(x, float) else (x, 0)


def test_descending_identities_vs_brute_force():
    rng = np.random.default_rng(77)
    for _ in range(200):
        na, nb = int(rng.integers(0, 12)), int(rng.integers(0, 12))
        a = np.sort(rng.integers(0, 4, na).astype(np.int32))[::-1].copy()
        b = np.sort(rng.integers(0, 4, nb).astype(np.int32))[::-1].copy()
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        tagged = [(int(x), int(v)) for x, v in zip(a, av)] + [(int(x), int(v)) for x, v in zip(b, bv)]
        brute = sorted(tagged, key=lambda t: -t[0])  # stable: A before B on ties
        k, v = desc_merge_expect(a, b, av, bv)
        assert [(int(x), int(y)) for x, y in zip(k, v)] == brute
        x = rng.integers(0, 5, na + nb).astype(np.int32)
        xv = np.arange(x.size, dtype=np.uint32)
        brute = sorted(zip(x.tolist(), xv.tolist()), key=lambda t: -t[0])
        k, v = desc_sort_expect(x, xv)
        assert list(zip(k.tolist(), v.tolist())) == brute


@pytest.mark.gpu
@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
def test_descending_merge_and_sort(dt):
    rng = np.random.default_rng(4000 + DTYPES.index(dt))
    for na, nb in [(0, 0), (1, 0), (3, 5), (40_001, 27_000), (1 << 18, (1 << 17) + 9)]:
        a = random_sorted(rng, dt, na, "ties")[::-1].copy()
        b = random_sorted(rng, dt, nb, "ties")[::-1].copy()
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        ek, ev = desc_merge_expect(a, b, av, bv)
        ok, ov = mp.mp_merge_pairs(to_dev(a), vals_to_dev(av), to_dev(b), vals_to_dev(bv), descending=True)
        assert first_mismatch(to_host(ok, dt), ek) is None, (na, nb)
        assert first_mismatch(to_host(ov, np.uint32), ev) is None, (na, nb)
        if na + nb:
            assert mp.mp_check_sorted(ok, descending=True) == mp.MP_OK
    for n in [2, 4097, 100_003]:
        x = random_sorted(rng, dt, n, "ties")[rng.permutation(n)]
        v = np.arange(n, dtype=np.uint32)
        ek, ev = desc_sort_expect(x, v)
        tk, tv = to_dev(x), vals_to_dev(v)
        mp.mp_sort(tk, tv, descending=True)
        assert first_mismatch(to_host(tk, dt), ek) is None, n
        assert first_mismatch(to_host(tv, np.uint32), ev) is None, n


@pytest.mark.gpu
def test_descending_batched():
    rng = np.random.default_rng(4100)
    la, lb = rng.integers(0, 3000, 50), rng.integers(0, 3000, 50)
    a_off = np.concatenate([[0], np.cumsum(la)]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(lb)]).astype(np.int64)
    a = np.concatenate([random_sorted(rng, np.int32, int(x), "ties")[::-1] for x in la])
    b = np.concatenate([random_sorted(rng, np.int32, int(x), "ties")[::-1] for x in lb])
    out = mp.mp_merge_batched(to_dev(a), to_dev(a_off), to_dev(b), to_dev(b_off), descending=True)
    got = out.cpu().numpy()
    av = np.arange(a.size, dtype=np.uint32)
    bv = np.arange(b.size, dtype=np.uint32)
    for s in range(50):
        ek, _ = desc_merge_expect(a[a_off[s]:a_off[s + 1]], b[b_off[s]:b_off[s + 1]],
                                  av[a_off[s]:a_off[s + 1]], bv[b_off[s]:b_off[s + 1]])
        c0 = a_off[s] + b_off[s]
        assert np.array_equal(got[c0:c0 + ek.size], ek), s
