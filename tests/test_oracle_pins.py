"""Pins for the CPU oracle, independent of the oracle's own code.

The paper prints no worked example (its figures carry no values), so the
oracle is pinned by: brute force on tiny inputs (a tagged concatenation put
through a library stable sort -- the textbook fact that a stable merge of A
and B equals a stable sort of A followed by B), closed forms the paper names
(every A above every B, Sec. I), invariants (Lemma 8 / Cor. 12: split points
move by 0 or 1 per diagonal; Alg. 2's two-sided acceptance test; Thm 14's
bound on search steps) and hand-written golden fixtures.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

DTYPES = [np.int32, np.uint32, np.float32, np.uint64, np.int64]


# ---------------------------------------------------------------- brute force

def total_order_key(x):
    """Sort key for one key value: numeric, with -0.0 before +0.0."""
    if isinstance(x, float):
        return (x, math.copysign(1.0, x))
    return (x, 0)


def brute_merge(a, b):
    """Stable merge by definition: concatenate A then B, tag each element
    with its source, stable-sort by key (Python's sort is stable)."""
    tagged = [(x, "A", i) for i, x in enumerate(a)] + [(x, "B", j) for j, x in enumerate(b)]
    return sorted(tagged, key=lambda t: total_order_key(t[0]))


def brute_split(a, b, d):
    """a(d) by definition: number of A elements among the first d outputs."""
    return sum(1 for t in brute_merge(a, b)[:d] if t[1] == "A")


def sorted_seqs(max_len, alphabet):
    for n in range(max_len + 1):
        yield from itertools.combinations_with_replacement(alphabet, n)


def test_merge_and_split_exhaustive_tiny():
    """Every pair of sorted sequences of length <= 5 over {0, 1, 2}."""
    seqs = [np.array(s, dtype=np.int32) for s in sorted_seqs(5, (0, 1, 2))]
    assert len(seqs) == 56
    for a in seqs:
        for b in seqs:
            av = np.arange(a.size, dtype=np.uint32)
            bv = np.arange(100, 100 + b.size, dtype=np.uint32)
            keys, vals = oracle.merge(a, b, av, bv)
            expect = brute_merge(a.tolist(), b.tolist())
            assert keys.tolist() == [t[0] for t in expect]
            assert vals.tolist() == [t[2] if t[1] == "A" else 100 + t[2] for t in expect]
            n_a_so_far = 0
            for d in range(a.size + b.size + 1):
                s, _ = oracle.split(a, b, d)
                assert s == n_a_so_far, (a, b, d)
                if d < len(expect) and expect[d][1] == "A":
                    n_a_so_far += 1


def _random_sorted(rng, dtype, n, lo, hi):
    if np.dtype(dtype).kind == "f":
        x = rng.integers(lo, hi, n).astype(np.float32) * np.float32(0.5)
        # Put both zeros in: the sign of zero matters in the float order.
        zeros = rng.random(n) < 0.1
        x[zeros] = np.where(rng.random(zeros.sum()) < 0.5, np.float32(-0.0), np.float32(0.0))
        return np.array(sorted(x.tolist(), key=total_order_key), dtype=np.float32)
    return np.sort(rng.integers(lo, hi, n).astype(dtype))


@pytest.mark.parametrize("dtype", DTYPES)
def test_merge_random_vs_library_stable_sort(dtype):
    """Random sizes up to 10^4: the merge equals numpy's stable argsort of the
    tagged concatenation (for float32 via lexsort on (sign of zero, value))."""
    rng = np.random.default_rng(7)
    signed = np.dtype(dtype).kind in "if"
    for trial in range(40):
        na, nb = int(rng.integers(0, 10_000)), int(rng.integers(0, 10_000))
        if trial % 7 == 0:
            na = 0
        lo, hi = (-50, 50) if signed else (0, 100)
        if trial % 3 == 0:
            lo, hi = (-(1 << 30), 1 << 30) if signed else (0, 1 << 31)
        a = _random_sorted(rng, dtype, na, lo, hi)
        b = _random_sorted(rng, dtype, nb, lo, hi)
        av = rng.integers(0, 1 << 32, na, dtype=np.uint64).astype(np.uint32)
        bv = rng.integers(0, 1 << 32, nb, dtype=np.uint64).astype(np.uint32)
        keys, vals = oracle.merge(a, b, av, bv)
        cat = np.concatenate([a, b])
        if np.dtype(dtype).kind == "f":
            order = np.lexsort((~np.signbit(cat), cat))
        else:
            order = np.argsort(cat, kind="stable")
        assert np.array_equal(keys.view(np.uint8), cat[order].view(np.uint8))
        assert np.array_equal(vals, np.concatenate([av, bv])[order])
        keys_only, none = oracle.merge(a, b)
        assert none is None and np.array_equal(keys_only.view(np.uint8), keys.view(np.uint8))


# ---------------------------------------------------------------- closed forms

def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                tag, *vals = line.split()
                rows.append((tag, vals))
    return rows


def test_golden_adversarial_all_a_greater_than_b():
    rows = dict(_read_golden("adversarial_a_gt_b.txt"))
    a = np.array(rows["A"], dtype=np.int32)
    b = np.array(rows["B"], dtype=np.int32)
    keys, _ = oracle.merge(a, b)
    assert keys.tolist() == [int(x) for x in rows["S"]]
    assert [oracle.split(a, b, d)[0] for d in range(a.size + b.size + 1)] == \
        [int(x) for x in rows["SPLIT"]]
    # Naive equal splitting gives a different first part than the true merge.
    assert [int(x) for x in rows["NAIVE_FIRST_PART"]] != keys[:4].tolist()


def test_golden_alg2_bounds():
    a = b = None
    for tag, vals in _read_golden("alg2_bounds.txt"):
        if tag == "A":
            a = np.array(vals, dtype=np.int32)
        elif tag == "B":
            b = np.array(vals, dtype=np.int32)
        else:
            d, expect = int(vals[0]), int(vals[1])
            assert oracle.split(a, b, d)[0] == expect, (a, b, d)


def test_golden_f32_total_order():
    bits = [int(tag, 16) for tag, _ in _read_golden("f32_total_order.txt")]
    keys = np.array(bits, dtype=np.uint32).view(np.float32)
    n = keys.size
    # Sorting any permutation must give the fixture's order, bit for bit.
    rng = np.random.default_rng(3)
    for _ in range(20):
        perm = rng.permutation(n)
        s, _ = oracle.sort(keys[perm])
        assert s.view(np.uint32).tolist() == bits
    # Merging the even- and odd-indexed halves must interleave them back.
    m, _ = oracle.merge(keys[0::2], keys[1::2])
    assert m.view(np.uint32).tolist() == bits


@pytest.mark.parametrize("dtype", [np.int32, np.uint64, np.float32])
def test_closed_form_all_a_greater(dtype):
    """Sec. I: every A above every B -> S = B || A and a(d) = max(0, d - |B|)."""
    rng = np.random.default_rng(11)
    for na, nb in [(1, 1), (5, 9), (1000, 37), (0, 10), (10, 0)]:
        b = np.sort(rng.integers(0, 1000, nb)).astype(dtype)
        a = np.sort(rng.integers(2000, 3000, na)).astype(dtype)
        keys, _ = oracle.merge(a, b)
        assert np.array_equal(keys, np.concatenate([b, a]))
        for d in range(na + nb + 1):
            assert oracle.split(a, b, d)[0] == max(0, d - nb)


@pytest.mark.parametrize("dtype", [np.int32, np.uint64, np.float32])
def test_closed_form_all_equal(dtype):
    """All keys equal -> S = A || B (ties take A) and a(d) = min(d, |A|)."""
    for na, nb in [(1, 1), (7, 3), (300, 800), (0, 4)]:
        a = np.full(na, 5, dtype=dtype)
        b = np.full(nb, 5, dtype=dtype)
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        keys, vals = oracle.merge(a, b, av, bv)
        assert np.array_equal(vals, np.arange(na + nb, dtype=np.uint32))
        for d in range(na + nb + 1):
            assert oracle.split(a, b, d)[0] == min(d, na)


def test_closed_form_interleaved():
    """Distinct keys key(r) = r * step dealt to A and B: S[r] = key(r)."""
    for na, nb in [(16, 4), (400, 100), (37, 91), (1, 50)]:
        a, av, b, bv = gen.large_kv("interleaved", na, nb)
        keys, vals = oracle.merge(a, b, av, bv)
        n = na + nb
        step = np.uint64((1 << 64) // n)
        assert np.array_equal(keys, np.arange(n, dtype=np.uint64) * step)


def test_closed_form_distinct16_groups():
    """16 distinct values: S is grouped by value in ascending order; inside a
    group A's elements come first, in order, then B's (payload = source index)."""
    a, av, b, bv = gen.large_kv("distinct16", 3000, 1200)
    keys, vals = oracle.merge(a, b, av, bv)
    pos = 0
    for v in np.unique(np.concatenate([a, b])):
        ca, cb = int((a == v).sum()), int((b == v).sum())
        grp_keys = keys[pos:pos + ca + cb]
        grp_vals = vals[pos:pos + ca + cb]
        assert np.all(grp_keys == v)
        assert np.array_equal(grp_vals[:ca], av[a == v])
        assert np.array_equal(grp_vals[ca:], bv[b == v])
        pos += ca + cb
    assert pos == keys.size


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("dtype", DTYPES)
def test_split_invariants(dtype):
    """Lemma 8 / Cor. 12: a(d) is nondecreasing with steps of 0 or 1; Alg. 2's
    acceptance test holds at every split; Thm 14: the search needs at most
    floor(log2(w)) + 1 probes, w = number of grid points on the diagonal
    (w <= min(|A|, |B|) + 1)."""
    rng = np.random.default_rng(5)
    for na, nb in [(0, 0), (1, 0), (0, 3), (13, 200), (257, 255), (1000, 1000), (3, 4000)]:
        a = _random_sorted(rng, dtype, na, 0, 40)
        b = _random_sorted(rng, dtype, nb, 0, 40)
        prev = 0
        for d in range(na + nb + 1):
            s, steps = oracle.split(a, b, d)
            assert s - prev in (0, 1) or d == 0
            prev = s
            t = d - s
            assert 0 <= s <= na and 0 <= t <= nb
            # A[s] > B[t-1] and A[s-1] <= B[t], with sentinels.
            if s < na and t > 0:
                assert total_order_key(a[s].item()) > total_order_key(b[t - 1].item())
            if s > 0 and t < nb:
                assert total_order_key(a[s - 1].item()) <= total_order_key(b[t].item())
            w = min(d, na) - max(0, d - nb) + 1
            assert steps <= int(math.floor(math.log2(w))) + 1
            assert w <= min(na, nb) + 1


def test_split_rejects_out_of_range():
    a = np.arange(3, dtype=np.int32)
    with pytest.raises(ValueError):
        oracle.split(a, a, 7)
    with pytest.raises(ValueError):
        oracle.split(a, a, -1)


# ---------------------------------------------------------------- sort

@pytest.mark.parametrize("dtype", DTYPES)
def test_sort_vs_brute_force(dtype):
    rng = np.random.default_rng(9)
    for n in [0, 1, 2, 3, 5, 8, 17, 100, 1023, 4097]:
        lo, hi = (-20, 20) if np.dtype(dtype).kind in "if" else (0, 40)
        if np.dtype(dtype).kind == "f":
            k = (rng.integers(lo, hi, n) * 0.25).astype(np.float32)
            k[rng.random(n) < 0.1] = np.float32(-0.0)
        else:
            k = rng.integers(lo, hi, n).astype(dtype)
        v = np.arange(n, dtype=np.uint32)
        sk, sv = oracle.sort(k, v)
        expect = sorted(zip(k.tolist(), range(n)), key=lambda t: total_order_key(t[0]))
        assert sk.view(np.uint8).tolist() == np.array([t[0] for t in expect], dtype=dtype).view(np.uint8).tolist()
        assert sv.tolist() == [t[1] for t in expect]


def test_sort_special_orders():
    rng = np.random.default_rng(2)
    # sorted input -> identity
    k = np.sort(rng.integers(-1000, 1000, 5000).astype(np.int32))
    sk, sv = oracle.sort(k, np.arange(k.size))
    assert np.array_equal(sk, k) and np.array_equal(sv, np.arange(k.size))
    # reverse-sorted distinct input -> reversal
    k = np.arange(4096, dtype=np.int32)[::-1] * 3 - 7
    sk, sv = oracle.sort(k, np.arange(k.size))
    assert np.array_equal(sk, k[::-1]) and np.array_equal(sv, np.arange(k.size)[::-1])
    # 256 distinct values -> a counting sort: values ascending, payloads of
    # each value in increasing source position.
    vals256 = np.sort(rng.choice(1 << 20, 256, replace=False)).astype(np.int32)
    k = vals256[rng.integers(0, 256, 20000)]
    sk, sv = oracle.sort(k, np.arange(k.size))
    counts = np.array([(k == v).sum() for v in vals256])
    assert np.array_equal(sk, np.repeat(vals256, counts))
    assert np.array_equal(sv, np.concatenate([np.flatnonzero(k == v) for v in vals256]))


def test_sort_is_permutation_and_stable_f32():
    k = gen.sort_input("f32", "random", n=5000)
    sk, sv = oracle.sort(k, np.arange(k.size, dtype=np.uint32))
    assert np.array_equal(np.sort(sk.view(np.uint32)), np.sort(k.view(np.uint32)))
    assert np.array_equal(k[sv].view(np.uint32), sk.view(np.uint32))
    kk = [total_order_key(x) for x in sk.tolist()]
    assert all(kk[i] <= kk[i + 1] for i in range(len(kk) - 1))
    for i in range(len(kk) - 1):
        if kk[i] == kk[i + 1]:
            assert sv[i] < sv[i + 1]


# ---------------------------------------------------------------- batched

def test_merge_batched_vs_brute_force():
    rng = np.random.default_rng(4)
    len_a = rng.integers(0, 30, 200)
    len_b = rng.integers(0, 30, 200)
    len_a[::17] = 0
    len_b[::13] = 0
    a, a_off, b, b_off, av, bv = gen.batched(len_a=len_a, len_b=len_b, with_values=True)
    keys, vals = oracle.merge_batched(a, a_off, b, b_off, av, bv)
    for s in range(len_a.size):
        sa = a[a_off[s]:a_off[s + 1]].tolist()
        sb = b[b_off[s]:b_off[s + 1]].tolist()
        expect = brute_merge(sa, sb)
        c = a_off[s] + b_off[s]
        got_k = keys[c:c + len(expect)].tolist()
        got_v = vals[c:c + len(expect)].tolist()
        assert got_k == [t[0] for t in expect]
        assert got_v == [int(av[a_off[s] + t[2]]) if t[1] == "A" else int(bv[b_off[s] + t[2]])
                         for t in expect]
