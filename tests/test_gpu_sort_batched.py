"""GPU parity of the merge sort (block sort + Merge Path passes) and of the
batched segmented merge against the CPU oracle, bit-exact, through the C ABI."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1406_2628_gb300 as mp
from _util import first_mismatch, random_sorted, to_dev, to_host, vals_to_dev

pytestmark = pytest.mark.gpu

DTYPES = [np.int32, np.uint32, np.float32, np.uint64, np.int64]
SORT_SIZES = [2, 3, 17, 100, 2047, 2048, 2049, 4095, 4096, 4097, 8193, 3 * 4096 + 5, 100_003,
              (1 << 18) + 7]


def _unsorted(rng, dt, n, kind):
    x = random_sorted(rng, dt, n, "random" if kind != "ties" else "ties")
    x = x[rng.permutation(n)]
    if kind == "sorted":
        return random_sorted(rng, dt, n, "ties")
    if kind == "reverse":
        return random_sorted(rng, dt, n, "random")[::-1].copy()
    return x


@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
@pytest.mark.parametrize("kind", ["random", "ties", "sorted", "reverse"])
def test_sort_keys(dt, kind):
    rng = np.random.default_rng(700 + DTYPES.index(dt))
    for n in SORT_SIZES:
        k = _unsorted(rng, dt, n, kind)
        t = to_dev(k)
        mp.mp_sort(t)
        ek, _ = oracle.sort(k)
        assert first_mismatch(to_host(t, dt), ek) is None, (n, first_mismatch(to_host(t, dt), ek))


@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
@pytest.mark.parametrize("kind", ["random", "ties"])
def test_sort_pairs_stable(dt, kind):
    rng = np.random.default_rng(800 + DTYPES.index(dt))
    for n in SORT_SIZES:
        k = _unsorted(rng, dt, n, kind)
        v = np.arange(n, dtype=np.uint32)
        tk, tv = to_dev(k), vals_to_dev(v)
        mp.mp_sort(tk, tv)
        ek, ev = oracle.sort(k, v)
        assert first_mismatch(to_host(tk, dt), ek) is None, n
        assert first_mismatch(to_host(tv, np.uint32), ev) is None, n


def test_sort_trivial_sizes():
    for n in [0, 1]:
        t = torch.arange(n, dtype=torch.int32, device="cuda")
        mp.mp_sort(t)
        assert t.numel() == n


@pytest.mark.parametrize("order", gen.SORT_ORDERS)
@pytest.mark.parametrize("dtype", ["i32", "f32"])
def test_sort_workload_scaled(order, dtype):
    """The merge sort workload (all int32 / all float32 bit patterns, four
    orders) at 2^20 keys, bit-exact against the oracle."""
    k = gen.sort_input(dtype, order, n=1 << 20)
    t = to_dev(k)
    mp.mp_sort(t)
    ek, _ = oracle.sort(k)
    assert first_mismatch(to_host(t, k.dtype), ek) is None


# ----------------------------------------------------------------- batched

BATCH_PLANS = [None, (128, 8), (256, 8), (128, 16), (256, 16),
               (128, 8, mp.MP_STAGE_VECTOR), (256, 16, mp.MP_STAGE_VECTOR),
               (128, 16, mp.MP_STAGE_BULK), (256, 12, mp.MP_STAGE_BULK), (128, 12, mp.MP_STAGE_VECTOR),
               (128, 27, mp.MP_STAGE_BULK), (128, 33, mp.MP_STAGE_BULK)]


def _batched_case(rng, nseg, max_len, dt=np.int32, empty_every=0):
    la = rng.integers(0, max_len + 1, nseg)
    lb = rng.integers(0, max_len + 1, nseg)
    if empty_every:
        la[::empty_every] = 0
        lb[::empty_every] = 0
    a_off = np.concatenate([[0], np.cumsum(la)]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(lb)]).astype(np.int64)
    a = np.concatenate([random_sorted(rng, dt, int(x), "ties") for x in la]) if nseg else np.empty(0, dt)
    b = np.concatenate([random_sorted(rng, dt, int(x), "ties") for x in lb]) if nseg else np.empty(0, dt)
    return a.astype(dt), a_off, b.astype(dt), b_off


@pytest.mark.parametrize("plan", BATCH_PLANS, ids=str)
@pytest.mark.parametrize("dt", [np.int32, np.float32, np.uint64], ids=lambda d: np.dtype(d).name)
def test_batched_pairs(plan, dt):
    rng = np.random.default_rng(900)
    for nseg, max_len, empty_every in [(1, 5000, 0), (7, 3, 0), (500, 40, 3), (300, 3000, 7),
                                       (2000, 1, 5), (64, 20_000, 0)]:
        a, a_off, b, b_off = _batched_case(rng, nseg, max_len, dt, empty_every)
        av = np.arange(a.size, dtype=np.uint32)
        bv = np.arange(a.size, a.size + b.size, dtype=np.uint32)
        out, outv = mp.mp_merge_batched(to_dev(a), to_dev(a_off), to_dev(b), to_dev(b_off),
                                        a_vals=vals_to_dev(av), b_vals=vals_to_dev(bv), plan=plan)
        ek, ev = oracle.merge_batched(a, a_off, b, b_off, av, bv)
        assert first_mismatch(to_host(out, dt), ek) is None, (nseg, max_len)
        assert first_mismatch(to_host(outv, np.uint32), ev) is None, (nseg, max_len)
        ko = mp.mp_merge_batched(to_dev(a), to_dev(a_off), to_dev(b), to_dev(b_off), plan=plan)
        assert first_mismatch(to_host(ko, dt), ek) is None, (nseg, max_len)


def test_batched_edge_cases():
    rng = np.random.default_rng(901)
    # All segments empty but one; one segment only A, one only B.
    for la, lb in [([0, 0, 5, 0], [0, 0, 0, 0]), ([0, 9], [4, 0]), ([3], [0]), ([0], [3])]:
        la, lb = np.array(la), np.array(lb)
        a_off = np.concatenate([[0], np.cumsum(la)]).astype(np.int64)
        b_off = np.concatenate([[0], np.cumsum(lb)]).astype(np.int64)
        a = np.concatenate([random_sorted(rng, np.int32, int(x)) for x in la])
        b = np.concatenate([random_sorted(rng, np.int32, int(x)) for x in lb])
        out = mp.mp_merge_batched(to_dev(a), to_dev(a_off), to_dev(b), to_dev(b_off))
        ek, _ = oracle.merge_batched(a, a_off, b, b_off)
        assert np.array_equal(out.cpu().numpy(), ek)
    # Zero segments, zero totals: no-op.
    z = torch.zeros(1, dtype=torch.int64, device="cuda")
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    out = mp.mp_merge_batched(e, z, e, z)
    assert out.numel() == 0


def test_batched_workload_scaled():
    """The batched workload's shape (log-uniform lengths from 1) with
    2048 segments of up to 2^12 per side."""
    a, a_off, b, b_off = gen.batched(n_seg=2048, log2_max=12.0)
    out = mp.mp_merge_batched(to_dev(a), to_dev(a_off), to_dev(b), to_dev(b_off))
    ek, _ = oracle.merge_batched(a, a_off, b, b_off)
    assert first_mismatch(out.cpu().numpy(), ek) is None
