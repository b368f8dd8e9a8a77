"""GPU parity of 128-bit (multi-word) keys, MP_U128 and MP_I128, against the
CPU oracle, bit-exact: merges under every compiled plan (TMA tiles and the
streaming merge), split points, sort, set operations, descending order, and
the entry points that refuse 128-bit keys.  Keys are (n, 2) tensors of
64-bit words, low word first; all calls go through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_2628_gb300 as mp
from _util import first_mismatch, vals_to_dev

pytestmark = pytest.mark.gpu

KINDS = ["u128", "i128"]
PLANS = [None, (128, 8, mp.MP_STAGE_BULK), (256, 8, mp.MP_STAGE_BULK), (128, 12, mp.MP_STAGE_BULK),
         (128, 9, mp.MP_STAGE_BULK),
         (128, 8, mp.MP_STAGE_STREAM),
         (256, 4, mp.MP_STAGE_STREAM)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mp.lib()
    torch.cuda.init()


def wide_sorted(rng, n, kind, ties=True):
    """n sorted 128-bit keys as (n, 2) uint64 (low, high).  With ties the high
    word takes few values and the low word a small range, so equal keys and
    keys equal in one word only are common."""
    hi = rng.integers(0, 16 if ties else 1 << 62, n, dtype=np.uint64)
    lo = rng.integers(0, 64 if ties else 1 << 63, n, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    if kind == "i128":
        hi = hi - np.uint64(8)  # wraps: half of the keys are negative
    hi_order = hi.view(np.int64) if kind == "i128" else hi
    order = np.lexsort((lo, hi_order))
    return np.stack([lo[order], hi[order]], axis=1)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def to_host(t):
    return t.cpu().numpy().view(np.uint64).reshape(-1, 2)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("plan", PLANS, ids=str)
def test_wide_merge_every_plan(kind, plan):
    rng = np.random.default_rng(3000 + KINDS.index(kind))
    for na, nb in [(0, 0), (1, 0), (0, 3), (5, 7), (1023, 1025), (30_011, 17_003), (400_000, 300_001)]:
        a, b = wide_sorted(rng, na, kind), wide_sorted(rng, nb, kind)
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        ek, ev = oracle.merge(a, b, av, bv, kind=kind)
        ok, ov = mp.mp_merge_plan(to_dev(a), to_dev(b), vals_to_dev(av), vals_to_dev(bv), plan=plan, wide=kind)
        assert np.array_equal(to_host(ok), ek), (na, nb, plan)
        assert first_mismatch(ov.cpu().numpy().view(np.uint32), ev) is None, (na, nb, plan)
        ko = mp.mp_merge_plan(to_dev(a), to_dev(b), plan=plan, wide=kind)
        assert np.array_equal(to_host(ko), ek), (na, nb, plan)
    assert mp.mp_kernel_error(reset=True) == 0


@pytest.mark.parametrize("kind", KINDS)
def test_wide_partition_and_keys_entry_points(kind):
    rng = np.random.default_rng(3100)
    a, b = wide_sorted(rng, 50_000, kind), wide_sorted(rng, 70_001, kind)
    A, B = to_dev(a), to_dev(b)
    got = mp.mp_merge_path_partition(A, B, 4096, wide=kind).cpu().numpy()
    n = 120_001
    diags = [min(t * 4096, n) for t in range((n + 4095) // 4096 + 1)]
    assert got.tolist() == [oracle.split(a, b, d, kind=kind)[0] for d in diags]
    ek, _ = oracle.merge(a, b, kind=kind)
    assert np.array_equal(to_host(mp.mp_merge_keys(A, B, wide=kind)), ek)
    av = torch.arange(50_000, dtype=torch.int32, device="cuda")
    bv = torch.arange(70_001, dtype=torch.int32, device="cuda")
    k, _ = mp.mp_merge_pairs(A, av, B, bv, wide=kind)
    assert np.array_equal(to_host(k), ek)
    assert mp.mp_check_sorted(k, wide=kind) == mp.MP_OK
    if n > 2:
        bad = k.clone()
        bad[[0, n - 1]] = bad[[n - 1, 0]]
        assert mp.mp_check_sorted(bad, wide=kind) == mp.MP_ERR_NOT_SORTED


@pytest.mark.parametrize("kind", KINDS)
def test_wide_sort(kind):
    rng = np.random.default_rng(3200)
    for n in [2, 1023, 1024, 1025, 5000, 100_003, 1 << 20]:
        keys = wide_sorted(rng, n, kind, ties=n < 10_000)[rng.permutation(n)]
        vals = np.arange(n, dtype=np.uint32)
        ek, ev = oracle.sort(keys, vals, kind=kind)
        tk, tv = to_dev(keys), vals_to_dev(vals)
        mp.mp_sort(tk, tv, wide=kind)
        assert np.array_equal(to_host(tk), ek), n
        assert first_mismatch(tv.cpu().numpy().view(np.uint32), ev) is None, n
        tk = to_dev(keys)
        mp.mp_sort(tk, wide=kind)
        assert np.array_equal(to_host(tk), ek), n


@pytest.mark.parametrize("kind", KINDS)
def test_wide_set_ops(kind):
    rng = np.random.default_rng(3300)
    for na, nb in [(0, 10), (9, 0), (30_000, 20_001), (300_000, 250_003)]:
        a, b = wide_sorted(rng, na, kind), wide_sorted(rng, nb, kind)
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        for op in ["union", "intersection", "difference", "symmetric_difference"]:
            ek, ev = oracle.set_op(op, a, b, av, bv, kind=kind)
            k, v, cnt = mp.mp_set_operation(op, to_dev(a), to_dev(b), vals_to_dev(av), vals_to_dev(bv), wide=kind)
            assert int(cnt.item()) == ek.shape[0], (op, na, nb)
            assert np.array_equal(to_host(k), ek), (op, na, nb)
            assert first_mismatch(v.cpu().numpy().view(np.uint32), ev) is None, (op, na, nb)
    assert mp.mp_kernel_error(reset=True) == 0


@pytest.mark.parametrize("kind", KINDS)
def test_wide_descending(kind):
    """Stable descending merge = reversed ascending merge of reversed B with
    reversed A; descending sort = reversed ascending sort of reversed input."""
    rng = np.random.default_rng(3400)
    a, b = wide_sorted(rng, 60_001, kind)[::-1].copy(), wide_sorted(rng, 40_000, kind)[::-1].copy()
    av = np.arange(a.shape[0], dtype=np.uint32)
    bv = np.arange(a.shape[0], a.shape[0] + b.shape[0], dtype=np.uint32)
    k, v = oracle.merge(b[::-1].copy(), a[::-1].copy(), bv[::-1].copy(), av[::-1].copy(), kind=kind)
    for plan in [None, (128, 8, mp.MP_STAGE_BULK)]:
        ok, ov = mp.mp_merge_plan(to_dev(a), to_dev(b), vals_to_dev(av), vals_to_dev(bv), plan=plan,
                                  descending=True, wide=kind)
        assert np.array_equal(to_host(ok), k[::-1])
        assert np.array_equal(ov.cpu().numpy().view(np.uint32), v[::-1])
    x = wide_sorted(rng, 70_000, kind)[rng.permutation(70_000)]
    xv = np.arange(70_000, dtype=np.uint32)
    sk, sv = oracle.sort(x[::-1].copy(), xv[::-1].copy(), kind=kind)
    tk, tv = to_dev(x), vals_to_dev(xv)
    mp.mp_sort(tk, tv, descending=True, wide=kind)
    assert np.array_equal(to_host(tk), sk[::-1])
    assert np.array_equal(tv.cpu().numpy().view(np.uint32), sv[::-1])


def test_wide_unsupported_entry_points():
    x = torch.zeros((4, 2), dtype=torch.int64, device="cuda")
    off = torch.tensor([0, 4], dtype=torch.int64, device="cuda")
    out = torch.empty((8, 2), dtype=torch.int64, device="cuda")
    lib = mp.lib()
    st = lib.mp_merge_batched(mp.MP_U128, x.data_ptr(), off.data_ptr(), x.data_ptr(), off.data_ptr(), 1, 4, 4,
                              out.data_ptr(), None, None, None, None, None)
    assert st == mp.MP_ERR_UNSUPPORTED_DTYPE
    cs = torch.empty(1, dtype=torch.int64, device="cuda")
    st = lib.mp_merge_checksum(mp.MP_I128, x.data_ptr(), None, 4, x.data_ptr(), None, 4, cs.data_ptr(), None)
    assert st == mp.MP_ERR_UNSUPPORTED_DTYPE
    st = lib.mp_merge_noalloc(mp.MP_U128, x.data_ptr(), None, 4, x.data_ptr(), None, 4, out.data_ptr(), None,
                              None)
    assert st == mp.MP_ERR_UNSUPPORTED_DTYPE
