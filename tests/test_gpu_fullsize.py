"""Parity at the workloads' full sizes, in the launch configuration the
bench times (automatic plans, default stream).

* large key-value merge, A 2^28 + B 2^26 uint64 keys with uint32 payloads,
  all four key distributions: the whole output against the oracle's merge
  (bit-exact; the payload = source index shows stability);
* plain keys, 2 x 2^20 int32: the whole output against the oracle;
* batched, 16,384 segments with per-side lengths up to 2^18 (~7e8 keys):
  the whole output against the oracle's per-segment merge;
* an int32 merge of 2^31 + 4097 outputs (past every 32-bit offset): the
  whole output and the split points past 2^31 against the oracle;
* set operations on two duplicate-free sets of about 2^27 int32 keys each
  sharing half (universe 2^28): all four operations on keys alone and the
  union with values, the whole output against the oracle's;
* sort of 2^28 keys (int32 and float32, four orders): properties that hold
  at any size -- the output is ascending under the key order (float: -0.0
  before +0.0) and is a permutation of the input (same multiset of bit
  patterns, checked with numpy's sort of the raw bits)."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1406_2628_gb300 as mp
from _util import first_mismatch, to_dev, to_host, vals_to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.parametrize("dist", gen.LARGE_KV_DISTS)
def test_large_kv_full_size(dist):
    a, av, b, bv = gen.large_kv(dist)
    ok, ov = mp.mp_merge_pairs(to_dev(a), vals_to_dev(av), to_dev(b), vals_to_dev(bv))
    got_k = to_host(ok, np.uint64)
    got_v = to_host(ov, np.uint32)
    del ok, ov
    torch.cuda.empty_cache()
    ek, ev = oracle.merge(a, b, av, bv)
    assert first_mismatch(got_k, ek) is None, dist
    assert first_mismatch(got_v, ev) is None, dist


def test_plain_keys_full_size():
    a, b = gen.plain_keys()
    out = mp.mp_merge_keys(to_dev(a), to_dev(b))
    ek, _ = oracle.merge(a, b)
    assert np.array_equal(out.cpu().numpy(), ek)


def test_batched_full_size():
    a, a_off, b, b_off = gen.batched()
    assert a.size + b.size > 5e8
    out = mp.mp_merge_batched(to_dev(a), to_dev(a_off), to_dev(b), to_dev(b_off)).cpu().numpy()
    torch.cuda.empty_cache()
    # Every one of the 16,384 segments against the oracle's per-segment merge.
    ek, _ = oracle.merge_batched(a, a_off, b, b_off)
    assert first_mismatch(out, ek) is None


def _chunks_equal(x: np.ndarray, y: np.ndarray, chunk: int = 1 << 27):
    """First index where x and y differ (bit patterns), or None."""
    assert x.shape == y.shape
    for i in range(0, x.size, chunk):
        bad = np.flatnonzero(x[i:i + chunk] != y[i:i + chunk])
        if bad.size:
            return i + int(bad[0])
    return None


def _sorted_int32_with_ties(seed: int, n: int, start: int, max_gap: int) -> np.ndarray:
    """n sorted int32 keys from start, gaps uniform in [0, max_gap) (gap 0 =
    a tie), made sorted by construction (a running sum)."""
    rng = np.random.default_rng(seed)
    x = rng.integers(0, max_gap, n, dtype=np.int8).astype(np.int64)
    np.cumsum(x, out=x)
    x += start
    assert x[-1] < 2**31
    return x.astype(np.int32)


def test_set_operations_full_size():
    a, b = gen.sets()
    assert a.size > 1.3e8 and b.size > 1.3e8
    A, B = to_dev(a), to_dev(b)
    for op in ["union", "intersection", "difference", "symmetric_difference"]:
        k, _, _ = mp.mp_set_operation(op, A, B)
        got = to_host(k, np.int32)
        del k
        ek, _ = oracle.set_op(op, a, b)
        assert first_mismatch(got, ek) is None, op
    av = np.arange(a.size, dtype=np.uint32)
    bv = np.arange(a.size, a.size + b.size, dtype=np.uint64).astype(np.uint32)
    k, v, _ = mp.mp_set_operation("union", A, B, vals_to_dev(av), vals_to_dev(bv))
    got_k, got_v = to_host(k, np.int32), to_host(v, np.uint32)
    del k, v, A, B
    torch.cuda.empty_cache()
    ek, ev = oracle.set_op("union", a, b, av, bv)
    assert first_mismatch(got_k, ek) is None
    assert first_mismatch(got_v, ev) is None
    assert mp.mp_kernel_status(reset=True) == mp.MP_OK


def test_merge_above_2e31_outputs():
    """int32 keys, |A| = |B| = 2^30, plus 4097 more in B: 2^31 + 4097
    outputs, so every output offset, split point and tile index past 2^31
    goes through the 64-bit paths (Thm 14 / Cor. 6 make the method
    independent of n).  The whole output against the oracle's merge, and the
    partition's split points at diagonals past 2^31 against the oracle's
    Alg. 2."""
    na, nb = 1 << 30, (1 << 30) + 4097
    a = _sorted_int32_with_ties(31, na, -(1 << 30), 3)
    b = _sorted_int32_with_ties(32, nb, -(1 << 30) + 1, 3)
    A, B = to_dev(a), to_dev(b)
    out = mp.mp_merge_keys(A, B)
    spacing = mp.mp_merge_tile_items(torch.int32, False, na + nb)
    splits = mp.mp_merge_path_partition(A, B, spacing).cpu().numpy()
    got = out.cpu().numpy()
    del A, B, out
    torch.cuda.empty_cache()
    ek, _ = oracle.merge(a, b)
    assert _chunks_equal(got, ek) is None
    del ek
    # Tile boundaries past 2^31 from the partition kernel.
    n_bounds = splits.size
    for t in [n_bounds - 1, n_bounds - 2, (1 << 31) // spacing, (1 << 31) // spacing + 1]:
        d = min(t * spacing, na + nb)
        assert splits[t] == oracle.split(a, b, d)[0], t


def _ascending_total_order(x: np.ndarray) -> bool:
    if x.dtype == np.float32:
        u = x.view(np.uint32)
        enc = np.where(u >> 31 == 1, ~u, u | np.uint32(0x80000000))
        return bool(np.all(enc[1:] >= enc[:-1]))
    return bool(np.all(x[1:] >= x[:-1]))


@pytest.mark.parametrize("order", gen.SORT_ORDERS)
@pytest.mark.parametrize("dtype", ["i32", "f32"])
def test_sort_full_size_properties(dtype, order):
    k = gen.sort_input(dtype, order)
    t = to_dev(k)
    mp.mp_sort(t)
    got = t.cpu().numpy()
    del t
    torch.cuda.empty_cache()
    assert _ascending_total_order(got)
    bits = np.uint32 if dtype == "f32" else np.int32
    assert np.array_equal(np.sort(got.view(bits)), np.sort(k.view(bits)))
