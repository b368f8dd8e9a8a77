"""Parity at the workloads' full sizes, in the launch configuration the
bench times (automatic plans, default stream).

* large key-value merge, A 2^28 + B 2^26 uint64 keys with uint32 payloads,
  all four key distributions: the whole output against the oracle's merge
  (bit-exact; the payload = source index shows stability);
* plain keys, 2 x 2^20 int32: the whole output against the oracle;
* batched, 16,384 segments with per-side lengths up to 2^18 (~7e8 keys):
  a seeded sample of segments merged one by one by the oracle, plus the
  sortedness of every segment's output;
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


def test_batched_full_size_sampled():
    a, a_off, b, b_off = gen.batched()
    assert a.size + b.size > 5e8
    out = mp.mp_merge_batched(to_dev(a), to_dev(a_off), to_dev(b), to_dev(b_off)).cpu().numpy()
    rng = np.random.default_rng(99)
    nseg = a_off.size - 1
    for s in list(rng.choice(nseg, 200, replace=False)) + [0, nseg - 1]:
        ek, _ = oracle.merge(a[a_off[s]:a_off[s + 1]], b[b_off[s]:b_off[s + 1]])
        c0, c1 = a_off[s] + b_off[s], a_off[s + 1] + b_off[s + 1]
        assert np.array_equal(out[c0:c1], ek), s
    # Every segment's output is ascending (segment starts excluded).
    c = a_off + b_off
    ok = np.ones(out.size, dtype=bool)
    ok[1:] = out[1:] >= out[:-1]
    ok[c[1:-1]] = True
    assert ok.all()


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
