"""GPU parity of the merge-based set operations (mp_set_operation) against
the CPU oracle, bit-exact, keys and values: every dtype and op, sizes
spanning many tiles with ragged tails, duplicate-free sets, multisets with
short runs, runs far longer than a tile (16 distinct keys), all keys equal,
disjoint and identical inputs, empty sides, descending order.  All calls go
through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_2628_gb300 as mp
from _util import first_mismatch, random_sorted, to_dev, to_host, vals_to_dev

pytestmark = pytest.mark.gpu

DTYPES = [np.int32, np.uint32, np.float32, np.uint64, np.int64]
OPS = ["union", "intersection", "difference", "symmetric_difference"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mp.lib()
    torch.cuda.init()


def _check(op, a, b, dt, with_vals=True):
    av = np.arange(a.size, dtype=np.uint32)
    bv = np.arange(a.size, a.size + b.size, dtype=np.uint32) + np.uint32(1 << 30)
    ek, ev = oracle.set_op(op, a, b, av, bv)
    if with_vals:
        k, v, cnt = mp.mp_set_operation(op, to_dev(a), to_dev(b), vals_to_dev(av), vals_to_dev(bv))
        assert int(cnt.item()) == ek.size, (op, a.size, b.size)
        assert first_mismatch(to_host(k, dt), ek) is None, (op, a.size, b.size)
        assert first_mismatch(to_host(v, np.uint32), ev) is None, (op, a.size, b.size)
    k, _, cnt = mp.mp_set_operation(op, to_dev(a), to_dev(b))
    assert int(cnt.item()) == ek.size, (op, a.size, b.size)
    assert first_mismatch(to_host(k, dt), ek) is None, (op, a.size, b.size)


def _distinct16(rng, dt, n):
    vals = np.unique(random_sorted(rng, dt, 64, "random"))[:16]
    return np.sort(rng.choice(vals, n)).astype(dt)


@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
@pytest.mark.parametrize("op", OPS)
def test_set_ops_match_oracle(op, dt):
    rng = np.random.default_rng(2000 + DTYPES.index(dt) * 7 + OPS.index(op))
    for na, nb in [(0, 0), (1, 0), (0, 1), (1, 1), (5, 3), (2047, 2049), (30_011, 17_003),
                   (262_144, 100_000), (1_000_003, 1_200_001)]:
        _check(op, random_sorted(rng, dt, na, "ties"), random_sorted(rng, dt, nb, "ties"), dt)
        _check(op, random_sorted(rng, dt, na, "random"), random_sorted(rng, dt, nb, "random"), dt,
               with_vals=na < 100_000)
    assert mp.mp_kernel_error(reset=True) == 0


@pytest.mark.parametrize("dt", [np.int32, np.uint64, np.float32], ids=lambda d: np.dtype(d).name)
def test_set_ops_long_runs_and_special_inputs(dt):
    """Runs of equal keys that span many tiles (16 distinct keys), all keys
    equal, disjoint inputs (every A below every B and the reverse), A equal
    to B, sets (no duplicates) with a large overlap."""
    rng = np.random.default_rng(2100)
    one = np.array([7], dtype=dt)
    cases = [
        (_distinct16(rng, dt, 300_001), _distinct16(rng, dt, 200_003)),
        (np.repeat(one, 50_000), np.repeat(one, 70_001)),
        (np.repeat(one, 70_001), np.repeat(one, 50_000)),
    ]
    lo = random_sorted(rng, dt, 90_000, "random")
    cases += [(lo[:40_000], lo[40_000:]), (lo[40_000:], lo[:40_000])]
    x = random_sorted(rng, dt, 120_000, "ties")
    cases += [(x, x.copy())]
    pool = np.unique(random_sorted(rng, dt, 600_000, "random"))
    a = np.sort(rng.choice(pool, 300_000, replace=False)).astype(dt)
    b = np.sort(rng.choice(pool, 250_000, replace=False)).astype(dt)
    cases += [(a, b)]
    for a, b in cases:
        for op in OPS:
            _check(op, a, b, dt)
    assert mp.mp_kernel_error(reset=True) == 0


def _flip(x):
    """An order-reversing bijection on keys: descending order of x is the
    ascending order of _flip(x) (bitwise NOT for integers, negation for
    float32, which also swaps -0.0 and +0.0)."""
    if x.dtype == np.float32:
        return (-x).astype(np.float32)
    return ~x


@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
def test_set_ops_descending(dt):
    rng = np.random.default_rng(2200)
    for na, nb in [(40_001, 27_000), (300_000, 310_007)]:
        a = random_sorted(rng, dt, na, "ties")[::-1].copy()
        b = random_sorted(rng, dt, nb, "ties")[::-1].copy()
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        for op in OPS:
            fk, ev = oracle.set_op(op, _flip(a), _flip(b), av, bv)
            ek = _flip(fk)
            k, v, _ = mp.mp_set_operation(op, to_dev(a), to_dev(b), vals_to_dev(av), vals_to_dev(bv),
                                          descending=True)
            assert first_mismatch(to_host(k, dt), ek) is None, (op, na, nb)
            assert first_mismatch(to_host(v, np.uint32), ev) is None, (op, na, nb)


def test_set_ops_capacity_and_errors():
    assert mp.mp_set_capacity("union", 5, 7) == 12
    assert mp.mp_set_capacity("intersection", 5, 7) == 5
    assert mp.mp_set_capacity("difference", 5, 7) == 5
    assert mp.mp_set_capacity("symmetric_difference", 5, 7) == 12
    assert mp.mp_set_capacity(9, 5, 7) == -1
    a = torch.arange(10, dtype=torch.int32, device="cuda")
    with pytest.raises(mp.MPError) as ei:
        mp.mp_set_operation("union", a, a[2:], out_keys=a)  # output overlaps the inputs
    assert ei.value.status == mp.MP_ERR_INVALID_ARG
