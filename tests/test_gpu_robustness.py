"""Broken preconditions must give wrong output, never an out-of-range access:
unsorted inputs (whose split points need not be monotone) through the tiled,
streaming, batched and set-operation kernels, and foreign split arrays
through mp_merge_partitioned.  Each call must return normally, leave no
CUDA error, report only the documented kernel flags, and leave the context
able to merge exactly again.  (Every window these kernels stage is clamped
into its array, clamp_end_split; walks that skip end tests read only into
spare slots of their own shared memory.)"""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_2628_gb300 as mp
from _util import first_mismatch, random_sorted, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mp.lib()
    torch.cuda.init()


def _healthy():
    """The device still merges exactly (no sticky error, no leftover flag)."""
    torch.cuda.synchronize()
    rng = np.random.default_rng(77)
    a, b = random_sorted(rng, np.int32, 50_001, "ties"), random_sorted(rng, np.int32, 30_007, "ties")
    out = mp.mp_merge_keys(to_dev(a), to_dev(b))
    assert first_mismatch(to_host(out, np.int32), oracle.merge(a, b)[0]) is None
    assert mp.mp_kernel_status() == mp.MP_OK


def _unsorted(rng, dt, n):
    if np.dtype(dt).itemsize == 8:
        return rng.integers(0, 1 << 62, n, dtype=np.uint64).astype(dt)
    return rng.integers(-(1 << 31), 1 << 31, n).astype(dt)


@pytest.mark.parametrize("plan", [None, (128, 33, mp.MP_STAGE_BULK), (256, 12, mp.MP_STAGE_BULK),
                                  (128, 8, mp.MP_STAGE_VECTOR), (0, 0, mp.MP_STAGE_STREAM)],
                         ids=["auto", "128x33", "256x12", "vector", "stream"])
@pytest.mark.parametrize("vals", [False, True])
def test_unsorted_inputs_merge_without_fault(plan, vals):
    rng = np.random.default_rng(3000)
    for na, nb in [(300_001, 200_003), (1 << 20, 7), (5, 400_000)]:
        a, b = _unsorted(rng, np.int32, na), _unsorted(rng, np.int32, nb)
        A, B = to_dev(a), to_dev(b)
        if vals:
            AV = torch.arange(na, dtype=torch.int32, device="cuda")
            BV = torch.arange(nb, dtype=torch.int32, device="cuda")
            mp.mp_merge_plan(A, B, AV, BV, plan=plan)
        else:
            mp.mp_merge_plan(A, B, plan=plan)
        assert mp.mp_kernel_status(reset=True) == mp.MP_OK
        assert mp.mp_check_sorted(A) == mp.MP_ERR_NOT_SORTED
    _healthy()


@pytest.mark.parametrize("plan", [(128, 33, mp.MP_STAGE_BULK), (256, 12, mp.MP_STAGE_BULK),
                                  (128, 8, mp.MP_STAGE_VECTOR)], ids=["128x33", "256x12", "vector"])
def test_foreign_split_arrays_without_fault(plan):
    rng = np.random.default_rng(3100)
    na, nb = 400_000, 333_333
    a, b = random_sorted(rng, np.uint64, na, "random"), random_sorted(rng, np.uint64, nb, "random")
    A, B = to_dev(a), to_dev(b)
    AV = torch.arange(na, dtype=torch.int32, device="cuda")
    BV = torch.arange(na, na + nb, dtype=torch.int32, device="cuda")
    tile = mp.mp_merge_tile_items(torch.uint64, True, na + nb, plan)
    nbounds = (na + nb + tile - 1) // tile + 1
    for kind in ["random", "decreasing", "extreme"]:
        if kind == "random":
            s = rng.integers(-(1 << 40), 1 << 40, nbounds)
        elif kind == "decreasing":
            s = np.arange(nbounds, dtype=np.int64)[::-1] * tile
        else:
            s = np.where(np.arange(nbounds) % 2 == 0, np.int64(-(1 << 62)), np.int64(1 << 62))
        splits = torch.from_numpy(np.ascontiguousarray(s, dtype=np.int64)).cuda()
        mp.mp_merge_partitioned(A, B, splits, AV, BV, plan=plan)
        assert mp.mp_kernel_status(reset=True) == mp.MP_OK
    # The true splits still give the exact merge.
    splits = mp.mp_merge_path_partition(A, B, tile)
    ok, ov = mp.mp_merge_partitioned(A, B, splits, AV, BV, plan=plan)
    ek, ev = oracle.merge(a, b, np.arange(na, dtype=np.uint32), np.arange(na, na + nb, dtype=np.uint32))
    assert first_mismatch(to_host(ok, np.uint64), ek) is None
    assert first_mismatch(to_host(ov, np.uint32), ev) is None
    _healthy()


@pytest.mark.parametrize("op", ["union", "intersection", "difference", "symmetric_difference"])
@pytest.mark.parametrize("dt", [np.int32, np.uint64], ids=["i32", "u64"])
@pytest.mark.parametrize("vals", [False, True])
def test_unsorted_inputs_set_operations_without_fault(op, dt, vals):
    rng = np.random.default_rng(3200)
    for na, nb in [(300_001, 250_003), (40_000, 1)]:
        a, b = _unsorted(rng, dt, na), _unsorted(rng, dt, nb)
        A, B = to_dev(a), to_dev(b)
        if vals:
            AV = torch.arange(na, dtype=torch.int32, device="cuda")
            BV = torch.arange(nb, dtype=torch.int32, device="cuda")
            mp.mp_set_operation(op, A, B, AV, BV, trim=False)
        else:
            mp.mp_set_operation(op, A, B, trim=False)
        # Flag 2 (output would pass the capacity) is the documented report.
        assert mp.mp_kernel_status(reset=True) in (mp.MP_OK, mp.MP_ERR_NOT_SORTED)
    _healthy()


def test_unsorted_segments_batched_without_fault():
    rng = np.random.default_rng(3300)
    nseg = 500
    la = rng.integers(0, 3000, nseg)
    lb = rng.integers(0, 3000, nseg)
    a_off = np.concatenate([[0], np.cumsum(la)]).astype(np.int64)
    b_off = np.concatenate([[0], np.cumsum(lb)]).astype(np.int64)
    a, b = _unsorted(rng, np.int32, int(a_off[-1])), _unsorted(rng, np.int32, int(b_off[-1]))
    for plan in [None, (128, 12, mp.MP_STAGE_BULK), (128, 8, mp.MP_STAGE_VECTOR)]:
        mp.mp_merge_batched(to_dev(a), to_dev(a_off), to_dev(b), to_dev(b_off), plan=plan)
        assert mp.mp_kernel_status(reset=True) == mp.MP_OK
    _healthy()
