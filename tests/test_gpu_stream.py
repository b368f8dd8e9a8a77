"""GPU parity of the partition-free streaming merge (MP_STAGE_STREAM, Alg. 3)
against the CPU oracle, bit-exact: every compiled shape, every dtype, both
orders, shares of one and of many tiles per CTA, one side exhausted for
long stretches, unaligned pointers, graphs, and no kernel error reported by
its bounded waits.  All calls go through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_2628_gb300 as mp
from _util import first_mismatch, random_sorted, to_dev, to_host, vals_to_dev

pytestmark = pytest.mark.gpu

DTYPES = [np.int32, np.uint32, np.float32, np.uint64, np.int64]
S = mp.MP_STAGE_STREAM


def _shapes():
    out = []
    for nt in (64, 128, 256, 512):
        for vt in (4, 8, 16):
            if mp.mp_plan_supported((nt, vt, S)):
                out.append((nt, vt, S))
    return out


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mp.lib()
    torch.cuda.init()


def _expect(a, b, av, bv, desc):
    if not desc:
        return oracle.merge(a, b, av, bv)
    # Stable descending merge = reversed ascending merge of reversed B with
    # reversed A (pinned against brute force in test_gpu_descending.py).
    k, v = oracle.merge(b[::-1].copy(), a[::-1].copy(), bv[::-1].copy(), av[::-1].copy())
    return k[::-1].copy(), v[::-1].copy()


def _check(a, b, dt, plan, desc=False):
    av = np.arange(a.size, dtype=np.uint32)
    bv = np.arange(a.size, a.size + b.size, dtype=np.uint32)
    ek, ev = _expect(a, b, av, bv, desc)
    ok, ov = mp.mp_merge_plan(to_dev(a), to_dev(b), vals_to_dev(av), vals_to_dev(bv), plan=plan,
                              descending=desc)
    assert first_mismatch(to_host(ok, dt), ek) is None, (a.size, b.size, plan)
    assert first_mismatch(to_host(ov, np.uint32), ev) is None, (a.size, b.size, plan)
    ko = mp.mp_merge_plan(to_dev(a), to_dev(b), plan=plan, descending=desc)
    assert first_mismatch(to_host(ko, dt), ek) is None, (a.size, b.size, plan)


def test_stream_shapes_compiled():
    assert len(_shapes()) >= 3


@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
def test_stream_every_shape(dt):
    rng = np.random.default_rng(1300 + DTYPES.index(dt))
    for plan in _shapes():
        for na, nb, kind in [(1, 1, "ties"), (5, 3, "random"), (4095, 1, "ties"), (30_011, 17_003, "ties"),
                             (262_144, 262_144, "random"), (7, 100_000, "ties"),
                             (2_000_000, 1_500_001, "ties")]:
            _check(random_sorted(rng, dt, na, kind), random_sorted(rng, dt, nb, kind), dt, plan)
    assert mp.mp_kernel_error(reset=True) == 0


@pytest.mark.parametrize("dt", [np.int32, np.uint64, np.float32], ids=lambda d: np.dtype(d).name)
def test_stream_edge_sizes(dt):
    """Empty sides, inputs shorter than a 16-byte granule, one side used up
    for many tiles (every A above every B; all keys equal), shares of many
    tiles per CTA."""
    rng = np.random.default_rng(1350)
    for plan in _shapes()[:3]:
        for na, nb in [(1, 0), (0, 1), (3, 2), (5, 17), (0, 300_001), (1_000_003, 0), (3, 4_000_000)]:
            _check(random_sorted(rng, dt, na, "ties"), random_sorted(rng, dt, nb, "ties"), dt, plan)
        for na, nb in [(1_500_000, 2_500_007), (4096, 3_000_000)]:
            b = random_sorted(rng, dt, nb, "ties")
            a = np.full(na, np.array([100], dtype=dt)[0], dtype=dt)
            _check(a, b, dt, plan)          # all of B first, then all of A
            eq = np.full(nb, np.array([7], dtype=dt)[0], dtype=dt)
            _check(eq[:na].copy(), eq, dt, plan)  # all keys equal: A, then B
    assert mp.mp_kernel_error(reset=True) == 0


@pytest.mark.parametrize("dt", [np.int32, np.uint64, np.float32], ids=lambda d: np.dtype(d).name)
def test_stream_unaligned_pointers(dt):
    rng = np.random.default_rng(1400)
    plan = _shapes()[0]
    for off_a, off_b, off_o in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 3, 2), (3, 2, 1)]:
        na, nb = 1_200_011, 909_007
        a, b = random_sorted(rng, dt, na, "ties"), random_sorted(rng, dt, nb, "ties")
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        A = to_dev(np.concatenate([np.zeros(off_a, dt), a]))[off_a:]
        B = to_dev(np.concatenate([np.zeros(off_b, dt), b]))[off_b:]
        AV = vals_to_dev(np.concatenate([np.zeros(off_a, np.uint32), av]))[off_a:]
        BV = vals_to_dev(np.concatenate([np.zeros(off_b, np.uint32), bv]))[off_b:]
        OK = torch.empty(na + nb + off_o, dtype=A.dtype, device="cuda")[off_o:]
        OV = torch.empty(na + nb + off_o, dtype=torch.int32, device="cuda")[off_o:]
        mp.mp_merge_plan(A, B, AV, BV, OK, OV, plan=plan)
        ek, ev = oracle.merge(a, b, av, bv)
        assert first_mismatch(to_host(OK, dt), ek) is None, (off_a, off_b, off_o)
        assert first_mismatch(to_host(OV, np.uint32), ev) is None, (off_a, off_b, off_o)


@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
def test_stream_descending(dt):
    rng = np.random.default_rng(1450)
    for plan in _shapes()[:2]:
        for na, nb in [(70_001, 33_333), (1_000_000, 1_400_003)]:
            a = random_sorted(rng, dt, na, "ties")[::-1].copy()
            b = random_sorted(rng, dt, nb, "ties")[::-1].copy()
            _check(a, b, dt, plan, desc=True)


def test_stream_graph_and_partitioned():
    rng = np.random.default_rng(1500)
    a, b = random_sorted(rng, np.uint64, 800_000, "ties"), random_sorted(rng, np.uint64, 600_001, "ties")
    A, B = to_dev(a), to_dev(b)
    out = torch.empty(a.size + b.size, dtype=A.dtype, device="cuda")
    plan = _shapes()[0]
    g = mp.mp_graph_merge_create(A, B, out, plan=plan)
    try:
        g.replay()
        g.replay()
        torch.cuda.synchronize()
    finally:
        g.close()
    ek, _ = oracle.merge(a, b)
    assert first_mismatch(to_host(out, np.uint64), ek) is None
    # The streaming plan takes no split points.
    splits = mp.mp_merge_path_partition(A, B, 1024)
    with pytest.raises(mp.MPError) as ei:
        mp.mp_merge_partitioned(A, B, splits, plan=plan)
    assert ei.value.status == mp.MP_ERR_INVALID_ARG
