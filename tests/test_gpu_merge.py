"""GPU parity of the merge path (partition + merge-tile kernels) against the
CPU oracle: bit-exact, every dtype, sizes spanning several tiles with ragged
tails, the edge cases (empty inputs, one element, every A above every B, all
keys equal, unaligned pointers) and every compiled tile plan.  All calls go
through the C ABI (libmp.so) via the Python binding."""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_2628_gb300 as mp
from _util import first_mismatch, random_sorted, to_dev, to_host, vals_to_dev

pytestmark = pytest.mark.gpu

DTYPES = [np.int32, np.uint32, np.float32, np.uint64, np.int64]
SIZES = [(0, 0), (1, 0), (0, 1), (1, 1), (5, 3), (4095, 1), (4096, 4096), (12_305, 8_209),
         (70_001, 33_333), (100_000, 0), (0, 65_537), (3, 200_000)]
PLANS = [(128, 8), (256, 8), (128, 16), (256, 16), (512, 8),
         (128, 8, mp.MP_STAGE_BULK), (256, 8, mp.MP_STAGE_BULK), (128, 16, mp.MP_STAGE_BULK),
         (256, 16, mp.MP_STAGE_BULK), (128, 12, mp.MP_STAGE_BULK), (256, 12, mp.MP_STAGE_BULK),
         (128, 27, mp.MP_STAGE_BULK), (128, 33, mp.MP_STAGE_BULK), (256, 33, mp.MP_STAGE_BULK),
         (128, 8, mp.MP_STAGE_WARP), (256, 8, mp.MP_STAGE_WARP), (128, 16, mp.MP_STAGE_WARP),
         (256, 16, mp.MP_STAGE_WARP)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mp.lib()
    torch.cuda.init()


def _case(rng, dt, na, nb, kind):
    if kind == "a_gt_b":
        b = random_sorted(rng, dt, nb, "ties") if nb else np.empty(0, dt)
        hi = np.array([100], dtype=dt)[0]
        a = np.full(na, hi, dtype=dt)
        return a, b
    return random_sorted(rng, dt, na, kind), random_sorted(rng, dt, nb, kind)


@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
@pytest.mark.parametrize("kind", ["random", "ties", "equal", "a_gt_b"])
def test_merge_keys(dt, kind):
    rng = np.random.default_rng(100 + DTYPES.index(dt))
    for na, nb in SIZES:
        a, b = _case(rng, dt, na, nb, kind)
        out = mp.mp_merge_keys(to_dev(a), to_dev(b))
        expect, _ = oracle.merge(a, b)
        got = to_host(out, dt)
        assert first_mismatch(got, expect) is None, (na, nb, first_mismatch(got, expect))


@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
@pytest.mark.parametrize("kind", ["random", "ties", "a_gt_b"])
def test_merge_pairs(dt, kind):
    rng = np.random.default_rng(200 + DTYPES.index(dt))
    for na, nb in SIZES:
        a, b = _case(rng, dt, na, nb, kind)
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        ok, ov = mp.mp_merge_pairs(to_dev(a), vals_to_dev(av), to_dev(b), vals_to_dev(bv))
        ek, ev = oracle.merge(a, b, av, bv)
        assert first_mismatch(to_host(ok, dt), ek) is None, (na, nb)
        assert first_mismatch(to_host(ov, np.uint32), ev) is None, (na, nb)


@pytest.mark.parametrize("plan", PLANS, ids=str)
@pytest.mark.parametrize("dt", [np.int32, np.float32, np.uint64], ids=lambda d: np.dtype(d).name)
def test_merge_every_plan(plan, dt):
    rng = np.random.default_rng(300)
    for na, nb in [(1, 1), (30_011, 17_003), (262_144, 262_144), (7, 100_000)]:
        a, b = random_sorted(rng, dt, na, "ties"), random_sorted(rng, dt, nb, "ties")
        av = rng.integers(0, 1 << 32, na, dtype=np.uint64).astype(np.uint32)
        bv = rng.integers(0, 1 << 32, nb, dtype=np.uint64).astype(np.uint32)
        ok = mp.mp_merge_plan(to_dev(a), to_dev(b), plan=plan)
        ek, _ = oracle.merge(a, b)
        assert first_mismatch(to_host(ok, dt), ek) is None
        ok, ov = mp.mp_merge_plan(to_dev(a), to_dev(b), vals_to_dev(av), vals_to_dev(bv), plan=plan)
        ek, ev = oracle.merge(a, b, av, bv)
        assert first_mismatch(to_host(ok, dt), ek) is None
        assert first_mismatch(to_host(ov, np.uint32), ev) is None


@pytest.mark.parametrize("plan", [None, (128, 8, mp.MP_STAGE_BULK), (256, 16, mp.MP_STAGE_BULK),
                                  (256, 8, mp.MP_STAGE_WARP)], ids=str)
@pytest.mark.parametrize("dt", [np.int32, np.uint64, np.float32], ids=lambda d: np.dtype(d).name)
def test_unaligned_pointers(dt, plan):
    """Windows and outputs at every 16-byte phase: sub-views offset by one
    element exercise the scalar head/tail staging and the scalar store path."""
    rng = np.random.default_rng(400)
    for off_a, off_b, off_o in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 3, 2), (3, 2, 1)]:
        na, nb = 20_011, 9_007
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
def test_partition_matches_oracle_split(dt):
    """mp_merge_path_partition vs the oracle's Alg. 2 at every requested
    diagonal, including spacing 1 (every diagonal) on small inputs."""
    rng = np.random.default_rng(500)
    for na, nb, spacing in [(0, 5, 1), (7, 0, 2), (33, 47, 1), (1000, 10, 3), (5000, 7000, 257),
                            (100_000, 100_000, 4096)]:
        a, b = random_sorted(rng, dt, na, "ties"), random_sorted(rng, dt, nb, "ties")
        got = mp.mp_merge_path_partition(to_dev(a), to_dev(b), spacing).cpu().numpy()
        n = na + nb
        diags = [min(t * spacing, n) for t in range((n + spacing - 1) // spacing + 1)]
        expect = [oracle.split(a, b, d)[0] for d in diags]
        assert got.tolist() == expect


@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
def test_bulk_staging_edge_sizes(dt):
    """TMA-staged persistent merge: empty sides, windows shorter than one
    16-byte granule, many tiles per CTA (large inputs), and no kernel error
    reported by its bounded waits."""
    rng = np.random.default_rng(550)
    for na, nb in [(1, 0), (0, 1), (1, 1), (3, 2), (5, 17), (4096, 1), (2_000_000, 1_500_001),
                   (0, 300_001), (1_000_003, 0)]:
        a, b = random_sorted(rng, dt, na, "ties"), random_sorted(rng, dt, nb, "ties")
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        for plan in [(128, 8, mp.MP_STAGE_BULK), (256, 16, mp.MP_STAGE_BULK),
                     (128, 8, mp.MP_STAGE_WARP), (256, 16, mp.MP_STAGE_WARP)]:
            ok, ov = mp.mp_merge_plan(to_dev(a), to_dev(b), vals_to_dev(av), vals_to_dev(bv), plan=plan)
            ek, ev = oracle.merge(a, b, av, bv)
            assert first_mismatch(to_host(ok, dt), ek) is None, (na, nb, plan)
            assert first_mismatch(to_host(ov, np.uint32), ev) is None, (na, nb, plan)
            ko = mp.mp_merge_plan(to_dev(a), to_dev(b), plan=plan)
            assert first_mismatch(to_host(ko, dt), ek) is None, (na, nb, plan)
    assert mp.mp_kernel_error(reset=True) == 0


def test_merge_on_side_stream():
    rng = np.random.default_rng(600)
    a, b = random_sorted(rng, np.int32, 300_000), random_sorted(rng, np.int32, 200_000)
    s = torch.cuda.Stream()
    A, B = to_dev(a), to_dev(b)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        out = mp.mp_merge_keys(A, B)
    s.synchronize()
    expect, _ = oracle.merge(a, b)
    assert np.array_equal(out.cpu().numpy(), expect)


def test_check_sorted():
    x = torch.arange(1000, dtype=torch.int32, device="cuda")
    assert mp.mp_check_sorted(x) == mp.MP_OK
    x[500] = -5
    assert mp.mp_check_sorted(x) == mp.MP_ERR_NOT_SORTED
    f = torch.tensor([-1.0, -0.0, 0.0, 1.0], device="cuda")
    assert mp.mp_check_sorted(f) == mp.MP_OK
    f2 = torch.tensor([-1.0, 0.0, -0.0, 1.0], device="cuda")
    assert mp.mp_check_sorted(f2) == mp.MP_ERR_NOT_SORTED
    f3 = torch.tensor([-1.0, float("nan"), 1.0], device="cuda")
    assert mp.mp_check_sorted(f3) == mp.MP_ERR_NAN
    u = torch.tensor([1, 2, 3], dtype=torch.int64, device="cuda").view(torch.uint64)
    assert mp.mp_check_sorted(u) == mp.MP_OK


def test_device_errors_are_status_codes():
    a = torch.arange(10, dtype=torch.int32, device="cuda")
    with pytest.raises(mp.MPError) as ei:
        mp.mp_merge_keys(a, a[2:], out=a)  # output overlaps the inputs
    assert ei.value.status == mp.MP_ERR_INVALID_ARG
    with pytest.raises(mp.MPError) as ei:
        mp.mp_merge_plan(a, a, plan=(100, 3))
    assert ei.value.status == mp.MP_ERR_INVALID_ARG
