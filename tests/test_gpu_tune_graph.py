"""GPU tests of the autotuner and of the CUDA-graph objects."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1406_2628_gb300 as mp
from _util import first_mismatch, random_sorted, to_dev, to_host, vals_to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _clean_tune_table():
    mp.lib()
    mp.mp_tune_clear()
    yield
    mp.mp_tune_clear()


def test_autotune_merge_records_a_compiled_plan(tmp_path):
    rng = np.random.default_rng(1300)
    a, b = random_sorted(rng, np.uint64, 1 << 20, "ties"), random_sorted(rng, np.uint64, 1 << 19, "ties")
    av = np.arange(a.size, dtype=np.uint32)
    bv = np.arange(a.size, a.size + b.size, dtype=np.uint32)
    A, B, AV, BV = to_dev(a), to_dev(b), vals_to_dev(av), vals_to_dev(bv)
    n = a.size + b.size
    default_tile = mp.mp_merge_tile_items(torch.uint64, True, n)
    nt, vt, stg = mp.mp_autotune_merge(A, B, AV, BV, reps=2)
    assert mp.mp_plan_supported((nt, vt, stg))
    # A streaming winner uses no split points, so the partitioned tile stays.
    tuned_tile = default_tile if stg == mp.MP_STAGE_STREAM else nt * vt
    assert mp.mp_merge_tile_items(torch.uint64, True, n) == tuned_tile
    # Automatic plans now use the tuned shape and still merge exactly.
    ok, ov = mp.mp_merge_pairs(A, AV, B, BV)
    ek, ev = oracle.merge(a, b, av, bv)
    assert first_mismatch(to_host(ok, np.uint64), ek) is None
    assert first_mismatch(to_host(ov, np.uint32), ev) is None
    # Save / clear / load round trip.
    path = str(tmp_path / "tune.txt")
    mp.mp_tune_save(path)
    mp.mp_tune_clear()
    assert mp.mp_merge_tile_items(torch.uint64, True, n) == default_tile
    mp.mp_tune_load(path)
    assert mp.mp_merge_tile_items(torch.uint64, True, n) == tuned_tile


def test_autotune_batched():
    a, a_off, b, b_off = gen.batched(n_seg=512, log2_max=12.0)
    A, AO, B, BO = to_dev(a), to_dev(a_off), to_dev(b), to_dev(b_off)
    nt, vt, stg = mp.mp_autotune_batched(A, AO, B, BO, reps=2)
    assert nt * vt > 0
    out = mp.mp_merge_batched(A, AO, B, BO)
    ek, _ = oracle.merge_batched(a, a_off, b, b_off)
    assert np.array_equal(out.cpu().numpy(), ek)


def test_graph_merge_replays_with_new_contents():
    rng = np.random.default_rng(1400)
    na, nb = 300_001, 123_457
    A = torch.empty(na, dtype=torch.float32, device="cuda")
    B = torch.empty(nb, dtype=torch.float32, device="cuda")
    AV = torch.empty(na, dtype=torch.int32, device="cuda")
    BV = torch.empty(nb, dtype=torch.int32, device="cuda")
    OK = torch.empty(na + nb, dtype=torch.float32, device="cuda")
    OV = torch.empty(na + nb, dtype=torch.int32, device="cuda")
    g = mp.mp_graph_merge_create(A, B, OK, AV, BV, OV)
    for rep in range(3):
        a, b = random_sorted(rng, np.float32, na, "ties"), random_sorted(rng, np.float32, nb, "ties")
        av = rng.integers(0, 1 << 32, na, dtype=np.uint64).astype(np.uint32)
        bv = rng.integers(0, 1 << 32, nb, dtype=np.uint64).astype(np.uint32)
        A.copy_(to_dev(a)); B.copy_(to_dev(b)); AV.copy_(vals_to_dev(av)); BV.copy_(vals_to_dev(bv))
        g.replay()
        torch.cuda.synchronize()
        ek, ev = oracle.merge(a, b, av, bv)
        assert first_mismatch(OK.cpu().numpy(), ek) is None, rep
        assert first_mismatch(OV.cpu().numpy().view(np.uint32), ev) is None, rep
    g.close()


def test_graph_batched_replay():
    a, a_off, b, b_off = gen.batched(n_seg=1000, log2_max=11.0)
    A, AO, B, BO = to_dev(a), to_dev(a_off), to_dev(b), to_dev(b_off)
    OUT = torch.empty(a.size + b.size, dtype=torch.int32, device="cuda")
    g = mp.mp_graph_batched_create(A, AO, B, BO, OUT)
    ek, _ = oracle.merge_batched(a, a_off, b, b_off)
    for _ in range(3):
        OUT.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(OUT.cpu().numpy(), ek)
    g.close()


def test_resolve_plan_reports_the_shape_that_runs():
    big = 335_544_320
    assert mp.mp_merge_resolve_plan(torch.uint64, True, big) == (256, 12, mp.MP_STAGE_BULK)
    assert mp.mp_merge_resolve_plan(torch.int32, False, big) == (128, 33, mp.MP_STAGE_BULK)
    assert mp.mp_merge_resolve_plan(torch.int64, False, big) == (128, 27, mp.MP_STAGE_BULK)
    small = mp.mp_merge_resolve_plan(torch.int32, False, 1 << 20)
    assert small[2] == mp.MP_STAGE_STREAM
    assert mp.mp_merge_resolve_plan(torch.uint64, True, big, (128, 8, mp.MP_STAGE_BULK)) == (128, 8, mp.MP_STAGE_BULK)
    tile = mp.mp_merge_tile_items(torch.uint64, True, big)
    assert tile == 256 * 12
    with pytest.raises(mp.MPError):
        mp.mp_merge_resolve_plan(torch.uint64, True, big, (100, 3))
