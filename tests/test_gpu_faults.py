"""Error paths, exercised with faults made on the host or with a device wait
that runs out on purpose (never a GPU fault): a TMA staging wait that gives
up, a scratch allocation that fails, a request-queue step that fails to
launch.  After each, the library must report the right status and the next
call must again be bit-exact against the oracle."""
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


@pytest.fixture(autouse=True)
def _no_faults_left():
    yield
    mp.mp_inject_fault(mp.MP_FAULT_STAGE_WAIT, 0)
    mp.mp_inject_fault(mp.MP_FAULT_SCRATCH_ALLOC, 0)
    mp.mp_inject_fault(mp.MP_FAULT_QUEUE_STEP, 0)
    mp.mp_kernel_error(reset=True)


def _case(seed, na=90_001, nb=70_003, dt=np.int32):
    rng = np.random.default_rng(seed)
    a, b = random_sorted(rng, dt, na, "ties"), random_sorted(rng, dt, nb, "ties")
    return a, b


# TMA-staged tile plans: the only kernels whose first wait the switch affects.
_BULK_PLANS = [(256, 12, mp.MP_STAGE_BULK), (128, 33, mp.MP_STAGE_BULK)]


@pytest.mark.parametrize("plan", _BULK_PLANS, ids=["256x12", "128x33"])
def test_stage_wait_that_runs_out_is_reported_then_recovers(plan):
    a, b = _case(5000)
    expect, _ = oracle.merge(a, b)
    A, B = to_dev(a), to_dev(b)
    assert mp.mp_kernel_error(reset=True) == 0
    mp.mp_inject_fault(mp.MP_FAULT_STAGE_WAIT, 1)
    out = torch.full((a.size + b.size,), -1, dtype=torch.int32, device="cuda")
    mp.mp_merge_plan(A, B, out_keys=out, plan=plan)
    # Every tile gave up before merging: flag 1 is set, the status says so,
    # and no tile wrote its output.
    assert mp.mp_kernel_error() & 1
    assert mp.mp_kernel_status(reset=False) == mp.MP_ERR_TIMEOUT
    assert "ran out" in mp.mp_last_error()
    assert bool((out == -1).all())
    # Switch off, clear the flags: the same merge is exact again.
    mp.mp_inject_fault(mp.MP_FAULT_STAGE_WAIT, 0)
    assert mp.mp_kernel_status(reset=True) == mp.MP_ERR_TIMEOUT
    assert mp.mp_kernel_error() == 0
    out = mp.mp_merge_plan(A, B, plan=plan)
    assert mp.mp_kernel_status() == mp.MP_OK
    assert first_mismatch(to_host(out, np.int32), expect) is None


def test_stage_wait_switch_leaves_batched_and_setop_paths_reporting():
    # The batched merge and the set operations stage their tiles the same
    # way; with the switch on they report flag 1 too and recover after.
    a, b = _case(5001, 50_000, 40_000, np.uint32)
    A, B = to_dev(a), to_dev(b)
    mp.mp_inject_fault(mp.MP_FAULT_STAGE_WAIT, 1)
    mp.mp_set_operation("union", A, B, trim=False)
    assert mp.mp_kernel_status(reset=True) == mp.MP_ERR_TIMEOUT
    a_off = torch.tensor([0, 30_000, a.size], dtype=torch.int64, device="cuda")
    b_off = torch.tensor([0, 10_000, b.size], dtype=torch.int64, device="cuda")
    mp.mp_merge_batched(A, a_off, B, b_off)
    assert mp.mp_kernel_status(reset=True) == mp.MP_ERR_TIMEOUT
    mp.mp_inject_fault(mp.MP_FAULT_STAGE_WAIT, 0)
    out, _, _ = mp.mp_set_operation("union", A, B)
    ek, _ = oracle.set_op("union", a, b)
    assert mp.mp_kernel_status() == mp.MP_OK
    assert first_mismatch(to_host(out, np.uint32), ek) is None
    got = mp.mp_merge_batched(A, a_off, B, b_off)
    ek, _ = oracle.merge_batched(a, np.array([0, 30_000, a.size]), b, np.array([0, 10_000, b.size]))
    assert first_mismatch(to_host(got, np.uint32), ek) is None


def test_scratch_allocation_failure_returns_no_memory():
    a, b = _case(5002, 300_000, 200_000)
    A, B = to_dev(a), to_dev(b)
    out = torch.empty(a.size + b.size, dtype=torch.int32, device="cuda")
    mp.mp_inject_fault(mp.MP_FAULT_SCRATCH_ALLOC, 1)
    with pytest.raises(mp.MPError) as ei:
        mp.mp_merge_plan(A, B, out_keys=out, plan=(128, 33, mp.MP_STAGE_BULK))
    assert ei.value.status == mp.MP_ERR_NO_MEMORY
    assert "injected" in mp.mp_last_error()
    # The fault was used up: the next call allocates and merges exactly.
    mp.mp_merge_plan(A, B, out_keys=out, plan=(128, 33, mp.MP_STAGE_BULK))
    expect, _ = oracle.merge(a, b)
    assert first_mismatch(to_host(out, np.int32), expect) is None
    # A set operation's scratch (splits, counts, offsets) comes from the
    # same pool.
    mp.mp_inject_fault(mp.MP_FAULT_SCRATCH_ALLOC, 1)
    with pytest.raises(mp.MPError) as ei:
        mp.mp_set_operation("intersection", A, B, trim=False)
    assert ei.value.status == mp.MP_ERR_NO_MEMORY
    got, _, _ = mp.mp_set_operation("intersection", A, B)
    ek, _ = oracle.set_op("intersection", a, b)
    assert first_mismatch(to_host(got, np.int32), ek) is None


def test_queue_step_failure_is_reported_on_its_ticket():
    rng = np.random.default_rng(5004)
    a, b = random_sorted(rng, np.uint32, 100_000, "ties"), random_sorted(rng, np.uint32, 80_000, "ties")
    ta = torch.from_numpy(a.view(np.int32)).view(torch.uint32)
    tb = torch.from_numpy(b.view(np.int32)).view(torch.uint32)
    with mp.Queue(budget_bytes=64 << 20, max_active=8) as q:
        mp.mp_inject_fault(mp.MP_FAULT_QUEUE_STEP, 1)
        out1 = torch.empty(a.size + b.size, dtype=torch.uint32)
        t1 = q.submit_merge(ta, tb, out1)
        r1 = q.wait(t1, timeout_s=60)
        assert r1.status == mp.MP_ERR_CUDA
        st = q.stats()
        assert st["failed"] == 1 and st["completed"] == 1
        # The queue keeps serving: the next request is exact.
        out2 = torch.empty(a.size + b.size, dtype=torch.uint32)
        t2 = q.submit_merge(ta, tb, out2)
        r2 = q.wait(t2, timeout_s=60)
        assert r2.status == mp.MP_OK
        expect, _ = oracle.merge(a, b)
        assert first_mismatch(out2.view(torch.int32).numpy().view(np.uint32), expect) is None
        st = q.stats()
        assert st["failed"] == 1 and st["completed"] == 2
