"""GPU tests of the grouped merge and of the continuous-batching request
queue: every result equals the oracle's, and equals the same request run
alone (tolerance 0: merging and sorting are exact)."""
import time

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1406_2628_gb300 as mp
from _util import first_mismatch, random_sorted, to_dev, to_host, vals_to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mp.lib()
    torch.cuda.init()


# ----------------------------------------------------------------- grouped

@pytest.mark.parametrize("dts", [(np.int32, np.float32, np.uint32), (np.uint64, np.int64)],
                         ids=["w4", "w8"])
@pytest.mark.parametrize("vals", [False, True])
@pytest.mark.parametrize("prepared", [False, True], ids=["tuples", "descs"])
def test_merge_grouped(dts, vals, prepared):
    rng = np.random.default_rng(1000)
    probs, expect = [], []
    sizes = [(0, 0), (1, 0), (0, 7), (5000, 3), (12_345, 54_321), (4096, 4096), (1, 1), (70_000, 1)]
    for i, (na, nb) in enumerate(sizes):
        dt = dts[i % len(dts)]
        a, b = random_sorted(rng, dt, na, "ties"), random_sorted(rng, dt, nb, "ties")
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        A, B = to_dev(a), to_dev(b)
        OK = torch.empty(na + nb, dtype=A.dtype, device="cuda")
        if vals:
            OV = torch.empty(na + nb, dtype=torch.int32, device="cuda")
            probs.append((A, vals_to_dev(av), B, vals_to_dev(bv), OK, OV))
            expect.append((dt, *oracle.merge(a, b, av, bv)))
        else:
            probs.append((A, B, OK))
            expect.append((dt, *oracle.merge(a, b)))
    if prepared:
        mp.mp_merge_grouped(mp.mp_merge_grouped_descs(probs, with_values=vals), with_values=vals)
    else:
        mp.mp_merge_grouped(probs, with_values=vals)
    torch.cuda.synchronize()
    for pr, (dt, ek, ev) in zip(probs, expect):
        assert first_mismatch(to_host(pr[-2] if vals else pr[-1], dt), ek) is None
        if vals:
            assert first_mismatch(to_host(pr[-1], np.uint32), ev) is None


# ----------------------------------------------------------------- queue

def _host_merge_case(rng, dt, na, nb):
    a, b = random_sorted(rng, dt, na, "ties"), random_sorted(rng, dt, nb, "ties")
    av = np.arange(na, dtype=np.uint32)
    bv = np.arange(na, na + nb, dtype=np.uint32)
    return a, av, b, bv


def _t(x):
    """numpy -> contiguous CPU tensor with the same bits."""
    if x.dtype == np.uint64:
        return torch.from_numpy(x.view(np.int64)).view(torch.uint64)
    if x.dtype == np.uint32:
        return torch.from_numpy(x.view(np.int32)).view(torch.uint32)
    return torch.from_numpy(x)


def test_queue_mixed_requests_match_oracle_and_alone():
    rng = np.random.default_rng(1100)
    reqs = []
    with mp.Queue(budget_bytes=256 << 20, max_active=64) as q:
        for i in range(40):
            dt = [np.int32, np.uint32, np.float32, np.uint64, np.int64][i % 5]
            if i % 3 == 2:
                n = int(rng.integers(0, 200_000))
                k = random_sorted(rng, dt, n, "ties")[rng.permutation(n)]
                v = np.arange(n, dtype=np.uint32)
                ok = torch.empty(n, dtype=_t(k).dtype)
                ov = torch.empty(n, dtype=torch.int32)
                t = q.submit_sort(_t(k), ok, _t(v), ov)
                reqs.append(("sort", t, dt, (k, v), ok, ov))
            else:
                na, nb = int(rng.integers(0, 150_000)), int(rng.integers(0, 150_000))
                a, av, b, bv = _host_merge_case(rng, dt, na, nb)
                ok = torch.empty(na + nb, dtype=_t(a).dtype)
                ov = torch.empty(na + nb, dtype=torch.int32)
                t = q.submit_merge(_t(a), _t(b), ok, _t(av), _t(bv), ov)
                reqs.append(("merge", t, dt, (a, av, b, bv), ok, ov))
        for kind, t, dt, inp, ok, ov in reqs:
            r = q.wait(t, timeout_s=120)
            assert r.status == mp.MP_OK
            assert r.t_submit <= r.t_admit <= r.t_done
            got_k = ok.view(torch.int64 if np.dtype(dt).itemsize == 8 else torch.int32).numpy().view(dt)
            got_v = ov.numpy().view(np.uint32)
            if kind == "sort":
                ek, ev = oracle.sort(inp[0], inp[1])
            else:
                ek, ev = oracle.merge(inp[0], inp[2], inp[1], inp[3])
            assert first_mismatch(got_k, ek) is None, kind
            assert first_mismatch(got_v, ev) is None, kind
            # The same request alone through the plain API gives the same bits.
            if kind == "merge" and inp[0].size + inp[2].size > 0:
                alone_k, alone_v = mp.mp_merge_pairs(to_dev(inp[0]), vals_to_dev(inp[1]),
                                                     to_dev(inp[2]), vals_to_dev(inp[3]))
                assert first_mismatch(to_host(alone_k, dt), got_k) is None
                assert first_mismatch(to_host(alone_v, np.uint32), got_v) is None
            if kind == "sort" and inp[0].size > 0:
                tk, tv = to_dev(inp[0]), vals_to_dev(inp[1])
                mp.mp_sort(tk, tv)
                assert first_mismatch(to_host(tk, dt), got_k) is None
                assert first_mismatch(to_host(tv, np.uint32), got_v) is None
        st = q.stats()
        assert st["completed"] == 40 and st["failed"] == 0
        assert st["peak_bytes"] <= 256 << 20


def test_queue_device_buffers_and_keys_only():
    rng = np.random.default_rng(1200)
    a, b = random_sorted(rng, np.int32, 100_000, "ties"), random_sorted(rng, np.int32, 77_777, "ties")
    A, B = to_dev(a), to_dev(b)
    out = torch.empty(a.size + b.size, dtype=torch.int32, device="cuda")
    k = random_sorted(rng, np.float32, 60_001, "ties")[rng.permutation(60_001)]
    K = to_dev(k)
    sout = torch.empty_like(K)
    with mp.Queue(budget_bytes=64 << 20) as q:
        t1 = q.submit_merge(A, B, out)
        t2 = q.submit_sort(K, sout)
        assert q.wait(t1).status == mp.MP_OK
        assert q.wait(t2).status == mp.MP_OK
    assert np.array_equal(out.cpu().numpy(), oracle.merge(a, b)[0])
    assert first_mismatch(sout.cpu().numpy(), oracle.sort(k)[0]) is None


def test_queue_generated_requests_and_budget_pressure():
    """Generated inputs (device generator) checked with the generator's host
    restatement and the oracle; a small budget forces requests to wait for
    memory, and every result is still exact."""
    budget = 24 << 20
    specs = [("merge", 300_000, 200_000), ("sort", 250_000, 0), ("merge", 1, 0), ("sort", 70_000, 0),
             ("merge", 500_000, 123), ("sort", 2, 0), ("merge", 0, 40_000)]
    with mp.Queue(budget_bytes=budget, max_active=8) as q:
        ts = []
        for i, (op, na, nb) in enumerate(specs):
            n = na + nb
            ok = torch.empty(n, dtype=torch.int32)
            ov = torch.empty(n, dtype=torch.int32)
            t = q.submit_generated(mp.MP_OP_MERGE if op == "merge" else mp.MP_OP_SORT, mp.MP_U32,
                                   na, nb, seed=77 + i, with_values=True, out_keys=ok, out_vals=ov)
            ts.append((t, op, na, nb, 77 + i, ok, ov))
        for t, op, na, nb, seed, ok, ov in ts:
            assert q.wait(t, timeout_s=120).status == mp.MP_OK
            if op == "merge":
                a, av, b, bv = gen.serving_request("merge", na, nb, seed)
                ek, ev = oracle.merge(a, b, av, bv)
            else:
                k, v = gen.serving_request("sort", na, 0, seed)
                ek, ev = oracle.sort(k, v)
            assert first_mismatch(ok.numpy().view(np.uint32), ek) is None, (op, na, nb)
            assert first_mismatch(ov.numpy().view(np.uint32), ev) is None, (op, na, nb)
        st = q.stats()
        assert st["peak_bytes"] <= budget


def test_queue_rejects_request_over_budget_and_bad_args():
    with mp.Queue(budget_bytes=1 << 20) as q:
        with pytest.raises(mp.MPError) as ei:
            q.submit_generated(mp.MP_OP_MERGE, mp.MP_U32, 1 << 20, 1 << 20, seed=1)
        assert ei.value.status == mp.MP_ERR_BUDGET
        with pytest.raises(mp.MPError) as ei:
            q.submit_generated(mp.MP_OP_MERGE, mp.MP_F32, 10, 10, seed=1)
        assert ei.value.status == mp.MP_ERR_INVALID_ARG
        with pytest.raises(mp.MPError) as ei:
            mp.mp_queue_wait(q.handle, 987654321, 0)
        assert ei.value.status == mp.MP_ERR_INVALID_ARG


def test_queue_bounded_wait_times_out_then_completes():
    """A wait shorter than the work returns MP_ERR_TIMEOUT (or NOT_READY for
    a poll) and leaves the request running; a later wait collects it."""
    with mp.Queue(budget_bytes=2 << 30) as q:
        t = q.submit_generated(mp.MP_OP_SORT, mp.MP_U64, 1 << 25, 0, seed=5)
        with pytest.raises(mp.MPError) as ei:
            mp.mp_queue_wait(q.handle, t, 0)
        assert ei.value.status in (mp.MP_ERR_NOT_READY,)
        with pytest.raises(mp.MPError) as ei:
            mp.mp_queue_wait(q.handle, t, 1000)  # 1 microsecond
        assert ei.value.status == mp.MP_ERR_TIMEOUT
        assert q.wait(t, timeout_s=120).status == mp.MP_OK


def test_queue_continuous_batching_overlaps_requests():
    """Requests submitted while others run are admitted and batched into the
    same steps: fewer steps than the sum of the requests' stages."""
    with mp.Queue(budget_bytes=2 << 30, max_active=256) as q:
        ts = [q.submit_generated(mp.MP_OP_SORT if i % 2 else mp.MP_OP_MERGE, mp.MP_U32,
                                 1 << 18, 0 if i % 2 else 1 << 18, seed=i) for i in range(64)]
        for t in ts:
            assert q.wait(t, timeout_s=120).status == mp.MP_OK
        st = q.stats()
    # 32 merges (1 stage each) + 32 sorts (1 + 6 stages each) = 256 stages.
    assert st["steps"] < 256


@pytest.mark.slow
def test_queue_serving_distribution_at_bench_sizes():
    """About 200 generated requests from the serving recipe (70 % merges,
    30 % sorts, uint32 keys + uint32 values, sizes log-uniform in
    [2^10, 2^24]) plus three merges and three sorts of 2^22..2^24 per side,
    all submitted at once under a 1 GiB budget so that large multi-pass
    sorts advance step by step beside other requests.  Every result against
    the generator's host restatement run through the oracle, and against the
    same request run alone through the plain calls; the budget holds."""
    budget = 1 << 30
    rng = np.random.default_rng(0x5E7)
    specs = []
    for i in range(194):
        is_sort = rng.random() < 0.3
        na = int(np.floor(2.0 ** (10 + 14 * rng.random())))
        nb = 0 if is_sort else int(np.floor(2.0 ** (10 + 14 * rng.random())))
        specs.append(("sort" if is_sort else "merge", na, nb))
    big = [("merge", 1 << 24, 1 << 22), ("sort", 1 << 24, 0), ("merge", 3 << 21, 1 << 24),
           ("sort", (1 << 22) + 12345, 0), ("merge", 1 << 22, (1 << 23) + 1), ("sort", 3 << 22, 0)]
    for j, s in enumerate(big):
        specs.insert(20 + 30 * j, s)
    with mp.Queue(budget_bytes=budget, max_active=64) as q:
        ts = []
        for i, (op, na, nb) in enumerate(specs):
            n = na + nb
            ok = torch.empty(n, dtype=torch.int32)
            ov = torch.empty(n, dtype=torch.int32)
            seed = 9000 + i
            t = q.submit_generated(mp.MP_OP_MERGE if op == "merge" else mp.MP_OP_SORT, mp.MP_U32,
                                   na, nb, seed=seed, with_values=True, out_keys=ok, out_vals=ov)
            ts.append((t, op, na, nb, seed, ok, ov))
        for t, op, na, nb, seed, ok, ov in ts:
            assert q.wait(t, timeout_s=300).status == mp.MP_OK, (op, na, nb)
            got_k, got_v = ok.numpy().view(np.uint32), ov.numpy().view(np.uint32)
            if op == "merge":
                a, av, b, bv = gen.serving_request("merge", na, nb, seed)
                ek, ev = oracle.merge(a, b, av, bv)
                alone_k, alone_v = mp.mp_merge_pairs(to_dev(a), vals_to_dev(av), to_dev(b), vals_to_dev(bv))
            else:
                k, v = gen.serving_request("sort", na, 0, seed)
                ek, ev = oracle.sort(k, v)
                alone_k, alone_v = to_dev(k), vals_to_dev(v)
                mp.mp_sort(alone_k, alone_v)
            assert first_mismatch(got_k, ek) is None, (op, na, nb)
            assert first_mismatch(got_v, ev) is None, (op, na, nb)
            assert first_mismatch(to_host(alone_k, np.uint32), got_k) is None, (op, na, nb)
            assert first_mismatch(to_host(alone_v, np.uint32), got_v) is None, (op, na, nb)
        st = q.stats()
        assert st["completed"] == len(specs) and st["failed"] == 0
        assert st["peak_bytes"] <= budget
