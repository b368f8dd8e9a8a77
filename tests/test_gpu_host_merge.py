"""GPU parity of the end-to-end merge of host arrays (mp_merge_pairs_host):
one chunk and many (inputs from 64 MB are copied in chunks and each settled
piece of the output is merged and copied back while later inputs arrive),
with the inputs that make the chunk cuts uneven: every A above every B (no
output is settled until B has arrived), all keys equal, long runs, keys
only and with values, pinned and pageable host memory."""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_2628_gb300 as mp
from _util import first_mismatch, random_sorted

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    mp.lib()
    torch.cuda.init()


def _host(x, pinned):
    t = torch.from_numpy(np.ascontiguousarray(x))
    return t.pin_memory() if pinned else t


def _run(a, b, with_vals, pinned):
    na, nb = a.size, b.size
    av = np.arange(na, dtype=np.uint32)
    bv = np.arange(na, na + nb, dtype=np.uint32)
    hA, hB = _host(a, pinned), _host(b, pinned)
    hOK = torch.empty(na + nb, dtype=hA.dtype)
    hOK = hOK.pin_memory() if pinned else hOK
    if with_vals:
        hAV, hBV = _host(av.view(np.int32), pinned), _host(bv.view(np.int32), pinned)
        hOV = torch.empty(na + nb, dtype=torch.int32)
        hOV = hOV.pin_memory() if pinned else hOV
        mp.mp_merge_pairs_host(hA, hAV, hB, hBV, hOK, hOV)
        ek, ev = oracle.merge(a, b, av, bv)
        assert first_mismatch(hOV.numpy().view(np.uint32), ev) is None, (na, nb)
    else:
        mp.mp_merge_pairs_host(hA, None, hB, None, hOK, None)
        ek, _ = oracle.merge(a, b)
    assert first_mismatch(hOK.numpy().view(a.dtype), ek) is None, (na, nb)


@pytest.mark.parametrize("dt", [np.int32, np.uint64, np.float32], ids=lambda d: np.dtype(d).name)
def test_host_merge_one_chunk(dt):
    rng = np.random.default_rng(5000)
    for na, nb in [(1, 0), (0, 5), (1000, 3), (300_001, 200_000)]:
        a, b = random_sorted(rng, dt, na, "ties"), random_sorted(rng, dt, nb, "ties")
        _run(a, b, True, pinned=True)
        _run(a, b, False, pinned=False)


@pytest.mark.parametrize("kind", ["random", "a_gt_b", "b_gt_a", "equal", "runs"])
def test_host_merge_many_chunks(kind):
    """About 300 MB of uint64 keys + values: five 64 MB chunks."""
    rng = np.random.default_rng(5100)
    na, nb = 15_000_007, 10_000_001
    if kind == "random":
        a, b = random_sorted(rng, np.uint64, na, "random"), random_sorted(rng, np.uint64, nb, "random")
    elif kind in ("a_gt_b", "b_gt_a"):
        lo = np.sort(rng.integers(0, 1 << 62, na, dtype=np.uint64))
        hi = np.sort(rng.integers(1 << 62, 1 << 63, nb, dtype=np.uint64))
        a, b = (hi[:nb].copy(), lo[:na].copy()) if kind == "a_gt_b" else (lo, hi)
    elif kind == "equal":
        a, b = np.full(na, 7, np.uint64), np.full(nb, 7, np.uint64)
    else:
        a = np.sort(rng.integers(0, 40, na).astype(np.uint64))
        b = np.sort(rng.integers(0, 40, nb).astype(np.uint64))
    _run(a, b, True, pinned=True)


def test_host_merge_many_chunks_keys_only_i32():
    rng = np.random.default_rng(5200)
    a = random_sorted(rng, np.int32, 25_000_000, "ties")
    b = random_sorted(rng, np.int32, 20_000_003, "ties")
    _run(a, b, False, pinned=True)
