"""The allocation-free merge entry point (mp_merge_noalloc).

It exists for callers that must not allocate device memory while merging
(code inside another runtime's memory arena, latency-critical loops); its
split-point scratch is a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test.  The GPU test calls the entry point through the C ABI
twice in a row and compares each result with mp_merge_pairs' (exact: a
merge has one correct output)."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1406_2628_gb300 as mp
from paper_1406_2628_gb300 import build as mpbuild
from _util import random_sorted


def test_noalloc_rejects_sizes_over_its_limit():
    mpbuild.build()
    lib = mp.lib()
    limit = 1073737728
    st = lib.mp_merge_noalloc(mp.MP_U32, 0x10000, None, limit, 0x100000000, None, 1,
                              0x200000000, None, None)
    assert st == mp.MP_ERR_INVALID_ARG
    assert "limit" in mp.mp_last_error()


@pytest.mark.gpu
def test_noalloc_matches_mp_merge_pairs_twice():
    lib = mp.lib()
    rng = np.random.default_rng(2024)
    dev = torch.device("cuda")
    for call in range(2):
        na, nb = 1_000_003 + call * 77, 654_321 - call * 5
        a = random_sorted(rng, np.uint64, na, "ties")
        b = random_sorted(rng, np.uint64, nb, "ties")
        A = torch.from_numpy(a.view(np.int64)).to(dev)
        B = torch.from_numpy(b.view(np.int64)).to(dev)
        AV = torch.arange(na, dtype=torch.int32, device=dev)
        BV = torch.arange(na, na + nb, dtype=torch.int32, device=dev)
        OK = torch.empty(na + nb, dtype=torch.int64, device=dev)
        OV = torch.empty(na + nb, dtype=torch.int32, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        st = lib.mp_merge_noalloc(mp.MP_U64, A.data_ptr(), AV.data_ptr(), na, B.data_ptr(),
                                  BV.data_ptr(), nb, OK.data_ptr(), OV.data_ptr(), stream)
        assert st == mp.MP_OK, mp.mp_last_error()
        RK = torch.empty_like(OK)
        RV = torch.empty_like(OV)
        st = lib.mp_merge_pairs(mp.MP_U64, A.data_ptr(), AV.data_ptr(), na, B.data_ptr(),
                                BV.data_ptr(), nb, RK.data_ptr(), RV.data_ptr(), stream)
        assert st == mp.MP_OK, mp.mp_last_error()
        torch.cuda.synchronize()
        assert torch.equal(OK, RK), call
        assert torch.equal(OV, RV), call
        # Keys only, through the same entry point.
        OK2 = torch.empty_like(OK)
        st = lib.mp_merge_noalloc(mp.MP_U64, A.data_ptr(), None, na, B.data_ptr(), None, nb,
                                  OK2.data_ptr(), None, stream)
        assert st == mp.MP_OK, mp.mp_last_error()
        torch.cuda.synchronize()
        assert torch.equal(OK2, RK), call
