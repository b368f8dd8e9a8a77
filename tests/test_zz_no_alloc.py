"""The allocation-free merge entry point (mp_merge_noalloc).

It exists for callers that must not allocate device memory while merging
(code inside another runtime's memory arena, latency-critical loops); its
split-point scratch is a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test.  The GPU test calls the entry point through the C ABI
twice in a row per case and compares each result with the CPU oracle and
with mp_merge_pairs (exact: a merge has one correct output), and checks that
a warm call takes no device memory."""
import numpy as np
import pytest
import torch

import oracle
import paper_1406_2628_gb300 as mp
from paper_1406_2628_gb300 import build as mpbuild
from _util import first_mismatch, random_sorted, to_dev, to_host

LIMIT = 1073737728  # 262,143 tiles of 4096 outputs


def test_noalloc_rejects_sizes_over_its_limit():
    mpbuild.build()
    lib = mp.lib()
    st = lib.mp_merge_noalloc(mp.MP_U32, 0x10000, None, LIMIT, 0x100000000, None, 1,
                              0x200000000, None, None)
    assert st == mp.MP_ERR_INVALID_ARG
    assert "limit" in mp.mp_last_error()
    # Sizes whose sum overflows int64 are rejected too (no wrap-around).
    big = (1 << 63) - 1
    st = lib.mp_merge_noalloc(mp.MP_U32, 0x10000, None, big, 0x100000000, None, big,
                              0x200000000, None, None)
    assert st == mp.MP_ERR_INVALID_ARG
    assert "limit" in mp.mp_last_error()


_CODE = {np.dtype(np.int32): mp.MP_I32, np.dtype(np.float32): mp.MP_F32,
         np.dtype(np.uint64): mp.MP_U64}


@pytest.mark.gpu
@pytest.mark.parametrize("dt", [np.int32, np.float32, np.uint64], ids=["i32", "f32", "u64"])
def test_noalloc_matches_oracle_twice_without_taking_memory(dt):
    lib = mp.lib()
    rng = np.random.default_rng(2024)
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    code = _CODE[np.dtype(dt)]
    # An exact multiple of the 4096-output tile, one past it, and a ragged
    # size with uneven sides.
    sizes = [(61 * 4096 - 1000, 1000), (40 * 4096, 9 * 4096 + 1), (1_000_003, 654_321)]
    cases = []
    for na, nb in sizes:
        a = random_sorted(rng, dt, na, "ties")
        b = random_sorted(rng, dt, nb, "random")
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        ek, ev = oracle.merge(a, b, av, bv)
        A, B = to_dev(a), to_dev(b)
        AV = torch.from_numpy(av.view(np.int32)).to(dev)
        BV = torch.from_numpy(bv.view(np.int32)).to(dev)
        outs = [(torch.empty(na + nb, dtype=A.dtype, device=dev),
                 torch.empty(na + nb, dtype=torch.int32, device=dev),
                 torch.empty(na + nb, dtype=A.dtype, device=dev)) for _ in range(2)]
        ref_k, ref_v = mp.mp_merge_pairs(A, AV, B, BV)
        cases.append((a, b, A, B, AV, BV, outs, ek, ev, ref_k, ref_v))
    # One call of each form first: on a fresh device the first resolves the
    # array (and, under lazy module loading, loads it and its kernels);
    # every later call must take nothing.
    a, b, A, B, AV, BV, outs, *_ = cases[0]
    st = lib.mp_merge_noalloc(code, A.data_ptr(), AV.data_ptr(), a.size, B.data_ptr(), BV.data_ptr(),
                              b.size, outs[0][0].data_ptr(), outs[0][1].data_ptr(), stream)
    assert st == mp.MP_OK, mp.mp_last_error()
    st = lib.mp_merge_noalloc(code, A.data_ptr(), None, a.size, B.data_ptr(), None, b.size,
                              outs[0][2].data_ptr(), None, stream)
    assert st == mp.MP_OK, mp.mp_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for a, b, A, B, AV, BV, outs, ek, ev, ref_k, ref_v in cases:
        for call in range(2):
            OK, OV, OK2 = outs[call]
            st = lib.mp_merge_noalloc(code, A.data_ptr(), AV.data_ptr(), a.size, B.data_ptr(),
                                      BV.data_ptr(), b.size, OK.data_ptr(), OV.data_ptr(), stream)
            assert st == mp.MP_OK, mp.mp_last_error()
            # Keys only, through the same entry point.
            st = lib.mp_merge_noalloc(code, A.data_ptr(), None, a.size, B.data_ptr(), None, b.size,
                                      OK2.data_ptr(), None, stream)
            assert st == mp.MP_OK, mp.mp_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device memory taken by warm calls: {free0 - free1} bytes"
    for a, b, A, B, AV, BV, outs, ek, ev, ref_k, ref_v in cases:
        for call in range(2):
            OK, OV, OK2 = outs[call]
            got_k, got_v, got_k2 = to_host(OK, dt), to_host(OV, np.uint32), to_host(OK2, dt)
            assert first_mismatch(got_k, ek) is None, (a.size, b.size, call)
            assert first_mismatch(got_v, ev) is None, (a.size, b.size, call)
            assert first_mismatch(got_k2, ek) is None, (a.size, b.size, call)
            assert first_mismatch(got_k, to_host(ref_k, dt)) is None
            assert first_mismatch(got_v, to_host(ref_v, np.uint32)) is None
