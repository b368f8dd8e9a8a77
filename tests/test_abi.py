"""C ABI checks that need no GPU: the library builds, loads and exports every
entry point include/mp.h declares; host-side argument errors and pure host
queries behave as documented (these return before any CUDA call)."""
import ctypes
import os
import re
from ctypes import byref as C_byref, c_void_p as C_void_p

import pytest

import paper_1406_2628_gb300 as mp
from paper_1406_2628_gb300 import build as mpbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_symbols():
    names = []
    for h in HEADERS:
        with open(h) as f:
            text = f.read()
        names += re.findall(r"^MP_API\s+[\w\s\*]+?\b(mp_\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    mpbuild.build()
    return mp.lib()


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ["mp_merge_keys", "mp_merge_pairs", "mp_sort", "mp_sort_workspace_bytes",
                     "mp_merge_batched", "mp_check_sorted", "mp_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(mp.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(raw, name), f"libmp.so does not export {name}"


def test_binding_covers_every_declared_symbol():
    assert set(declared_symbols()) <= set(mp.exported_symbols())


def test_status_strings(lib):
    for code in range(0, 11):
        s = mp.mp_status_string(code)
        assert s and s != "unknown mp_status"
    assert mp.mp_status_string(99) == "unknown mp_status"


def test_dtype_sizes(lib):
    assert [lib.mp_dtype_size(d) for d in range(5)] == [4, 4, 4, 8, 8]
    assert lib.mp_dtype_size(7) == 0


def test_sort_workspace_bytes(lib):
    assert mp.mp_sort_workspace_bytes(mp.MP_I32, 0, False) == 0
    assert mp.mp_sort_workspace_bytes(mp.MP_I32, 1, False) == 0
    n = 1 << 20
    k = mp.mp_sort_workspace_bytes(mp.MP_I32, n, False)
    kv = mp.mp_sort_workspace_bytes(mp.MP_I32, n, True)
    assert k >= n * 4 and kv >= k + n * 4
    assert mp.mp_sort_workspace_bytes(mp.MP_U64, n, False) >= n * 8
    assert mp.mp_sort_workspace_bytes(9, n, False) == 0


def test_host_argument_errors(lib):
    # Negative sizes and NULL pointers are rejected on the host, before any
    # CUDA call, with a detail message.
    st = lib.mp_merge_keys(mp.MP_I32, None, -1, None, 0, None, None)
    assert st == mp.MP_ERR_INVALID_ARG
    assert "negative" in mp.mp_last_error()
    st = lib.mp_merge_keys(mp.MP_I32, None, 5, None, 0, None, None)
    assert st == mp.MP_ERR_INVALID_ARG
    st = lib.mp_merge_keys(17, None, 0, None, 0, None, None)
    assert st == mp.MP_ERR_UNSUPPORTED_DTYPE
    # Misaligned key pointer.
    st = lib.mp_merge_keys(mp.MP_U64, 0x1004, 1, 0x2000, 1, 0x3000, None)
    assert st == mp.MP_ERR_INVALID_ARG and "aligned" in mp.mp_last_error()
    # Output overlapping an input.
    st = lib.mp_merge_keys(mp.MP_I32, 0x10000, 100, 0x20000, 100, 0x10100, None)
    assert st == mp.MP_ERR_INVALID_ARG and "overlap" in mp.mp_last_error()
    # Empty merge is a no-op.
    assert lib.mp_merge_keys(mp.MP_I32, None, 0, None, 0, None, None) == mp.MP_OK
    # Pairs need all value arrays.
    st = lib.mp_merge_pairs(mp.MP_I32, 0x1000, None, 1, 0x2000, None, 1, 0x3000, None, None)
    assert st == mp.MP_ERR_INVALID_ARG
    # Sort: workspace too small / misaligned; n <= 1 is a no-op.
    assert lib.mp_sort(mp.MP_I32, None, None, 1, None, 0, None) == mp.MP_OK
    st = lib.mp_sort(mp.MP_I32, 0x100000, None, 1 << 20, 0x8000000, 16, None)
    assert st == mp.MP_ERR_INVALID_ARG and "workspace" in mp.mp_last_error()
    # Batched: inconsistent totals, bad plan.
    st = lib.mp_merge_batched(mp.MP_I32, None, None, None, None, 0, 5, 0, None, None, None, None,
                              None, None)
    assert st == mp.MP_ERR_INVALID_ARG
    bad = mp.mp_plan(100, 3, 0, 0)
    st = lib.mp_merge_batched(mp.MP_I32, 0x1000, 0x2000, 0x3000, 0x4000, 1, 1, 1, 0x5000, None,
                              None, None, ctypes.byref(bad), None)
    assert st == mp.MP_ERR_INVALID_ARG and "plan" in mp.mp_last_error()


def test_plan_supported(lib):
    assert mp.mp_plan_supported((256, 8))
    assert mp.mp_plan_supported((128, 16, mp.MP_STAGE_VECTOR))
    assert not mp.mp_plan_supported((100, 3))
    assert not mp.mp_plan_supported((256, 7))


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(mp, "_lib", None)
    monkeypatch.setattr(mp, "LIB_PATH", str(tmp_path / "libmp.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        mp.lib()


def test_tune_table_round_trip_on_host(lib, tmp_path):
    """The tuned-shape table is host state: an entry loaded from a file is
    what automatic plans use (no GPU needed to resolve a plan)."""
    mp.mp_tune_clear()
    default = lib.mp_merge_tile_items(mp.MP_I32, 0, 1 << 20, None)
    assert default > 0
    # The device name is "unknown" when no GPU is visible.
    path = tmp_path / "tune.txt"
    path.write_text("unknown|merge|4|0|20 128 8 1\n")
    mp.mp_tune_load(str(path))
    try:
        assert lib.mp_merge_tile_items(mp.MP_I32, 0, 1 << 20, None) == 1024
        assert lib.mp_merge_tile_items(mp.MP_I32, 0, 1 << 21, None) == default
        mp.mp_tune_save(str(tmp_path / "out.txt"))
        assert "unknown|merge|4|0|20 128 8 1" in (tmp_path / "out.txt").read_text()
    finally:
        mp.mp_tune_clear()
    with pytest.raises(mp.MPError):
        mp.mp_tune_load(str(tmp_path / "missing.txt"))


def test_queue_argument_errors(lib):
    h = C_void_p()
    assert lib.mp_queue_create(0, 4, C_byref(h)) == mp.MP_ERR_INVALID_ARG
    assert lib.mp_queue_create(1 << 20, 0, C_byref(h)) == mp.MP_ERR_INVALID_ARG
    assert lib.mp_queue_submit(None, None, None) == mp.MP_ERR_INVALID_ARG
    assert lib.mp_queue_wait(None, 1, 0, None) == mp.MP_ERR_INVALID_ARG
    assert lib.mp_queue_destroy(None) == mp.MP_OK
    assert lib.mp_graph_launch(None, None) == mp.MP_ERR_INVALID_ARG
    assert lib.mp_graph_destroy(None) == mp.MP_OK


def test_default_plans_on_host(lib, monkeypatch):
    """The automatic plan of each key kind (a host-side choice, no CUDA call):
    the streaming merge (Alg. 3) up to its size limit, TMA-staged tiles above
    it; explicit plans are reported as given."""
    monkeypatch.delenv("MP_TUNE_CACHE", raising=False)
    mp.mp_tune_clear()
    bulk, stream = mp.MP_STAGE_BULK, mp.MP_STAGE_STREAM
    big = 335_544_320
    assert mp.mp_merge_resolve_plan(mp.MP_U64, True, big) == (256, 12, bulk)
    assert mp.mp_merge_resolve_plan(mp.MP_I32, False, big) == (128, 33, bulk)
    assert mp.mp_merge_resolve_plan(mp.MP_F32, False, big) == (128, 33, bulk)
    assert mp.mp_merge_resolve_plan(mp.MP_I64, False, big) == (128, 27, bulk)
    assert mp.mp_merge_resolve_plan(mp.MP_U128, False, big) == (128, 12, bulk)
    assert mp.mp_merge_tile_items(mp.MP_U64, True, big) == 256 * 12
    assert mp.mp_merge_tile_items(mp.MP_U32, False, big) == 128 * 33
    # Small merges: the partition-free streaming plan, up to 2^22 outputs
    # for 4-byte keys alone and 3 * 2^20 otherwise.
    assert mp.mp_merge_resolve_plan(mp.MP_I32, False, 1 << 22) == (256, 8, stream)
    assert mp.mp_merge_resolve_plan(mp.MP_I32, False, (1 << 22) + 1) == (128, 33, bulk)
    assert mp.mp_merge_resolve_plan(mp.MP_U64, True, 3 << 20) == (128, 8, stream)
    assert mp.mp_merge_resolve_plan(mp.MP_U64, True, (3 << 20) + 1) == (256, 12, bulk)
    # Tile queries never report a streaming shape: they size split arrays.
    assert mp.mp_merge_tile_items(mp.MP_I32, False, 1 << 20) == 128 * 33
    # An explicit plan wins.
    assert mp.mp_merge_resolve_plan(mp.MP_U64, True, big, (128, 8, bulk)) == (128, 8, bulk)


def test_inject_fault_rejects_bad_arguments(lib):
    # Both checks return before any CUDA call.
    assert lib.mp_inject_fault(99, 1) == mp.MP_ERR_INVALID_ARG
    assert "unknown" in mp.mp_last_error()
    assert lib.mp_inject_fault(mp.MP_FAULT_SCRATCH_ALLOC, -1) == mp.MP_ERR_INVALID_ARG
    assert "negative" in mp.mp_last_error()
    # Host-side counters: setting and cancelling needs no GPU.
    assert lib.mp_inject_fault(mp.MP_FAULT_SCRATCH_ALLOC, 3) == mp.MP_OK
    assert lib.mp_inject_fault(mp.MP_FAULT_SCRATCH_ALLOC, 0) == mp.MP_OK
    assert lib.mp_inject_fault(mp.MP_FAULT_QUEUE_STEP, 0) == mp.MP_OK


def test_force_plan_override_of_automatic_plans(lib, monkeypatch):
    # MP_FORCE_PLAN replaces the automatic plan (a host-side decision: no GPU).
    big = 1 << 30
    monkeypatch.delenv("MP_FORCE_PLAN", raising=False)
    auto = mp.mp_merge_resolve_plan(mp.MP_U64, True, big)
    assert auto[2] == mp.MP_STAGE_BULK
    monkeypatch.setenv("MP_FORCE_PLAN", "128,8,vector")
    assert mp.mp_merge_resolve_plan(mp.MP_U64, True, big) == (128, 8, mp.MP_STAGE_VECTOR)
    monkeypatch.setenv("MP_FORCE_PLAN", "256,12,2")
    assert mp.mp_merge_resolve_plan(mp.MP_I32, False, 1000) == (256, 12, mp.MP_STAGE_BULK)
    # An explicit plan is not overridden.
    assert mp.mp_merge_resolve_plan(mp.MP_U64, True, big, (128, 16, mp.MP_STAGE_BULK)) == \
        (128, 16, mp.MP_STAGE_BULK)
    # An unsupported forced plan is an argument error naming the variable.
    monkeypatch.setenv("MP_FORCE_PLAN", "100,3,bulk")
    with pytest.raises(mp.MPError) as ei:
        mp.mp_merge_resolve_plan(mp.MP_U64, True, big)
    assert ei.value.status == mp.MP_ERR_INVALID_ARG
    assert "MP_FORCE_PLAN" in mp.mp_last_error()
    monkeypatch.delenv("MP_FORCE_PLAN")
    assert mp.mp_merge_resolve_plan(mp.MP_U64, True, big) == auto


def test_set_operation_and_grouped_host_errors(lib):
    # Output capacities per operation (multiset semantics bound the result).
    assert lib.mp_set_capacity(mp.MP_SET_UNION, 5, 7) == 12
    assert lib.mp_set_capacity(mp.MP_SET_INTERSECTION, 5, 7) == 5
    assert lib.mp_set_capacity(mp.MP_SET_DIFFERENCE, 5, 7) == 5
    assert lib.mp_set_capacity(mp.MP_SET_SYMMETRIC_DIFFERENCE, 5, 7) == 12
    assert lib.mp_set_capacity(9, 5, 7) == -1
    assert lib.mp_set_capacity(mp.MP_SET_UNION, -1, 7) == -1
    # Set operations: rejected on the host, before any CUDA call.
    cnt = 0x9000
    st = lib.mp_set_operation(9, mp.MP_I32, 0x1000, None, 1, 0x2000, None, 1, 0x3000, None, cnt, None)
    assert st == mp.MP_ERR_INVALID_ARG
    st = lib.mp_set_operation(mp.MP_SET_UNION, 17, 0x1000, None, 1, 0x2000, None, 1, 0x3000, None, cnt, None)
    assert st == mp.MP_ERR_UNSUPPORTED_DTYPE
    st = lib.mp_set_operation(mp.MP_SET_UNION, mp.MP_I32, 0x1000, None, 1, 0x2000, None, 1, 0x3000, None, None,
                              None)
    assert st == mp.MP_ERR_INVALID_ARG and "out_count" in mp.mp_last_error()
    st = lib.mp_set_operation(mp.MP_SET_UNION, mp.MP_I32, 0x1000, None, 1, 0x2000, None, 1, 0x3000, None,
                              cnt + 4, None)
    assert st == mp.MP_ERR_INVALID_ARG and "aligned" in mp.mp_last_error()
    st = lib.mp_set_operation(mp.MP_SET_UNION, mp.MP_I32, 0x1000, None, 100, 0x2000, None, 100, 0x1000, None,
                              cnt, None)
    assert st == mp.MP_ERR_INVALID_ARG and "overlap" in mp.mp_last_error()
    # Grouped merges: descriptor array and key widths checked first.
    assert lib.mp_merge_grouped(None, 0, 0, None) == mp.MP_OK
    assert lib.mp_merge_grouped(None, 1, 0, None) == mp.MP_ERR_INVALID_ARG
    assert lib.mp_merge_grouped(None, -1, 0, None) == mp.MP_ERR_INVALID_ARG
    arr = (mp.mp_merge_desc * 2)()
    for i, d in enumerate(arr):
        d.dtype = mp.MP_I32
        d.a_keys, d.na = 0x10000 + i * 0x1000, 4
        d.b_keys, d.nb = 0x20000 + i * 0x1000, 4
        d.out_keys = 0x30000 + i * 0x1000
    arr[1].dtype = mp.MP_U64
    assert lib.mp_merge_grouped(arr, 2, 0, None) == mp.MP_ERR_INVALID_ARG
    assert "widths" in mp.mp_last_error()
    arr[1].dtype = mp.MP_U128
    assert lib.mp_merge_grouped(arr, 2, 0, None) == mp.MP_ERR_UNSUPPORTED_DTYPE
    arr[1].dtype = mp.MP_I32
    arr[1].out_keys = arr[1].a_keys  # output overlapping an input
    assert lib.mp_merge_grouped(arr, 2, 0, None) == mp.MP_ERR_INVALID_ARG
