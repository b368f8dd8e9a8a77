"""GB300 Merge Path: Python binding of libmp.so (the C ABI in include/mp.h).

Merge Path (Green, Odeh, Birk): stable merging of two sorted arrays split
into equal independent pieces by binary searches along the cross diagonals
of the merge grid (Alg. 1, Alg. 2), and the merge sort built from it.

This module only marshals arguments: torch tensors supply device memory and
the current CUDA stream; every step of the computation runs in the library's
CUDA kernels.  There is no CPU fallback: if libmp.so has not been built, or
no GPU is present, calls raise.  Function names match the C entry points.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmp.so")

# mp_status
MP_OK = 0
MP_ERR_INVALID_ARG = 1
MP_ERR_UNSUPPORTED_DTYPE = 2
MP_ERR_NOT_SORTED = 3
MP_ERR_NAN = 4
MP_ERR_NO_MEMORY = 5
MP_ERR_BUDGET = 6
MP_ERR_TIMEOUT = 7
MP_ERR_CUDA = 8
MP_ERR_INTERNAL = 9
MP_ERR_NOT_READY = 10

# mp_dtype
MP_I32, MP_U32, MP_F32, MP_U64, MP_I64 = 0, 1, 2, 3, 4
MP_DESCENDING = 0x100  # OR'ed into a dtype: descending key order

# request queue enums
MP_OP_MERGE, MP_OP_SORT = 0, 1
MP_SRC_HOST, MP_SRC_DEVICE, MP_SRC_GENERATE = 0, 1, 2
MP_SINK_HOST, MP_SINK_DEVICE, MP_SINK_DISCARD = 0, 1, 2

MP_STAGE_AUTO, MP_STAGE_VECTOR, MP_STAGE_BULK, MP_STAGE_WARP, MP_STAGE_STREAM = 0, 1, 2, 3, 4

MP_SET_UNION, MP_SET_INTERSECTION, MP_SET_DIFFERENCE, MP_SET_SYMMETRIC_DIFFERENCE = 0, 1, 2, 3
_SET_OPS = {"union": MP_SET_UNION, "intersection": MP_SET_INTERSECTION,
            "difference": MP_SET_DIFFERENCE, "symmetric_difference": MP_SET_SYMMETRIC_DIFFERENCE}

_TORCH_DTYPE = {
    torch.int32: MP_I32,
    torch.uint32: MP_U32,
    torch.float32: MP_F32,
    torch.uint64: MP_U64,
    torch.int64: MP_I64,
}


class MPError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"{detail} [status {status}]")
        self.status = status


class mp_merge_desc(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("a_keys", ctypes.c_void_p), ("a_vals", ctypes.c_void_p), ("na", ctypes.c_int64),
                ("b_keys", ctypes.c_void_p), ("b_vals", ctypes.c_void_p), ("nb", ctypes.c_int64),
                ("out_keys", ctypes.c_void_p), ("out_vals", ctypes.c_void_p)]


class mp_request(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("dtype", ctypes.c_int32), ("with_values", ctypes.c_int32),
                ("source", ctypes.c_int32), ("sink", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("a_keys", ctypes.c_void_p), ("a_vals", ctypes.c_void_p), ("na", ctypes.c_int64),
                ("b_keys", ctypes.c_void_p), ("b_vals", ctypes.c_void_p), ("nb", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("out_keys", ctypes.c_void_p), ("out_vals", ctypes.c_void_p)]


class mp_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("op", ctypes.c_int32), ("n", ctypes.c_int64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class mp_queue_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "completed", "failed", "steps", "launches",
                                               "peak_bytes", "waiting", "active", "bytes_in_use")]


class mp_plan(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("items_per_thread", ctypes.c_int32),
                ("staging", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None

# Exported C symbols and their ctypes signatures.
_P, _I64, _I32, _SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
_SIGNATURES = {
    "mp_status_string": ([_I32], ctypes.c_char_p),
    "mp_last_error": ([], ctypes.c_char_p),
    "mp_dtype_size": ([_I32], _SZ),
    "mp_merge_keys": ([_I32, _P, _I64, _P, _I64, _P, _P], _I32),
    "mp_merge_pairs": ([_I32, _P, _P, _I64, _P, _P, _I64, _P, _P, _P], _I32),
    "mp_merge_plan": ([_I32, _P, _P, _I64, _P, _P, _I64, _P, _P, ctypes.POINTER(mp_plan), _P], _I32),
    "mp_plan_supported": ([ctypes.POINTER(mp_plan)], _I32),
    "mp_merge_tile_items": ([_I32, _I32, _I64, ctypes.POINTER(mp_plan)], _I64),
    "mp_merge_partitioned": ([_I32, _P, _P, _I64, _P, _P, _I64, _P, _P, _P,
                              ctypes.POINTER(mp_plan), _P], _I32),
    "mp_merge_pairs_host": ([_I32, _P, _P, _I64, _P, _P, _I64, _P, _P, _P], _I32),
    "mp_merge_path_partition": ([_I32, _P, _I64, _P, _I64, _I64, _P, _P], _I32),
    "mp_sort_workspace_bytes": ([_I32, _I64, _I32], _SZ),
    "mp_sort": ([_I32, _P, _P, _I64, _P, _SZ, _P], _I32),
    "mp_merge_batched": ([_I32, _P, _P, _P, _P, _I64, _I64, _I64, _P, _P, _P, _P,
                          ctypes.POINTER(mp_plan), _P], _I32),
    "mp_check_sorted": ([_I32, _P, _I64, _P], _I32),
    "mp_merge_grouped": ([ctypes.POINTER(mp_merge_desc), _I64, _I32, _P], _I32),
    "mp_clock_seconds": ([], ctypes.c_double),
    "mp_kernel_error": ([ctypes.POINTER(ctypes.c_uint), _I32], _I32),
    "mp_kernel_status": ([_P, _I32], _I32),
    "mp_inject_fault": ([_I32, _I64], _I32),
    "mp_merge_noalloc": ([_I32, _P, _P, _I64, _P, _P, _I64, _P, _P, _P], _I32),
    "mp_merge_checksum": ([_I32, _P, _P, _I64, _P, _P, _I64, _P, _P], _I32),
    "mp_autotune_merge": ([_I32, _P, _P, _I64, _P, _P, _I64, _P, _P, _I32, ctypes.POINTER(mp_plan), _P], _I32),
    "mp_autotune_batched": ([_I32, _P, _P, _P, _P, _I64, _I64, _I64, _P, _P, _P, _P, _I32,
                             ctypes.POINTER(mp_plan), _P], _I32),
    "mp_tune_save": ([ctypes.c_char_p], _I32),
    "mp_tune_load": ([ctypes.c_char_p], _I32),
    "mp_tune_clear": ([], None),
    "mp_graph_merge_create": ([_I32, _P, _P, _I64, _P, _P, _I64, _P, _P, ctypes.POINTER(mp_plan),
                               ctypes.POINTER(ctypes.c_void_p)], _I32),
    "mp_graph_batched_create": ([_I32, _P, _P, _P, _P, _I64, _I64, _I64, _P, _P, _P, _P,
                                 ctypes.POINTER(mp_plan), ctypes.POINTER(ctypes.c_void_p)], _I32),
    "mp_graph_launch": ([_P, _P], _I32),
    "mp_graph_destroy": ([_P], _I32),
    "mp_queue_create": ([_SZ, _I32, ctypes.POINTER(ctypes.c_void_p)], _I32),
    "mp_queue_submit": ([_P, ctypes.POINTER(mp_request), ctypes.POINTER(ctypes.c_uint64)], _I32),
    "mp_queue_wait": ([_P, ctypes.c_uint64, _I64, ctypes.POINTER(mp_result)], _I32),
    "mp_queue_get_stats": ([_P, ctypes.POINTER(mp_queue_stats)], _I32),
    "mp_queue_destroy": ([_P], _I32),
    "mp_generate": ([_I32, _P, _P, _I64, ctypes.c_uint64, ctypes.c_uint64, _I32, ctypes.c_uint32, _P], _I32),
    "mp_set_capacity": ([_I32, _I64, _I64], _I64),
    "mp_merge_resolve_plan": ([_I32, _I32, _I64, ctypes.POINTER(mp_plan), ctypes.POINTER(mp_plan)], _I32),
    "mp_set_operation": ([_I32, _I32, _P, _P, _I64, _P, _P, _I64, _P, _P, _P, _P], _I32),
}


def exported_symbols():
    """Names of the C entry points this binding declares."""
    return list(_SIGNATURES)


def lib():
    """Load libmp.so (built in-tree by paper_1406_2628_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with `python -m paper_1406_2628_gb300.build` "
                    "(the library has no CPU fallback)")
            h = ctypes.CDLL(LIB_PATH)
            for name, (argtypes, restype) in _SIGNATURES.items():
                f = getattr(h, name)
                f.argtypes = argtypes
                f.restype = restype
            _lib = h
    return _lib


def _check(status: int):
    if status != MP_OK:
        detail = lib().mp_last_error().decode() or lib().mp_status_string(status).decode()
        raise MPError(status, detail)


def _dtype_code(t: torch.Tensor, descending: bool = False) -> int:
    try:
        return _TORCH_DTYPE[t.dtype] | (MP_DESCENDING if descending else 0)
    except KeyError:
        raise TypeError(f"unsupported key dtype {t.dtype}") from None


# 128-bit keys: (n, 2) tensors of 64-bit words, low word first in each row.
_WIDE = {"u128": 5, "i128": 6}
MP_U128, MP_I128 = 5, 6


def _kcode(t: torch.Tensor, descending: bool = False, wide: str | None = None) -> int:
    """dtype code of a key tensor; wide="u128"/"i128" for 128-bit keys."""
    if wide is None:
        return _dtype_code(t, descending)
    if wide not in _WIDE:
        raise TypeError(f"unknown wide key kind {wide!r}")
    if t.dim() != 2 or t.shape[1] != 2 or t.element_size() != 8:
        raise TypeError("128-bit keys must be an (n, 2) tensor of 64-bit words")
    return _WIDE[wide] | (MP_DESCENDING if descending else 0)


def _count(t: torch.Tensor, wide: str | None = None) -> int:
    return t.shape[0] if wide is not None else t.numel()


def _new_keys(like: torch.Tensor, n: int, wide: str | None = None) -> torch.Tensor:
    return torch.empty((n, 2) if wide is not None else n, dtype=like.dtype, device=like.device)


def _dev(t: torch.Tensor, what: str) -> int:
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


def _vals(t, what):
    if t.dtype not in (torch.int32, torch.uint32):
        raise TypeError(f"{what} must be int32 or uint32 (uint32 payload bits)")
    return _dev(t, what)


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _plan(plan):
    if plan is None:
        return None
    if isinstance(plan, mp_plan):
        return ctypes.byref(plan)
    nt, vt, *rest = plan
    return ctypes.byref(mp_plan(int(nt), int(vt), int(rest[0]) if rest else 0, 0))


def mp_status_string(status: int) -> str:
    return lib().mp_status_string(int(status)).decode()


def mp_last_error() -> str:
    return lib().mp_last_error().decode()


def mp_merge_keys(a: torch.Tensor, b: torch.Tensor, out: torch.Tensor | None = None,
                  stream=None, descending: bool = False, wide: str | None = None) -> torch.Tensor:
    """Stable merge of sorted 1-D tensors a and b (ties: a first)."""
    if a.dtype != b.dtype:
        raise TypeError("a and b must have the same dtype")
    if out is None:
        out = _new_keys(a, _count(a, wide) + _count(b, wide), wide)
    _check(lib().mp_merge_keys(_kcode(a, descending, wide), _dev(a, "a"), _count(a, wide), _dev(b, "b"),
                               _count(b, wide), _dev(out, "out"), _stream(stream)))
    return out


def mp_merge_pairs(a_keys, a_vals, b_keys, b_vals, out_keys=None, out_vals=None, stream=None,
                   descending: bool = False, wide: str | None = None):
    """Stable merge moving a uint32 payload with each key."""
    if a_keys.dtype != b_keys.dtype:
        raise TypeError("key dtypes differ")
    n = _count(a_keys, wide) + _count(b_keys, wide)
    if out_keys is None:
        out_keys = _new_keys(a_keys, n, wide)
    if out_vals is None:
        out_vals = torch.empty(n, dtype=a_vals.dtype, device=a_keys.device)
    _check(lib().mp_merge_pairs(_kcode(a_keys, descending, wide), _dev(a_keys, "a_keys"), _vals(a_vals, "a_vals"),
                                _count(a_keys, wide), _dev(b_keys, "b_keys"), _vals(b_vals, "b_vals"),
                                _count(b_keys, wide), _dev(out_keys, "out_keys"), _vals(out_vals, "out_vals"),
                                _stream(stream)))
    return out_keys, out_vals


def mp_merge_plan(a_keys, b_keys, a_vals=None, b_vals=None, out_keys=None, out_vals=None,
                  plan=None, stream=None, descending: bool = False, wide: str | None = None):
    """Merge with an explicit tile plan (block_threads, items_per_thread[, staging])."""
    n = _count(a_keys, wide) + _count(b_keys, wide)
    if out_keys is None:
        out_keys = _new_keys(a_keys, n, wide)
    pairs = a_vals is not None
    if pairs and out_vals is None:
        out_vals = torch.empty(n, dtype=a_vals.dtype, device=a_keys.device)
    _check(lib().mp_merge_plan(_kcode(a_keys, descending, wide), _dev(a_keys, "a_keys"),
                               _vals(a_vals, "a_vals") if pairs else None, _count(a_keys, wide),
                               _dev(b_keys, "b_keys"), _vals(b_vals, "b_vals") if pairs else None,
                               _count(b_keys, wide), _dev(out_keys, "out_keys"),
                               _vals(out_vals, "out_vals") if pairs else None, _plan(plan),
                               _stream(stream)))
    return (out_keys, out_vals) if pairs else out_keys


def mp_plan_supported(plan) -> bool:
    p = plan if isinstance(plan, mp_plan) else mp_plan(int(plan[0]), int(plan[1]),
                                                       int(plan[2]) if len(plan) > 2 else 0, 0)
    return bool(lib().mp_plan_supported(ctypes.byref(p)))


def mp_merge_checksum(a_keys, b_keys, a_vals=None, b_vals=None, out=None, stream=None, descending: bool = False):
    """Merge without storing (results folded into an order-sensitive uint64
    digest on the device); returns the 1-element int64 device tensor."""
    if out is None:
        out = torch.empty(1, dtype=torch.int64, device=a_keys.device)
    pairs = a_vals is not None
    _check(lib().mp_merge_checksum(_dtype_code(a_keys, descending), _dev(a_keys, "a_keys"),
                                   _vals(a_vals, "a_vals") if pairs else None, a_keys.numel(),
                                   _dev(b_keys, "b_keys"), _vals(b_vals, "b_vals") if pairs else None,
                                   b_keys.numel(), _dev(out, "checksum"), _stream(stream)))
    return out


def mp_set_capacity(op, na: int, nb: int) -> int:
    code = _SET_OPS[op] if isinstance(op, str) else int(op)
    return int(lib().mp_set_capacity(code, int(na), int(nb)))


def mp_set_operation(op, a_keys, b_keys, a_vals=None, b_vals=None, out_keys=None, out_vals=None,
                     count=None, stream=None, descending: bool = False, trim: bool = True,
                     wide: str | None = None):
    """Set operation ``op`` ("union", "intersection", "difference",
    "symmetric_difference" or an MP_SET_* code) of sorted a_keys and b_keys
    (multiset semantics).  Returns (keys, values or None, count tensor); with
    trim=True the outputs are sliced to the result length (one device read)."""
    code = _SET_OPS[op] if isinstance(op, str) else int(op)
    cap = mp_set_capacity(code, _count(a_keys, wide), _count(b_keys, wide))
    if cap < 0:
        raise MPError(MP_ERR_INVALID_ARG, f"unknown set operation {op!r}")
    if out_keys is None:
        out_keys = _new_keys(a_keys, cap, wide)
    pairs = a_vals is not None
    if pairs and out_vals is None:
        out_vals = torch.empty(cap, dtype=a_vals.dtype, device=a_keys.device)
    if count is None:
        count = torch.empty(1, dtype=torch.int64, device=a_keys.device)
    _check(lib().mp_set_operation(code, _kcode(a_keys, descending, wide), _dev(a_keys, "a_keys"),
                                  _vals(a_vals, "a_vals") if pairs else None, _count(a_keys, wide),
                                  _dev(b_keys, "b_keys"), _vals(b_vals, "b_vals") if pairs else None,
                                  _count(b_keys, wide), _dev(out_keys, "out_keys"),
                                  _vals(out_vals, "out_vals") if pairs else None, _dev(count, "count"),
                                  _stream(stream)))
    if trim:
        n = int(count.item())
        out_keys = out_keys[:n]
        out_vals = out_vals[:n] if pairs else None
    return out_keys, (out_vals if pairs else None), count


def mp_merge_resolve_plan(dtype, with_values: bool, total: int, plan=None):
    """The (block_threads, items_per_thread, staging) mp_merge_plan would run."""
    code = dtype if isinstance(dtype, int) else _TORCH_DTYPE[dtype]
    out = mp_plan()
    _check(lib().mp_merge_resolve_plan(code, 1 if with_values else 0, int(total), _plan(plan), ctypes.byref(out)))
    return (out.block_threads, out.items_per_thread, out.staging)


def mp_merge_tile_items(dtype, with_values: bool, total: int, plan=None) -> int:
    code = dtype if isinstance(dtype, int) else _TORCH_DTYPE[dtype]
    return int(lib().mp_merge_tile_items(code, 1 if with_values else 0, int(total), _plan(plan)))


def mp_merge_partitioned(a_keys, b_keys, a_split, a_vals=None, b_vals=None, out_keys=None,
                         out_vals=None, plan=None, stream=None, wide: str | None = None):
    """The merge kernel alone over split points from mp_merge_path_partition
    (spacing = mp_merge_tile_items(...))."""
    n = _count(a_keys, wide) + _count(b_keys, wide)
    if out_keys is None:
        out_keys = _new_keys(a_keys, n, wide)
    pairs = a_vals is not None
    if pairs and out_vals is None:
        out_vals = torch.empty(n, dtype=a_vals.dtype, device=a_keys.device)
    _check(lib().mp_merge_partitioned(_kcode(a_keys, False, wide), _dev(a_keys, "a_keys"),
                                      _vals(a_vals, "a_vals") if pairs else None, _count(a_keys, wide),
                                      _dev(b_keys, "b_keys"), _vals(b_vals, "b_vals") if pairs else None,
                                      _count(b_keys, wide), _dev(out_keys, "out_keys"),
                                      _vals(out_vals, "out_vals") if pairs else None,
                                      _dev(a_split, "a_split"), _plan(plan), _stream(stream)))
    return (out_keys, out_vals) if pairs else out_keys


def _host(t, what):
    if t.is_cuda:
        raise ValueError(f"{what} must be a host (CPU) tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


def mp_merge_pairs_host(a_keys, a_vals, b_keys, b_vals, out_keys, out_vals, stream=None):
    """Synchronous end-to-end merge of host tensors (pinned for full copy
    speed); a_vals/b_vals/out_vals may all be None for keys only."""
    pairs = a_vals is not None
    _check(lib().mp_merge_pairs_host(_dtype_code(a_keys), _host(a_keys, "a_keys"),
                                     _host(a_vals, "a_vals") if pairs else None, a_keys.numel(),
                                     _host(b_keys, "b_keys"), _host(b_vals, "b_vals") if pairs else None,
                                     b_keys.numel(), _host(out_keys, "out_keys"),
                                     _host(out_vals, "out_vals") if pairs else None, _stream(stream)))
    return (out_keys, out_vals) if pairs else out_keys


def mp_merge_path_partition(a, b, spacing: int, out=None, stream=None, descending: bool = False,
                            wide: str | None = None):
    """Split points (Alg. 2) at diagonals min(t*spacing, |a|+|b|)."""
    n = _count(a, wide) + _count(b, wide)
    nb = (n + spacing - 1) // spacing + 1
    if out is None:
        out = torch.empty(nb, dtype=torch.int64, device=a.device)
    _check(lib().mp_merge_path_partition(_kcode(a, descending, wide), _dev(a, "a"), _count(a, wide), _dev(b, "b"),
                                         _count(b, wide), int(spacing), _dev(out, "a_split"),
                                         _stream(stream)))
    return out


def mp_sort_workspace_bytes(dtype, n: int, with_values: bool) -> int:
    code = dtype if isinstance(dtype, int) else _TORCH_DTYPE[dtype]
    return int(lib().mp_sort_workspace_bytes(code, int(n), 1 if with_values else 0))


def mp_sort(keys, vals=None, workspace=None, stream=None, descending: bool = False, wide: str | None = None):
    """Stable in-place merge sort of keys (and vals)."""
    n = _count(keys, wide)
    code = _kcode(keys, descending, wide)
    need = mp_sort_workspace_bytes(code & 0xFF, n, vals is not None)
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=keys.device)
    _check(lib().mp_sort(code, _dev(keys, "keys"),
                         _vals(vals, "vals") if vals is not None else None, n,
                         _dev(workspace, "workspace"), workspace.numel(), _stream(stream)))
    return (keys, vals) if vals is not None else keys


def mp_merge_batched(a, a_off, b, b_off, out=None, a_vals=None, b_vals=None, out_vals=None,
                     na_total=None, nb_total=None, plan=None, stream=None, descending: bool = False):
    """nseg independent stable merges (offsets: int64 device tensors, nseg+1)."""
    nseg = a_off.numel() - 1
    if na_total is None:
        na_total = a.numel()
    if nb_total is None:
        nb_total = b.numel()
    n = na_total + nb_total
    if out is None:
        out = torch.empty(n, dtype=a.dtype, device=a.device)
    pairs = a_vals is not None
    if pairs and out_vals is None:
        out_vals = torch.empty(n, dtype=a_vals.dtype, device=a.device)
    _check(lib().mp_merge_batched(_dtype_code(a, descending), _dev(a, "a"), _dev(a_off, "a_off"), _dev(b, "b"),
                                  _dev(b_off, "b_off"), nseg, int(na_total), int(nb_total),
                                  _dev(out, "out"), _vals(a_vals, "a_vals") if pairs else None,
                                  _vals(b_vals, "b_vals") if pairs else None,
                                  _vals(out_vals, "out_vals") if pairs else None, _plan(plan),
                                  _stream(stream)))
    return (out, out_vals) if pairs else out


def mp_merge_grouped(problems, with_values: bool = False, stream=None):
    """Merge many independent problems in one launch.  problems: list of
    (a_keys, b_keys, out_keys) or (a_keys, a_vals, b_keys, b_vals, out_keys,
    out_vals) tuples of device tensors (one key width for all), or the
    descriptor array mp_merge_grouped_descs built from such a list (the
    tensors must stay alive)."""
    if isinstance(problems, ctypes.Array):
        _check(lib().mp_merge_grouped(problems, len(problems), 1 if with_values else 0, _stream(stream)))
        return
    arr = mp_merge_grouped_descs(problems, with_values)
    _check(lib().mp_merge_grouped(arr, len(problems), 1 if with_values else 0, _stream(stream)))


def mp_merge_grouped_descs(problems, with_values: bool = False):
    """The C descriptor array of mp_merge_grouped for a list of problems
    (building it walks the list in Python, which for many problems costs
    more than the launch itself)."""
    n = len(problems)
    arr = (mp_merge_desc * n)()
    for i, pr in enumerate(problems):
        if with_values:
            ak, av, bk, bv, ok, ov = pr
        else:
            ak, bk, ok = pr
            av = bv = ov = None
        d = arr[i]
        d.dtype = _dtype_code(ak)
        d.a_keys, d.na = _dev(ak, "a_keys"), ak.numel()
        d.b_keys, d.nb = _dev(bk, "b_keys"), bk.numel()
        d.out_keys = _dev(ok, "out_keys")
        if with_values:
            d.a_vals, d.b_vals, d.out_vals = _vals(av, "a_vals"), _vals(bv, "b_vals"), _vals(ov, "out_vals")
    return arr


def mp_check_sorted(keys, stream=None, descending: bool = False, wide: str | None = None) -> int:
    """Synchronous: MP_OK, MP_ERR_NOT_SORTED or MP_ERR_NAN."""
    return int(lib().mp_check_sorted(_kcode(keys, descending, wide), _dev(keys, "keys"), _count(keys, wide),
                                     _stream(stream)))


# --------------------------------------------------------------------- queue

def mp_kernel_error(reset: bool = False) -> int:
    """Synchronous: flags set by kernels whose bounded waits ran out (0 = none)."""
    v = ctypes.c_uint()
    _check(lib().mp_kernel_error(ctypes.byref(v), 1 if reset else 0))
    return v.value


def mp_kernel_status(reset: bool = False, stream=None) -> int:
    """Waits for the stream; the kernel error flags as a status code
    (MP_OK, MP_ERR_TIMEOUT, MP_ERR_NOT_SORTED), returned, not raised."""
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(lib().mp_kernel_status(s.cuda_stream, 1 if reset else 0))


# mp_fault
MP_FAULT_SCRATCH_ALLOC, MP_FAULT_QUEUE_STEP, MP_FAULT_STAGE_WAIT = 1, 2, 3


def mp_inject_fault(kind: int, count: int) -> None:
    """Test hook: the next `count` events of this kind fail (see mp.h)."""
    _check(lib().mp_inject_fault(int(kind), int(count)))


def mp_clock_seconds() -> float:
    return float(lib().mp_clock_seconds())


def mp_queue_create(budget_bytes: int, max_active: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().mp_queue_create(int(budget_bytes), int(max_active), ctypes.byref(h)))
    return h.value


def mp_queue_submit(q: int, req: mp_request) -> int:
    t = ctypes.c_uint64()
    _check(lib().mp_queue_submit(q, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def mp_queue_wait(q: int, ticket: int, timeout_ns: int = -1) -> mp_result:
    """Raises MPError (MP_ERR_TIMEOUT / MP_ERR_NOT_READY) if not done in time."""
    r = mp_result()
    _check(lib().mp_queue_wait(q, int(ticket), int(timeout_ns), ctypes.byref(r)))
    return r


def mp_queue_get_stats(q: int) -> dict:
    s = mp_queue_stats()
    _check(lib().mp_queue_get_stats(q, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in mp_queue_stats._fields_}


def mp_queue_destroy(q: int) -> None:
    _check(lib().mp_queue_destroy(q))


def mp_generate(dtype, keys, n: int, seed: int, stream_id: int, sorted_: bool, vals=None,
                val_base: int = 0, stream=None):
    code = dtype if isinstance(dtype, int) else _TORCH_DTYPE[dtype]
    _check(lib().mp_generate(code, _dev(keys, "keys"), _vals(vals, "vals") if vals is not None else None,
                             int(n), int(seed), int(stream_id), 1 if sorted_ else 0, int(val_base),
                             _stream(stream)))


def _ptr_any(t):
    if t is None:
        return None, None
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return t.data_ptr(), t.is_cuda


class Queue:
    """Convenience wrapper over mp_queue_* (continuous-batching request queue)."""

    def __init__(self, budget_bytes: int, max_active: int = 1024):
        self.handle = mp_queue_create(budget_bytes, max_active)
        self._keep = {}

    def _submit(self, req, keep):
        t = mp_queue_submit(self.handle, req)
        self._keep[t] = keep
        return t

    def submit_merge(self, a_keys, b_keys, out_keys, a_vals=None, b_vals=None, out_vals=None):
        """Inputs and outputs may be host or CUDA tensors (each side's kind
        is taken from its key tensor)."""
        r = mp_request()
        r.op, r.dtype = MP_OP_MERGE, _dtype_code(a_keys)
        r.with_values = 1 if a_vals is not None else 0
        r.a_keys, cuda_in = _ptr_any(a_keys)
        r.b_keys, _ = _ptr_any(b_keys)
        r.na, r.nb = a_keys.numel(), b_keys.numel()
        r.source = MP_SRC_DEVICE if cuda_in else MP_SRC_HOST
        r.out_keys, cuda_out = _ptr_any(out_keys)
        r.sink = MP_SINK_DEVICE if cuda_out else MP_SINK_HOST
        if a_vals is not None:
            r.a_vals, _ = _ptr_any(a_vals)
            r.b_vals, _ = _ptr_any(b_vals)
            r.out_vals, _ = _ptr_any(out_vals)
        return self._submit(r, (a_keys, b_keys, out_keys, a_vals, b_vals, out_vals))

    def submit_sort(self, keys, out_keys, vals=None, out_vals=None):
        r = mp_request()
        r.op, r.dtype = MP_OP_SORT, _dtype_code(keys)
        r.with_values = 1 if vals is not None else 0
        r.a_keys, cuda_in = _ptr_any(keys)
        r.na = keys.numel()
        r.source = MP_SRC_DEVICE if cuda_in else MP_SRC_HOST
        r.out_keys, cuda_out = _ptr_any(out_keys)
        r.sink = MP_SINK_DEVICE if cuda_out else MP_SINK_HOST
        if vals is not None:
            r.a_vals, _ = _ptr_any(vals)
            r.out_vals, _ = _ptr_any(out_vals)
        return self._submit(r, (keys, out_keys, vals, out_vals))

    def submit_generated(self, op: int, dtype: int, na: int, nb: int, seed: int, with_values=True,
                         out_keys=None, out_vals=None):
        """Synthetic request generated on the device (mp_generate); result
        discarded unless output tensors are given."""
        r = mp_request()
        r.op, r.dtype, r.with_values = op, dtype, 1 if with_values else 0
        r.source, r.na, r.nb, r.seed = MP_SRC_GENERATE, int(na), int(nb), int(seed)
        if out_keys is None:
            r.sink = MP_SINK_DISCARD
        else:
            r.out_keys, cuda_out = _ptr_any(out_keys)
            r.out_vals, _ = _ptr_any(out_vals)
            r.sink = MP_SINK_DEVICE if cuda_out else MP_SINK_HOST
        return self._submit(r, (out_keys, out_vals))

    def wait(self, ticket: int, timeout_s: float | None = None) -> mp_result:
        ns = -1 if timeout_s is None else int(timeout_s * 1e9)
        r = mp_queue_wait(self.handle, ticket, ns)
        self._keep.pop(ticket, None)
        return r

    def stats(self) -> dict:
        return mp_queue_get_stats(self.handle)

    def close(self):
        if self.handle:
            mp_queue_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# --------------------------------------------------------------------- tuning

def mp_autotune_merge(a_keys, b_keys, a_vals=None, b_vals=None, out_keys=None, out_vals=None,
                      reps: int = 3, stream=None):
    """Time every compiled tile shape on this problem; returns the best
    (block_threads, items_per_thread, staging) and records it."""
    n = a_keys.numel() + b_keys.numel()
    if out_keys is None:
        out_keys = torch.empty(n, dtype=a_keys.dtype, device=a_keys.device)
    pairs = a_vals is not None
    if pairs and out_vals is None:
        out_vals = torch.empty(n, dtype=a_vals.dtype, device=a_keys.device)
    best = mp_plan()
    _check(lib().mp_autotune_merge(_dtype_code(a_keys), _dev(a_keys, "a_keys"),
                                   _vals(a_vals, "a_vals") if pairs else None, a_keys.numel(),
                                   _dev(b_keys, "b_keys"), _vals(b_vals, "b_vals") if pairs else None,
                                   b_keys.numel(), _dev(out_keys, "out_keys"),
                                   _vals(out_vals, "out_vals") if pairs else None, int(reps),
                                   ctypes.byref(best), _stream(stream)))
    return best.block_threads, best.items_per_thread, best.staging


def mp_autotune_batched(a, a_off, b, b_off, out=None, a_vals=None, b_vals=None, out_vals=None,
                        reps: int = 3, stream=None):
    nseg = a_off.numel() - 1
    n = a.numel() + b.numel()
    if out is None:
        out = torch.empty(n, dtype=a.dtype, device=a.device)
    pairs = a_vals is not None
    if pairs and out_vals is None:
        out_vals = torch.empty(n, dtype=a_vals.dtype, device=a.device)
    best = mp_plan()
    _check(lib().mp_autotune_batched(_dtype_code(a), _dev(a, "a"), _dev(a_off, "a_off"), _dev(b, "b"),
                                     _dev(b_off, "b_off"), nseg, a.numel(), b.numel(), _dev(out, "out"),
                                     _vals(a_vals, "a_vals") if pairs else None,
                                     _vals(b_vals, "b_vals") if pairs else None,
                                     _vals(out_vals, "out_vals") if pairs else None, int(reps),
                                     ctypes.byref(best), _stream(stream)))
    return best.block_threads, best.items_per_thread, best.staging


def mp_tune_save(path: str) -> None:
    _check(lib().mp_tune_save(os.fsencode(path)))


def mp_tune_load(path: str) -> None:
    _check(lib().mp_tune_load(os.fsencode(path)))


def mp_tune_clear() -> None:
    lib().mp_tune_clear()


# --------------------------------------------------------------------- graphs

class Graph:
    """A captured merge (mp_graph_*): replay() enqueues it with one launch."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def replay(self, stream=None):
        _check(lib().mp_graph_launch(self.handle, _stream(stream)))

    def close(self):
        if self.handle:
            _check(lib().mp_graph_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mp_graph_merge_create(a_keys, b_keys, out_keys, a_vals=None, b_vals=None, out_vals=None, plan=None):
    h = ctypes.c_void_p()
    pairs = a_vals is not None
    _check(lib().mp_graph_merge_create(_dtype_code(a_keys), _dev(a_keys, "a_keys"),
                                       _vals(a_vals, "a_vals") if pairs else None, a_keys.numel(),
                                       _dev(b_keys, "b_keys"), _vals(b_vals, "b_vals") if pairs else None,
                                       b_keys.numel(), _dev(out_keys, "out_keys"),
                                       _vals(out_vals, "out_vals") if pairs else None, _plan(plan),
                                       ctypes.byref(h)))
    return Graph(h.value, (a_keys, b_keys, out_keys, a_vals, b_vals, out_vals))


def mp_graph_batched_create(a, a_off, b, b_off, out, a_vals=None, b_vals=None, out_vals=None,
                            plan=None):
    h = ctypes.c_void_p()
    pairs = a_vals is not None
    _check(lib().mp_graph_batched_create(_dtype_code(a), _dev(a, "a"), _dev(a_off, "a_off"), _dev(b, "b"),
                                         _dev(b_off, "b_off"), a_off.numel() - 1, a.numel(), b.numel(),
                                         _dev(out, "out"), _vals(a_vals, "a_vals") if pairs else None,
                                         _vals(b_vals, "b_vals") if pairs else None,
                                         _vals(out_vals, "out_vals") if pairs else None, _plan(plan),
                                         ctypes.byref(h)))
    return Graph(h.value, (a, a_off, b, b_off, out, a_vals, b_vals, out_vals))
