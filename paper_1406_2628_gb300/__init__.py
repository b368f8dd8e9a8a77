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

MP_STAGE_AUTO, MP_STAGE_VECTOR, MP_STAGE_BULK = 0, 1, 2

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


def _dtype_code(t: torch.Tensor) -> int:
    try:
        return _TORCH_DTYPE[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported key dtype {t.dtype}") from None


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
                  stream=None) -> torch.Tensor:
    """Stable merge of sorted 1-D tensors a and b (ties: a first)."""
    if a.dtype != b.dtype:
        raise TypeError("a and b must have the same dtype")
    if out is None:
        out = torch.empty(a.numel() + b.numel(), dtype=a.dtype, device=a.device)
    _check(lib().mp_merge_keys(_dtype_code(a), _dev(a, "a"), a.numel(), _dev(b, "b"), b.numel(),
                               _dev(out, "out"), _stream(stream)))
    return out


def mp_merge_pairs(a_keys, a_vals, b_keys, b_vals, out_keys=None, out_vals=None, stream=None):
    """Stable merge moving a uint32 payload with each key."""
    if a_keys.dtype != b_keys.dtype:
        raise TypeError("key dtypes differ")
    n = a_keys.numel() + b_keys.numel()
    if out_keys is None:
        out_keys = torch.empty(n, dtype=a_keys.dtype, device=a_keys.device)
    if out_vals is None:
        out_vals = torch.empty(n, dtype=a_vals.dtype, device=a_keys.device)
    _check(lib().mp_merge_pairs(_dtype_code(a_keys), _dev(a_keys, "a_keys"), _vals(a_vals, "a_vals"),
                                a_keys.numel(), _dev(b_keys, "b_keys"), _vals(b_vals, "b_vals"),
                                b_keys.numel(), _dev(out_keys, "out_keys"), _vals(out_vals, "out_vals"),
                                _stream(stream)))
    return out_keys, out_vals


def mp_merge_plan(a_keys, b_keys, a_vals=None, b_vals=None, out_keys=None, out_vals=None,
                  plan=None, stream=None):
    """Merge with an explicit tile plan (block_threads, items_per_thread[, staging])."""
    n = a_keys.numel() + b_keys.numel()
    if out_keys is None:
        out_keys = torch.empty(n, dtype=a_keys.dtype, device=a_keys.device)
    pairs = a_vals is not None
    if pairs and out_vals is None:
        out_vals = torch.empty(n, dtype=a_vals.dtype, device=a_keys.device)
    _check(lib().mp_merge_plan(_dtype_code(a_keys), _dev(a_keys, "a_keys"),
                               _vals(a_vals, "a_vals") if pairs else None, a_keys.numel(),
                               _dev(b_keys, "b_keys"), _vals(b_vals, "b_vals") if pairs else None,
                               b_keys.numel(), _dev(out_keys, "out_keys"),
                               _vals(out_vals, "out_vals") if pairs else None, _plan(plan),
                               _stream(stream)))
    return (out_keys, out_vals) if pairs else out_keys


def mp_plan_supported(plan) -> bool:
    p = plan if isinstance(plan, mp_plan) else mp_plan(int(plan[0]), int(plan[1]),
                                                       int(plan[2]) if len(plan) > 2 else 0, 0)
    return bool(lib().mp_plan_supported(ctypes.byref(p)))


def mp_merge_tile_items(dtype, with_values: bool, total: int, plan=None) -> int:
    code = dtype if isinstance(dtype, int) else _TORCH_DTYPE[dtype]
    return int(lib().mp_merge_tile_items(code, 1 if with_values else 0, int(total), _plan(plan)))


def mp_merge_partitioned(a_keys, b_keys, a_split, a_vals=None, b_vals=None, out_keys=None,
                         out_vals=None, plan=None, stream=None):
    """The merge kernel alone over split points from mp_merge_path_partition
    (spacing = mp_merge_tile_items(...))."""
    n = a_keys.numel() + b_keys.numel()
    if out_keys is None:
        out_keys = torch.empty(n, dtype=a_keys.dtype, device=a_keys.device)
    pairs = a_vals is not None
    if pairs and out_vals is None:
        out_vals = torch.empty(n, dtype=a_vals.dtype, device=a_keys.device)
    _check(lib().mp_merge_partitioned(_dtype_code(a_keys), _dev(a_keys, "a_keys"),
                                      _vals(a_vals, "a_vals") if pairs else None, a_keys.numel(),
                                      _dev(b_keys, "b_keys"), _vals(b_vals, "b_vals") if pairs else None,
                                      b_keys.numel(), _dev(out_keys, "out_keys"),
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


def mp_merge_path_partition(a, b, spacing: int, out=None, stream=None):
    """Split points (Alg. 2) at diagonals min(t*spacing, |a|+|b|)."""
    n = a.numel() + b.numel()
    nb = (n + spacing - 1) // spacing + 1
    if out is None:
        out = torch.empty(nb, dtype=torch.int64, device=a.device)
    _check(lib().mp_merge_path_partition(_dtype_code(a), _dev(a, "a"), a.numel(), _dev(b, "b"),
                                         b.numel(), int(spacing), _dev(out, "a_split"),
                                         _stream(stream)))
    return out


def mp_sort_workspace_bytes(dtype, n: int, with_values: bool) -> int:
    code = dtype if isinstance(dtype, int) else _TORCH_DTYPE[dtype]
    return int(lib().mp_sort_workspace_bytes(code, int(n), 1 if with_values else 0))


def mp_sort(keys, vals=None, workspace=None, stream=None):
    """Stable in-place merge sort of keys (and vals)."""
    n = keys.numel()
    need = mp_sort_workspace_bytes(keys.dtype, n, vals is not None)
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=keys.device)
    _check(lib().mp_sort(_dtype_code(keys), _dev(keys, "keys"),
                         _vals(vals, "vals") if vals is not None else None, n,
                         _dev(workspace, "workspace"), workspace.numel(), _stream(stream)))
    return (keys, vals) if vals is not None else keys


def mp_merge_batched(a, a_off, b, b_off, out=None, a_vals=None, b_vals=None, out_vals=None,
                     na_total=None, nb_total=None, plan=None, stream=None):
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
    _check(lib().mp_merge_batched(_dtype_code(a), _dev(a, "a"), _dev(a_off, "a_off"), _dev(b, "b"),
                                  _dev(b_off, "b_off"), nseg, int(na_total), int(nb_total),
                                  _dev(out, "out"), _vals(a_vals, "a_vals") if pairs else None,
                                  _vals(b_vals, "b_vals") if pairs else None,
                                  _vals(out_vals, "out_vals") if pairs else None, _plan(plan),
                                  _stream(stream)))
    return (out, out_vals) if pairs else out


def mp_check_sorted(keys, stream=None) -> int:
    """Synchronous: MP_OK, MP_ERR_NOT_SORTED or MP_ERR_NAN."""
    return int(lib().mp_check_sorted(_dtype_code(keys), _dev(keys, "keys"), keys.numel(),
                                     _stream(stream)))
