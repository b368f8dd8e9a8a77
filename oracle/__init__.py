"""Plain CPU oracle for Merge Path (Green, Odeh, Birk) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never imports it and
the two share no code.

The arithmetic lives in ``mp_oracle.c`` (plain single-threaded C, one
function per step of the method, each citing the paper).  This module only
compiles that file with gcc, loads it with ctypes and marshals numpy arrays:

* ``merge``          stable two-pointer merge, ties take A (Sec. I, Sec. II.A)
* ``split``          Alg. 2 diagonal intersection -> (a_start, steps)
* ``sort``           bottom-up merge sort (Sec. I, Sec. III), stable
* ``merge_batched``  one merge per segment at offset a_off[s]+b_off[s] (Cor. 6)
* ``set_op``         union / intersection / difference / symmetric difference
                     of sorted inputs, multiset semantics (merge walk, Sec. I)

Key order: integers natural; float32 numeric with -0.0 before +0.0 (no NaN).
128-bit keys (``kind="u128"`` or ``"i128"``) are uint64 arrays of shape (n, 2),
the low word first in each row.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

_SFX = {
    np.dtype(np.int32): "i32",
    np.dtype(np.uint32): "u32",
    np.dtype(np.float32): "f32",
    np.dtype(np.uint64): "u64",
    np.dtype(np.int64): "i64",
}

_lock = threading.Lock()
_lib = None


def compile_source(src: str, out: str) -> str:
    """gcc -O2 a C source into a shared library (portable flags only)."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-Wall", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile mp_oracle.c into liboracle.so beside it."""
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        compile_source(_SRC, _LIB_PATH)
    return _LIB_PATH


def load_library(path: str):
    """ctypes-load an oracle build and declare its functions."""
    lib = ctypes.CDLL(path)
    p, i64 = ctypes.c_void_p, ctypes.c_int64
    for sfx in list(_SFX.values()) + list(WIDE):
        f = getattr(lib, f"oracle_merge_{sfx}")
        f.argtypes = [p, p, i64, p, p, i64, p, p]
        f.restype = None
        f = getattr(lib, f"oracle_split_{sfx}")
        f.argtypes = [p, i64, p, i64, i64, ctypes.POINTER(i64)]
        f.restype = i64
        f = getattr(lib, f"oracle_sort_{sfx}")
        f.argtypes = [p, p, i64]
        f.restype = ctypes.c_int
        f = getattr(lib, f"oracle_merge_batched_{sfx}")
        f.argtypes = [p, p, p, p, p, p, i64, p, p]
        f.restype = None
        f = getattr(lib, f"oracle_set_op_{sfx}")
        f.argtypes = [ctypes.c_int, p, p, i64, p, p, i64, p, p]
        f.restype = i64
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


WIDE = ("u128", "i128")


def _wide(x):
    """A 128-bit key array as a contiguous (n, 2) uint64 array."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    return x.reshape(-1, 2)


def _sfx(*arrays, kind=None):
    if kind is not None:
        if kind not in WIDE:
            raise TypeError(f"unknown key kind {kind}")
        return kind
    dt = arrays[0].dtype
    for x in arrays[1:]:
        if x.dtype != dt:
            raise TypeError(f"key dtypes differ: {dt} vs {x.dtype}")
    if dt not in _SFX:
        raise TypeError(f"unsupported key dtype {dt}")
    return _SFX[dt]


def _ptr(x):
    return None if x is None else x.ctypes.data_as(ctypes.c_void_p)


def _c(x, dtype=None):
    if x is None:
        return None
    return np.ascontiguousarray(x, dtype=dtype)


def _keys(x, kind):
    """(array, count) for a key array of the given kind (None: numpy dtype)."""
    if kind in WIDE:
        x = _wide(x)
        return x, x.shape[0]
    x = _c(x)
    return x, x.size


def _empty_like_keys(a, n, kind):
    return np.empty((n, 2), dtype=np.uint64) if kind in WIDE else np.empty(n, dtype=a.dtype)


def merge(a, b, av=None, bv=None, lib=None, kind=None):
    """Stable merge of sorted a and b; returns (keys, values or None)."""
    a, na = _keys(a, kind)
    b, nb = _keys(b, kind)
    sfx = _sfx(a, b, kind=kind)
    pairs = av is not None
    if pairs != (bv is not None):
        raise ValueError("give values for both sides or for neither")
    av, bv = _c(av, np.uint32), _c(bv, np.uint32)
    out = _empty_like_keys(a, na + nb, kind)
    outv = np.empty(na + nb, dtype=np.uint32) if pairs else None
    getattr(lib or _load(), f"oracle_merge_{sfx}")(_ptr(a), _ptr(av), na, _ptr(b),
                                            _ptr(bv), nb, _ptr(out), _ptr(outv))
    return out, outv


def split(a, b, diag, lib=None, kind=None):
    """Alg. 2: returns (a_start, steps) for cross diagonal ``diag``."""
    a, na = _keys(a, kind)
    b, nb = _keys(b, kind)
    sfx = _sfx(a, b, kind=kind)
    steps = ctypes.c_int64(0)
    r = getattr(lib or _load(), f"oracle_split_{sfx}")(_ptr(a), na, _ptr(b), nb,
                                                int(diag), ctypes.byref(steps))
    if r == -1:
        raise ValueError(f"diagonal {diag} outside [0, {na + nb}]")
    if r < 0:
        raise ValueError("diagonal search failed: inputs are not sorted")
    return int(r), int(steps.value)


def sort(keys, vals=None, lib=None, kind=None):
    """Stable bottom-up merge sort; returns sorted copies (keys, values)."""
    if kind in WIDE:
        k = _wide(keys).copy()
        n = k.shape[0]
    else:
        k = np.array(keys, copy=True)
        n = k.size
    sfx = _sfx(k, kind=kind)
    v = None if vals is None else np.array(vals, dtype=np.uint32, copy=True)
    if getattr(lib or _load(), f"oracle_sort_{sfx}")(_ptr(k), _ptr(v), n) != 0:
        raise MemoryError("oracle sort: out of host memory")
    return k, v


def merge_batched(a, a_off, b, b_off, av=None, bv=None, lib=None):
    """Per-segment stable merge; segment s lands at a_off[s] + b_off[s]."""
    a, b = _c(a), _c(b)
    sfx = _sfx(a, b)
    a_off = _c(a_off, np.int64)
    b_off = _c(b_off, np.int64)
    nseg = a_off.size - 1
    if b_off.size != a_off.size:
        raise ValueError("a_off and b_off must have the same length")
    pairs = av is not None
    av, bv = _c(av, np.uint32), _c(bv, np.uint32)
    out = np.empty(a.size + b.size, dtype=a.dtype)
    outv = np.empty(a.size + b.size, dtype=np.uint32) if pairs else None
    getattr(lib or _load(), f"oracle_merge_batched_{sfx}")(
        _ptr(a), _ptr(av), _ptr(a_off), _ptr(b), _ptr(bv), _ptr(b_off), nseg,
        _ptr(out), _ptr(outv))
    return out, outv


SET_OPS = {"union": 0, "intersection": 1, "difference": 2, "symmetric_difference": 3}


def set_op(op, a, b, av=None, bv=None, lib=None, kind=None):
    """Set operation ``op`` (a name in SET_OPS or its code) of sorted a and b,
    multiset semantics; returns (keys, values or None), trimmed to length."""
    code = SET_OPS[op] if isinstance(op, str) else int(op)
    a, na = _keys(a, kind)
    b, nb = _keys(b, kind)
    sfx = _sfx(a, b, kind=kind)
    pairs = av is not None
    if pairs != (bv is not None):
        raise ValueError("give values for both sides or for neither")
    av, bv = _c(av, np.uint32), _c(bv, np.uint32)
    out = _empty_like_keys(a, na + nb, kind)
    outv = np.empty(na + nb, dtype=np.uint32) if pairs else None
    k = getattr(lib or _load(), f"oracle_set_op_{sfx}")(code, _ptr(a), _ptr(av), na, _ptr(b),
                                                   _ptr(bv), nb, _ptr(out), _ptr(outv))
    return out[:k].copy(), (outv[:k].copy() if pairs else None)
