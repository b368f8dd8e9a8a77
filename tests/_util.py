"""Helpers for the GPU tests: numpy <-> torch transfers that keep bit
patterns (torch has limited uint32/uint64 support, so those travel as
int32/int64 and are viewed back)."""
import numpy as np
import torch

_SIGNED_VIEW = {
    np.dtype(np.uint32): (np.int32, torch.uint32),
    np.dtype(np.uint64): (np.int64, torch.uint64),
}


def to_dev(x: np.ndarray, dev="cuda") -> torch.Tensor:
    x = np.ascontiguousarray(x)
    if x.dtype in _SIGNED_VIEW:
        signed, tdt = _SIGNED_VIEW[x.dtype]
        return torch.from_numpy(x.view(signed)).to(dev).view(tdt)
    return torch.from_numpy(x).to(dev)


def vals_to_dev(v: np.ndarray, dev="cuda") -> torch.Tensor:
    """uint32 payloads as an int32 device tensor (bit pattern kept)."""
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.uint32).view(np.int32)).to(dev)


def to_host(t: torch.Tensor, np_dtype) -> np.ndarray:
    np_dtype = np.dtype(np_dtype)
    if np_dtype in _SIGNED_VIEW:
        signed, _ = _SIGNED_VIEW[np_dtype]
        tt = {np.int32: torch.int32, np.int64: torch.int64}[signed]
        return t.view(tt).cpu().numpy().view(np_dtype)
    return t.cpu().numpy().view(np_dtype)


def same_bits(x: np.ndarray, y: np.ndarray) -> bool:
    return x.shape == y.shape and np.array_equal(np.ascontiguousarray(x).view(np.uint8),
                                                 np.ascontiguousarray(y).view(np.uint8))


def first_mismatch(x: np.ndarray, y: np.ndarray):
    xb = np.ascontiguousarray(x)
    yb = np.ascontiguousarray(y)
    if xb.shape != yb.shape:
        return f"shape {xb.shape} vs {yb.shape}"
    w = xb.dtype.itemsize
    bad = np.flatnonzero((xb.view(np.uint8).reshape(-1, w) != yb.view(np.uint8).reshape(-1, w)).any(1))
    if bad.size == 0:
        return None
    i = int(bad[0])
    return f"{bad.size} mismatches, first at {i}: {xb[i]!r} vs {yb[i]!r}"


def random_sorted(rng, np_dtype, n, kind="random"):
    """Sorted keys of a given dtype; kinds: random (wide range), ties (few
    distinct values), equal (all equal)."""
    np_dtype = np.dtype(np_dtype)
    if kind == "equal":
        x = np.full(n, 7, dtype=np.int64)
    elif kind == "ties":
        x = rng.integers(-8 if np_dtype.kind in "if" else 0, 8, n)
    else:
        if np_dtype.itemsize == 8:
            x = rng.integers(0, 1 << 63, n, dtype=np.uint64)
            if np_dtype.kind == "i":
                x = x.view(np.int64) - np.int64(1 << 62)
        else:
            x = rng.integers(-(1 << 31) if np_dtype.kind in "if" else 0,
                             (1 << 31) if np_dtype.kind in "if" else (1 << 32), n)
    if np_dtype.kind == "f":
        x = np.asarray(x, dtype=np.float64).astype(np.float32)
        if kind != "equal" and n:
            # Both zeros (distinct under the float order) and infinities.
            pick = rng.random(n)
            x[pick < 0.05] = np.float32(-0.0)
            x[(pick >= 0.05) & (pick < 0.10)] = np.float32(0.0)
            x[(pick >= 0.10) & (pick < 0.11)] = np.float32(np.inf)
            x[(pick >= 0.11) & (pick < 0.12)] = np.float32(-np.inf)
        # Order by value, -0.0 before +0.0.
        order = np.lexsort((~np.signbit(x), x))
        return x[order]
    return np.sort(np.asarray(x).astype(np_dtype))
