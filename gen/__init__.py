"""Seeded synthetic inputs shaped like the paper's merge and sort workloads.

This module is shared by the tests, the bench and the smoke check.  It holds
no merge or sort arithmetic of the method: it draws random numbers and, where
a workload asks for sorted arrays, orders them with ``numpy.sort`` (input
preparation, not the operation under test).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: element i of stream s under seed k is
``mix(k ^ (s * 0xD1B54A32D192ED03) + (i + 1) * 0x9E3779B97F4A7C15)`` where
``mix`` is SplitMix64's finaliser.  The base seed is 0x14062628.

Workloads (sizes are parameters so that tests can run scaled-down copies):

* ``plain_keys``   two int32 arrays uniform in [0, 2^24), sorted (ties occur)
* ``large_kv``     uint64 keys + uint32 payload = global source index; four
                   key distributions: uniform, a_gt_b (every A key above
                   every B key, the case that defeats naive equal splitting),
                   interleaved (strictly alternating ranks), distinct16
* ``sort_input``   int32 or float32 (all bit patterns, NaN redrawn) in four
                   orders: random, sorted, reverse, distinct256
* ``batched``      many int32 merge pairs, per-side length floor(2^U),
                   U ~ Uniform[0, log2_max], each side uniform [0, 2^31), sorted
* ``sets``         two duplicate-free int32 sets: each key of [0, 2^u) is in A
                   with probability 1/2 and, independently, in B with
                   probability 1/2 (adjacency-list-like sets sharing half)
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 0x14062628

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n uint64 draws: elements start..start+n-1 of stream ``stream``."""
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * _STREAM_MUL)
        z = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z *= _GAMMA
        z += base
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def uniform_below(seed: int, stream: int, n: int, bound: int) -> np.ndarray:
    """n uint64 draws uniform in [0, bound) (high 64x64 product, bound <= 2^32
    exact; larger bounds use the multiply-high of the top 32 bits)."""
    x = splitmix64(seed, stream, n)
    if bound <= (1 << 32):
        return ((x >> np.uint64(32)) * np.uint64(bound)) >> np.uint64(32)
    if bound == (1 << 64):
        return x
    return x % np.uint64(bound)


# --------------------------------------------------------------------------
# Workload 1: plain keys-only merge.
# --------------------------------------------------------------------------

def plain_keys(n_a: int = 1 << 20, n_b: int = 1 << 20, key_range: int = 1 << 24,
               seed: int = BASE_SEED):
    a = np.sort(uniform_below(seed, 1, n_a, key_range).astype(np.int32))
    b = np.sort(uniform_below(seed, 2, n_b, key_range).astype(np.int32))
    return a, b


# --------------------------------------------------------------------------
# Workload 2: large unbalanced key-value merge (uint64 keys, uint32 payloads).
# --------------------------------------------------------------------------

LARGE_KV_DISTS = ("uniform", "a_gt_b", "interleaved", "distinct16")


def large_kv(dist: str, n_a: int = 1 << 28, n_b: int = 1 << 26, seed: int = BASE_SEED):
    """Returns (a_keys, a_vals, b_keys, b_vals); payload = global source index
    (A element i carries i, B element j carries n_a + j)."""
    if dist == "uniform":
        a = np.sort(splitmix64(seed, 11, n_a))
        b = np.sort(splitmix64(seed, 12, n_b))
    elif dist == "a_gt_b":
        top = np.uint64(1 << 63)
        a = np.sort(splitmix64(seed, 13, n_a) | top)
        b = np.sort(splitmix64(seed, 14, n_b) & ~top)
    elif dist == "interleaved":
        # Ranks 0..n-1 of the merged output are dealt to A and B as evenly as
        # the sizes allow (B takes rank r iff floor((r+1)nb/n) > floor(r nb/n)),
        # and rank r gets key r * floor(2^64 / n): all keys distinct.
        n = n_a + n_b
        r = np.arange(n, dtype=np.uint64)
        to_b = ((r + np.uint64(1)) * np.uint64(n_b)) // np.uint64(n) > (r * np.uint64(n_b)) // np.uint64(n) \
            if n_b else np.zeros(n, dtype=bool)
        step = np.uint64((1 << 64) // max(n, 1))
        with np.errstate(over="ignore"):
            keys = r * step
        a = keys[~to_b]
        b = keys[to_b]
    elif dist == "distinct16":
        values = splitmix64(seed, 15, 16)
        a = np.sort(values[uniform_below(seed, 16, n_a, 16)])
        b = np.sort(values[uniform_below(seed, 17, n_b, 16)])
    else:
        raise ValueError(f"unknown distribution {dist!r}")
    av = np.arange(n_a, dtype=np.uint32)
    bv = np.arange(n_a, n_a + n_b, dtype=np.uint64).astype(np.uint32)
    return a, av, b, bv


# --------------------------------------------------------------------------
# Workload 3: merge sort inputs.
# --------------------------------------------------------------------------

SORT_ORDERS = ("random", "sorted", "reverse", "distinct256")


def _f32_no_nan(seed: int, stream: int, n: int) -> np.ndarray:
    bits = (splitmix64(seed, stream, n) >> np.uint64(32)).astype(np.uint32)
    f = bits.view(np.float32)
    redraw = 0
    while True:
        bad = np.flatnonzero(np.isnan(f))
        if bad.size == 0:
            return f
        redraw += 1
        fresh = (splitmix64(seed, stream + 1000 * redraw, n)[bad] >> np.uint64(32)).astype(np.uint32)
        bits[bad] = fresh


def sort_input(dtype: str, order: str, n: int = 1 << 28, seed: int = BASE_SEED) -> np.ndarray:
    """dtype 'i32' (uniform over all int32) or 'f32' (uniform over all bit
    patterns, NaN redrawn: covers +-0, +-inf and denormals)."""
    if dtype == "i32":
        def draw(stream, m):
            return (splitmix64(seed, stream, m) >> np.uint64(32)).astype(np.uint32).view(np.int32)
    elif dtype == "f32":
        def draw(stream, m):
            return _f32_no_nan(seed, stream, m)
    else:
        raise ValueError(f"unknown dtype {dtype!r}")
    if order == "random":
        return draw(21, n)
    if order == "sorted":
        return np.sort(draw(22, n))
    if order == "reverse":
        return np.sort(draw(23, n))[::-1].copy()
    if order == "distinct256":
        values = draw(24, 256)
        return values[uniform_below(seed, 25, n, 256)]
    raise ValueError(f"unknown order {order!r}")


# --------------------------------------------------------------------------
# Workload 4: batched segmented merge.
# --------------------------------------------------------------------------

def batched_lengths(n_seg: int = 16384, log2_max: float = 18.0, seed: int = BASE_SEED,
                    min_len: int = 1):
    """Per-side lengths floor(2^U), U ~ Uniform[0, log2_max]; returns
    (len_a, len_b) int64 arrays."""
    def one(stream):
        u = (splitmix64(seed, stream, n_seg) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
        return np.maximum(np.floor(np.exp2(u * log2_max)).astype(np.int64), min_len)
    return one(31), one(32)


def batched(n_seg: int = 16384, log2_max: float = 18.0, seed: int = BASE_SEED,
            len_a=None, len_b=None, with_values: bool = False):
    """Returns (a, a_off, b, b_off[, av, bv]): int32 keys uniform in
    [0, 2^31), each segment sorted; offsets are int64 with n_seg+1 entries.
    Payloads (if asked) are global source indices, B after all of A."""
    if len_a is None:
        len_a, len_b = batched_lengths(n_seg, log2_max, seed)
    len_a = np.asarray(len_a, dtype=np.int64)
    len_b = np.asarray(len_b, dtype=np.int64)
    a_off = np.zeros(len_a.size + 1, dtype=np.int64)
    b_off = np.zeros(len_b.size + 1, dtype=np.int64)
    np.cumsum(len_a, out=a_off[1:])
    np.cumsum(len_b, out=b_off[1:])

    def side(stream, off, lens):
        keys = (splitmix64(seed, stream, int(off[-1])) >> np.uint64(33)).astype(np.int64)
        # Sort every segment at once: order by (segment id, key).
        seg = np.repeat(np.arange(lens.size, dtype=np.int64), lens)
        keys = np.sort((seg << 32) | keys) & 0xFFFFFFFF
        return keys.astype(np.int32)

    a = side(41, a_off, len_a)
    b = side(42, b_off, len_b)
    if not with_values:
        return a, a_off, b, b_off
    av = np.arange(a.size, dtype=np.uint32)
    bv = np.arange(a.size, a.size + b.size, dtype=np.uint64).astype(np.uint32)
    return a, a_off, b, b_off, av, bv


# --------------------------------------------------------------------------
# Set-operation inputs.
# --------------------------------------------------------------------------

def sets(log2_universe: int = 28, seed: int = BASE_SEED):
    """(a, b): the keys of [0, 2^log2_universe) whose membership bit is set,
    one independent fair bit per key and side (streams 51 and 52), ascending
    int32."""
    words = max(1, (1 << log2_universe) // 64)

    def side(stream):
        bits = np.unpackbits(splitmix64(seed, stream, words).view(np.uint8), bitorder="little")
        return np.flatnonzero(bits[: 1 << log2_universe]).astype(np.int32)

    return side(51), side(52)


# --------------------------------------------------------------------------
# The device generator's definition (mp_generate / MP_SRC_GENERATE), restated
# in numpy so that generated requests can be checked on the host.
# --------------------------------------------------------------------------

def device_generated(n: int, seed: int, stream: int, sorted_: bool, key_bits: int = 32,
                     val_base: int = 0):
    """keys (uint32 or uint64) and uint32 values val_base + i."""
    x = splitmix64(seed, stream, n)
    if sorted_:
        if key_bits == 32:
            stride = max(1, (1 << 32) // max(n, 1))
        else:
            stride = max(1, ((1 << 64) - 1) // max(n, 1))
        with np.errstate(over="ignore"):
            k = np.arange(n, dtype=np.uint64) * np.uint64(stride) + x % np.uint64(stride)
    else:
        k = x if key_bits == 64 else (x >> np.uint64(32))
    keys = k.astype(np.uint32) if key_bits == 32 else k
    vals = (np.arange(n, dtype=np.uint64) + np.uint64(val_base)).astype(np.uint32)
    return keys, vals


def serving_request(op: str, na: int, nb: int, seed: int, key_bits: int = 32):
    """Inputs of a generated queue request: merge -> (a, av, b, bv) with
    streams 1 and 2 (B's values continue after A's); sort -> (keys, vals)
    with stream 3."""
    if op == "merge":
        a, av = device_generated(na, seed, 1, True, key_bits, 0)
        b, bv = device_generated(nb, seed, 2, True, key_bits, na)
        return a, av, b, bv
    return device_generated(na, seed, 3, False, key_bits, 0)
