"""The on-chip merge (mp_merge_checksum, the paper's 'results written to a
register' experiment): its digest equals the same digest computed on the
host from the oracle's merged output, for every dtype, with and without
values, and for edge sizes."""
import numpy as np
import pytest

import oracle
import paper_1406_2628_gb300 as mp
from _util import random_sorted, to_dev, vals_to_dev

pytestmark = pytest.mark.gpu

DTYPES = [np.int32, np.uint32, np.float32, np.uint64, np.int64]


def digest(keys, vals):
    """sum_j f(k_j, v_j, j) mod 2^64, f as documented for mp_merge_checksum."""
    bits = keys.view(np.uint64 if keys.dtype.itemsize == 8 else np.uint32).astype(np.uint64)
    with np.errstate(over="ignore"):
        h = bits * np.uint64(0x9E3779B97F4A7C15)
        if vals is not None:
            h ^= vals.astype(np.uint64) * np.uint64(0xBF58476D1CE4E5B9)
        h ^= (np.arange(bits.size, dtype=np.uint64) + np.uint64(1)) * np.uint64(0x94D049BB133111EB)
        h ^= h >> np.uint64(29)
        return int(h.sum(dtype=np.uint64)) if h.size else 0


@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: np.dtype(d).name)
def test_checksum_matches_oracle_digest(dt):
    rng = np.random.default_rng(3000)
    for na, nb in [(0, 0), (1, 0), (0, 3), (5, 7), (70_001, 33_333), (1 << 20, (1 << 19) + 3)]:
        a, b = random_sorted(rng, dt, na, "ties"), random_sorted(rng, dt, nb, "ties")
        av = np.arange(na, dtype=np.uint32)
        bv = np.arange(na, na + nb, dtype=np.uint32)
        ek, ev = oracle.merge(a, b, av, bv)
        got = mp.mp_merge_checksum(to_dev(a), to_dev(b), vals_to_dev(av), vals_to_dev(bv))
        assert int(got.cpu().numpy().view(np.uint64)[0]) == digest(ek, ev), (na, nb)
        got = mp.mp_merge_checksum(to_dev(a), to_dev(b))
        assert int(got.cpu().numpy().view(np.uint64)[0]) == digest(ek, None), (na, nb)
    assert mp.mp_kernel_error(reset=True) == 0


def test_checksum_sees_order():
    """Swapping two outputs changes the digest (it is order-sensitive)."""
    k = np.arange(10, dtype=np.uint64)
    k2 = k.copy()
    k2[[3, 4]] = k2[[4, 3]]
    assert digest(k, None) != digest(k2, None)
