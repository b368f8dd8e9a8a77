"""The seeded input generator (gen/) against SplitMix64's published outputs.

gen.splitmix64 is a counter-based use of SplitMix64 (Steele, Lea, Flood,
OOPSLA 2014): element i of stream 0 under seed k is the (i+1)-th output of
the sequential generator started from state k.  Its first outputs from
state 0 and from state 1234567 are the values printed with the reference
implementation, so they pin the constants and the shift amounts here.
The workload recipes are checked for the shapes and structure they state.
"""
import numpy as np

import gen


def test_splitmix64_published_outputs():
    assert [int(v) for v in gen.splitmix64(0, 0, 5)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
        0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
    assert [int(v) for v in gen.splitmix64(1234567, 0, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_counter_offsets_and_streams():
    whole = gen.splitmix64(gen.BASE_SEED, 3, 1000)
    assert np.array_equal(gen.splitmix64(gen.BASE_SEED, 3, 100, start=900), whole[900:])
    other = gen.splitmix64(gen.BASE_SEED, 4, 1000)
    assert not np.array_equal(whole, other)
    assert len(np.intersect1d(whole, other)) == 0


def test_uniform_below_stays_below_its_bound():
    for bound in (1, 7, 1 << 24, 1 << 32, (1 << 40) + 3, 1 << 64):
        x = gen.uniform_below(gen.BASE_SEED, 9, 10_000, bound)
        assert x.dtype == np.uint64
        assert int(x.max()) < bound


def test_workload_shapes():
    a, b = gen.plain_keys(n_a=4096, n_b=3000)
    assert a.dtype == np.int32 and a.size == 4096 and b.size == 3000
    assert np.all(a[1:] >= a[:-1]) and np.all(b[1:] >= b[:-1])
    assert a.min() >= 0 and max(a.max(), b.max()) < (1 << 24)

    ak, av, bk, bv = gen.large_kv("a_gt_b", n_a=1000, n_b=300)
    assert ak.dtype == np.uint64 and av.dtype == np.uint32
    assert ak.min() > bk.max()  # every A key above every B key
    assert np.array_equal(av, np.arange(1000, dtype=np.uint32))
    assert np.array_equal(bv, np.arange(1000, 1300, dtype=np.uint32))

    ak, _, bk, _ = gen.large_kv("distinct16", n_a=5000, n_b=2000)
    assert len(np.union1d(ak, bk)) <= 16

    ak, _, bk, _ = gen.large_kv("interleaved", n_a=4000, n_b=1000)
    both = np.concatenate([ak, bk])
    assert len(np.unique(both)) == both.size  # distinct keys, ranks dealt out

    f = gen.sort_input("f32", "random", n=50_000)
    assert f.dtype == np.float32 and not np.isnan(f).any()
    s = gen.sort_input("i32", "reverse", n=10_000)
    assert np.all(s[1:] <= s[:-1])
    d = gen.sort_input("i32", "distinct256", n=10_000)
    assert len(np.unique(d)) <= 256

    a, a_off, b, b_off = gen.batched(n_seg=64, log2_max=8.0)
    assert a_off.dtype == np.int64 and a_off.size == 65 and a_off[-1] == a.size
    assert b_off.size == 65 and b_off[-1] == b.size
    for s_ in range(64):
        seg = a[a_off[s_]:a_off[s_ + 1]]
        assert np.all(seg[1:] >= seg[:-1])
        assert 1 <= seg.size <= 256

    a, b = gen.sets(log2_universe=16)
    assert a.dtype == np.int32 and np.all(np.diff(a) > 0) and np.all(np.diff(b) > 0)
    assert 0 <= a.min() and max(a.max(), b.max()) < (1 << 16)
    # Independent fair bits: each side and the overlap near 1/2 and 1/4 of the universe.
    assert abs(a.size - 32768) < 1000 and abs(b.size - 32768) < 1000
    assert abs(np.intersect1d(a, b).size - 16384) < 800
