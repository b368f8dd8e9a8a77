// mp_tile.cuh -- the pieces of a Merge Path tile shared by the merge kernels.
//
// One CTA owns one tile of T = NT * VT consecutive outputs (one Merge Path
// segment, Cor. 6).  stage_tile() copies the tile's A and B windows into
// shared memory (Lemma 16); each thread then finds its own split inside the
// window (Thm 17), merges VT outputs serially and records, per output, the
// index of its source in the logical window [A | B]; store_tile() gathers
// keys and values by those indices and writes the tile with coalesced
// 128-bit stores.
#pragma once

#include "mp_device.cuh"
#include "mp_internal.h"

namespace mp {

template <class K>
struct TileArgs {
    const K* a;
    const K* b;
    const uint32_t* av;
    const uint32_t* bv;
    K* out;
    uint32_t* outv;
    int64_t na, nb, run;
    int64_t total;
    const int64_t* a_split;
    Codec<K> codec;
};

// Kernel arguments of a merge problem (host side).
template <class K>
inline TileArgs<K> make_tile_args(const MergeProblem& p, const int64_t* a_split)
{
    TileArgs<K> t;
    t.a = static_cast<const K*>(p.a);
    t.b = static_cast<const K*>(p.b);
    t.av = p.av;
    t.bv = p.bv;
    t.out = static_cast<K*>(p.out);
    t.outv = p.outv;
    t.na = p.na;
    t.nb = p.nb;
    t.run = p.run;
    t.total = p.total();
    t.a_split = a_split;
    t.codec = make_codec<K>(p.kind.flip, p.kind.fmask, p.kind.inv);
    return t;
}

// The merge pair that output index d belongs to (run == 0: the only pair).
template <class K>
struct Pair {
    const K* A;
    const K* B;
    const uint32_t* AV;
    const uint32_t* BV;
    int64_t na, nb, base;
};

template <class K>
__device__ __forceinline__ Pair<K> pair_at(const TileArgs<K>& p, int64_t d)
{
    Pair<K> q;
    if (p.run == 0) {
        q.A = p.a; q.B = p.b; q.AV = p.av; q.BV = p.bv;
        q.na = p.na; q.nb = p.nb; q.base = 0;
    } else {
        const int64_t w2 = 2 * p.run;
        const int64_t base = (d / w2) * w2;
        const int64_t rest = p.na - base;
        q.na = rest < p.run ? rest : p.run;
        const int64_t rest_b = rest - q.na;
        q.nb = rest_b < p.run ? rest_b : p.run;
        q.A = p.a + base;
        q.B = p.a + base + q.na;
        q.AV = p.av ? p.av + base : nullptr;
        q.BV = p.av ? p.av + base + q.na : nullptr;
        q.base = base;
    }
    return q;
}

// Split point (Alg. 2) of output index d, clamped to [0, total], relative to
// the merge pair holding d.
template <class K>
__device__ __forceinline__ int64_t partition_point(const TileArgs<K>& p, int64_t d)
{
    d = d < p.total ? d : p.total;
    const Pair<K> q = pair_at(p, d < p.total ? d : p.total - 1);
    const K* A = q.A;
    const K* B = q.B;
    const Codec<K> c = p.codec;
    return diagonal_search<K>([&](int64_t i) { return key_enc(ld_global_nc(A + i), c); }, q.na,
                              [&](int64_t i) { return key_enc(ld_global_nc(B + i), c); }, q.nb,
                              d - q.base);
}

// Shared memory of a tile: keys [T + 3*EK] (room for the two windows at
// their 16-byte phases), values [T + 12] (if VALS), source indices [T] u16.
template <class K, bool VALS, int NT, int VT>
struct TileSmem {
    static constexpr int T = NT * VT;
    static constexpr int EK = 16 / sizeof(K);
    static constexpr int KEYS = T + 3 * EK;
    static constexpr int VALS_N = VALS ? T + 12 : 0;
    static constexpr size_t keys_bytes = ((size_t)KEYS * sizeof(K) + 15) / 16 * 16;
    static constexpr size_t vals_bytes = ((size_t)VALS_N * 4 + 15) / 16 * 16;
    static constexpr size_t idx_bytes = (size_t)T * 2;
    static constexpr size_t bytes = keys_bytes + vals_bytes + idx_bytes;
};

template <class K, bool VALS, int NT, int VT>
struct TileView {
    K* sA;
    K* sB;
    uint32_t* vA;
    uint32_t* vB;
    uint16_t* sidx;
    int la, lb;
};

// Copy A window gA[0..la) and B window gB[0..lb) (and their values) into
// shared memory; returns where they landed.  Ends with __syncthreads().
template <class K, bool VALS, int NT, int VT>
__device__ __forceinline__ TileView<K, VALS, NT, VT> stage_tile(unsigned char* smem, const K* gA,
                                                                 int la, const K* gB, int lb,
                                                                 const uint32_t* gvA,
                                                                 const uint32_t* gvB)
{
    using SM = TileSmem<K, VALS, NT, VT>;
    constexpr int T = SM::T;
    constexpr int EK = SM::EK;
    constexpr int RK = (T / EK + 2 + NT - 1) / NT;
    constexpr int RV = (T / 4 + 2 + NT - 1) / NT;
    TileView<K, VALS, NT, VT> v;
    K* sk = reinterpret_cast<K*>(smem);
    uint32_t* sv = reinterpret_cast<uint32_t*>(smem + SM::keys_bytes);
    v.sidx = reinterpret_cast<uint16_t*>(smem + SM::keys_bytes + SM::vals_bytes);
    v.la = la;
    v.lb = lb;
    // Windows keep the 16-byte phase of their global sources.
    v.sA = sk + phase16(gA);
    v.sB = sk + ((phase16(gA) + la + EK - 1) / EK) * EK + phase16(gB);
    WindowStager<K, NT, RK> kst;
    kst.load(gA, la, gB, lb);
    if constexpr (VALS) {
        v.vA = sv + phase16(gvA);
        v.vB = sv + ((phase16(gvA) + la + 3) / 4) * 4 + phase16(gvB);
        WindowStager<uint32_t, NT, RV> vst;
        vst.load(gvA, la, gvB, lb);
        kst.store(v.sA, v.sB);
        vst.store(v.vA, v.vB);
    } else {
        v.vA = v.vB = nullptr;
        kst.store(v.sA, v.sB);
    }
    __syncthreads();
    return v;
}

// Store this thread's VT packed source indices at sidx[tid*VT ...]: vector
// stores when VT is a multiple of 4, else one 16-bit store per output.
template <int VT>
__device__ __forceinline__ void put_indices(uint16_t* sidx, const uint32_t (&packed)[(VT + 1) / 2])
{
    const int tid = threadIdx.x;
    if constexpr (VT % 4 != 0) {
#pragma unroll
        for (int i = 0; i < VT; ++i) sidx[tid * VT + i] = (uint16_t)(packed[i / 2] >> (16 * (i & 1)));
    } else if constexpr (VT % 8 == 0) {
#pragma unroll
        for (int i = 0; i < VT / 8; ++i)
            reinterpret_cast<uint4*>(sidx + tid * VT)[i] =
                make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < VT / 4; ++i)
            reinterpret_cast<uint2*>(sidx + tid * VT)[i] = make_uint2(packed[2 * i], packed[2 * i + 1]);
    }
}

// Gather by source index and write the tile's L outputs to gout (and gvout).
// Call after a __syncthreads() that follows every put_indices().
// Encoded-input codec kinds (CK) decode each key on the way out.
template <class K, bool VALS, int NT, int VT, int CK = CODEC_IDENTITY>
__device__ __forceinline__ void store_tile(const TileView<K, VALS, NT, VT>& v, K* gout,
                                           uint32_t* gvout, Codec<K> c = Codec<K>{})
{
    constexpr int EK = 16 / sizeof(K);
    const int tid = threadIdx.x;
    const int la = v.la;
    const int L = v.la + v.lb;
    const uint16_t* sidx = v.sidx;
    const K* sA = v.sA;
    const K* sB = v.sB;
    if ((((uintptr_t)gout) & 15) == 0) {
        const int nvec = L / EK;
#pragma unroll
        for (int j = 0; j < (VT + EK - 1) / EK; ++j) {
            const int g = tid + j * NT;
            if (g < nvec) {
                K w[EK];
#pragma unroll
                for (int e = 0; e < EK; ++e) {
                    const int s = sidx[g * EK + e];
                    w[e] = key_out_ck<CK>(s < la ? sA[s] : sB[s - la], c);
                }
                st_global_cs_v4(gout + g * EK, *reinterpret_cast<uint4*>(w));
            }
        }
        for (int j = nvec * EK + tid; j < L; j += NT) {
            const int s = sidx[j];
            gout[j] = key_out_ck<CK>(s < la ? sA[s] : sB[s - la], c);
        }
    } else {
        for (int j = tid; j < L; j += NT) {
            const int s = sidx[j];
            gout[j] = key_out_ck<CK>(s < la ? sA[s] : sB[s - la], c);
        }
    }
    if constexpr (VALS) {
        const uint32_t* vA = v.vA;
        const uint32_t* vB = v.vB;
        if ((((uintptr_t)gvout) & 15) == 0) {
            const int nvec = L / 4;
#pragma unroll
            for (int j = 0; j < (VT + 3) / 4; ++j) {
                const int g = tid + j * NT;
                if (g < nvec) {
                    const uint2 pk = *reinterpret_cast<const uint2*>(sidx + g * 4);
                    const int s0 = pk.x & 0xFFFF, s1 = pk.x >> 16, s2 = pk.y & 0xFFFF, s3 = pk.y >> 16;
                    uint4 w;
                    w.x = s0 < la ? vA[s0] : vB[s0 - la];
                    w.y = s1 < la ? vA[s1] : vB[s1 - la];
                    w.z = s2 < la ? vA[s2] : vB[s2 - la];
                    w.w = s3 < la ? vA[s3] : vB[s3 - la];
                    st_global_cs_v4(gvout + g * 4, w);
                }
            }
            for (int j = nvec * 4 + tid; j < L; j += NT) {
                const int s = sidx[j];
                gvout[j] = s < la ? vA[s] : vB[s - la];
            }
        } else {
            for (int j = tid; j < L; j += NT) {
                const int s = sidx[j];
                gvout[j] = s < la ? vA[s] : vB[s - la];
            }
        }
    }
}

// Write the tile's L outputs, held in order at so[0..L), to gout: 128-bit
// shared loads and streaming stores when gout is 16-byte aligned.  so must
// be 16-byte aligned.  Call after a __syncthreads() that follows the last
// write of so.
template <class K, int NT, int VT>
__device__ __forceinline__ void store_linear(const K* so, int L, K* gout)
{
    constexpr int EK = 16 / sizeof(K);
    const int tid = threadIdx.x;
    if ((((uintptr_t)gout) & 15) == 0) {
        const int nvec = L / EK;
#pragma unroll
        for (int j = 0; j < (VT + EK - 1) / EK; ++j) {
            const int g = tid + j * NT;
            if (g < nvec) st_global_cs_v4(gout + g * EK, *reinterpret_cast<const uint4*>(so + g * EK));
        }
        for (int j = nvec * EK + tid; j < L; j += NT) gout[j] = so[j];
    } else {
        for (int j = tid; j < L; j += NT) gout[j] = so[j];
    }
}

// One tile of a merge problem (plain merge or sort pass): stage, split,
// merge, store.  a_split holds the problem's split points at multiples of T.
template <class K, bool VALS, int NT, int VT, int CK = CODEC_RUNTIME>
__device__ __forceinline__ void merge_tile_body(const TileArgs<K>& p, int64_t tile,
                                                const int64_t* a_split, unsigned char* smem)
{
    static_assert(VT % 4 == 0, "VT must be a multiple of 4");
    constexpr int T = NT * VT;
    const int tid = threadIdx.x;
    const int64_t d0 = tile * T;
    const int64_t d1 = d0 + T < p.total ? d0 + T : p.total;
    const Pair<K> q = pair_at(p, d0);
    const int64_t d0l = d0 - q.base, d1l = d1 - q.base;

    // Split points are clamped into the grid and made monotone, so that
    // unsorted inputs or foreign split arrays give wrong output rather than
    // out-of-range accesses; for valid inputs the clamps change nothing.
    const int64_t a0 = clamp_split(a_split[tile], d0l, q.na, q.nb);
    const int64_t a1 = (d1l == q.na + q.nb) ? q.na : clamp_end_split(a_split[tile + 1], a0, d0l, d1l, q.na, q.nb);
    const int64_t b0 = d0l - a0, b1 = d1l - a1;
    const int la = (int)(a1 - a0), lb = (int)(b1 - b0);
    const int L = la + lb;

    const auto v = stage_tile<K, VALS, NT, VT>(smem, q.A + a0, la, q.B + b0, lb,
                                               VALS ? q.AV + a0 : nullptr,
                                               VALS ? q.BV + b0 : nullptr);
    // Per-thread split inside the window (Thm 17), then VT serial steps.
    {
        const int diag = tid * VT < L ? tid * VT : L;
        const int ai = smem_diagonal_search_ck<CK>(v.sA, la, v.sB, lb, diag, p.codec);
        uint32_t packed[(VT + 1) / 2];
        serial_merge_indices_ck<K, VT, CK>(v.sA, la, v.sB, lb, ai, diag - ai, p.codec, packed);
        put_indices<VT>(v.sidx, packed);
    }
    __syncthreads();
    store_tile<K, VALS, NT, VT>(v, p.out + d0, VALS ? p.outv + d0 : nullptr);
}

}  // namespace mp
