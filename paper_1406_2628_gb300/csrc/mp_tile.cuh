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

namespace mp {

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

// Store this thread's VT packed source indices at sidx[tid*VT ...].
template <int VT>
__device__ __forceinline__ void put_indices(uint16_t* sidx, const uint32_t (&packed)[VT / 2])
{
    const int tid = threadIdx.x;
    if constexpr (VT % 8 == 0) {
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
template <class K, bool VALS, int NT, int VT>
__device__ __forceinline__ void store_tile(const TileView<K, VALS, NT, VT>& v, K* gout,
                                           uint32_t* gvout)
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
        for (int j = 0; j < VT / EK; ++j) {
            const int g = tid + j * NT;
            if (g < nvec) {
                K w[EK];
#pragma unroll
                for (int e = 0; e < EK; ++e) {
                    const int s = sidx[g * EK + e];
                    w[e] = s < la ? sA[s] : sB[s - la];
                }
                st_global_cs_v4(gout + g * EK, *reinterpret_cast<uint4*>(w));
            }
        }
        for (int j = nvec * EK + tid; j < L; j += NT) {
            const int s = sidx[j];
            gout[j] = s < la ? sA[s] : sB[s - la];
        }
    } else {
        for (int j = tid; j < L; j += NT) {
            const int s = sidx[j];
            gout[j] = s < la ? sA[s] : sB[s - la];
        }
    }
    if constexpr (VALS) {
        const uint32_t* vA = v.vA;
        const uint32_t* vB = v.vB;
        if ((((uintptr_t)gvout) & 15) == 0) {
            const int nvec = L / 4;
#pragma unroll
            for (int j = 0; j < VT / 4; ++j) {
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

}  // namespace mp
