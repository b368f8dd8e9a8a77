// mp_device.cuh -- device building blocks of the Merge Path kernels.
//
// Merge Path (Green, Odeh, Birk): the merged output of sorted A and B is a
// monotone staircase through the |A| x |B| grid; the path moves right (emits
// B[j]) iff A[i] > B[j] and down (emits A[i]) otherwise (Sec. II.A).  Its
// crossing with cross diagonal d (the point after d outputs) is found by a
// binary search along the diagonal (Alg. 2; Cor. 12 makes the diagonal a
// 1...1 0...0 sequence, Prop. 13 puts the path at its transition), so the
// output splits into equal, independent pieces (Thm 5, Cor. 6, Cor. 7).
//
// Everything here works on keys held as unsigned integers (uint32_t,
// uint64_t or 128-bit bit patterns) and compares them through an
// order-preserving codec, so one kernel body serves signed, unsigned and
// float keys.
#pragma once

#include <cstdint>
#include <cstring>
#include <type_traits>
#include <cuda_runtime.h>

namespace mp {

// 128-bit keys (multi-word: two 64-bit words, low word first in memory).
using u128 = unsigned __int128;

// Signed integer of a key's width (for the sign fill of the codec).
template <class K>
using signed_of = typename std::conditional<
    sizeof(K) == 16, __int128, typename std::conditional<sizeof(K) == 8, int64_t, int32_t>::type>::type;

// ---------------------------------------------------------------------------
// Key codec.  enc(x) = x ^ ((signfill(x) & fmask) | flip), compared as
// unsigned:
//   unsigned ints: flip = 0,        fmask = 0        (identity)
//   signed ints:   flip = top bit,  fmask = 0        (sign bit flipped)
//   float32:       flip = top bit,  fmask = all ones (negatives: all bits
//                  flipped; positives: sign bit set), which orders -0.0
//                  before +0.0 and keeps IEEE numeric order otherwise.
// ---------------------------------------------------------------------------
// Descending order adds inv = all ones: the encoded keys are complemented,
// so ascending comparison of them is descending order of the keys.
template <class K>
struct Codec {
    K flip;
    K fmask;
    K inv;
};

template <class K>
__device__ __forceinline__ K key_enc(K x, Codec<K> c)
{
    using S = signed_of<K>;
    K fill = (K)((S)x >> (8 * sizeof(K) - 1));
    return x ^ ((fill & c.fmask) | c.flip) ^ c.inv;
}

// The codec of a key kind given by its top-word masks: flip and fmask act
// on the key's top 64 bits (for 128-bit keys flip is moved to the top word;
// fmask, used by float keys only, widens to all bits), inv != 0 complements
// every bit.
template <class K>
__host__ __device__ inline Codec<K> make_codec(uint64_t flip, uint64_t fmask, uint64_t inv)
{
    Codec<K> c;
    if constexpr (sizeof(K) == 16) {
        c.flip = (K)flip << 64;
        c.fmask = fmask ? ~(K)0 : (K)0;
        c.inv = inv ? ~(K)0 : (K)0;
    } else {
        c.flip = (K)flip;
        c.fmask = (K)fmask;
        c.inv = (K)inv;
    }
    return c;
}

// Codec kinds known at compile time: identity (unsigned keys: the
// comparison needs no encoding at all), signed integers (the top bit
// flipped), ascending floats (the top bit of positives flipped, every bit of
// negatives) and the runtime flip/fmask/inv codec (descending order).  Each
// fixed kind computes key_enc with its codec's constants folded in.
enum { CODEC_IDENTITY = 0, CODEC_RUNTIME = 1, CODEC_SIGNED = 2, CODEC_FLOAT = 3 };
// The same three codecs for keys that are already encoded (the merge sort
// keeps its intermediate runs encoded): compared as they are, decoded with
// the codec on output.
enum { CODEC_ENCODED_SIGNED = 4, CODEC_ENCODED_FLOAT = 5, CODEC_ENCODED_RUNTIME = 6 };
template <int CK>
constexpr bool codec_encoded_input()
{
    return CK >= CODEC_ENCODED_SIGNED;
}

template <int CK, class K>
__device__ __forceinline__ K key_enc_ck(K x, Codec<K> c)
{
    constexpr K top = (K)1 << (8 * sizeof(K) - 1);
    if constexpr (CK == CODEC_IDENTITY || codec_encoded_input<CK>()) {
        (void)c;
        return x;
    } else if constexpr (CK == CODEC_SIGNED) {
        (void)c;
        return x ^ top;
    } else if constexpr (CK == CODEC_FLOAT) {
        (void)c;
        using S = signed_of<K>;
        return x ^ ((K)((S)x >> (8 * sizeof(K) - 1)) | top);
    } else {
        return key_enc(x, c);
    }
}

// Inverse of key_enc: the sign of the original is the complement of the
// encoded top bit when fmask is set.
template <class K>
__device__ __forceinline__ K key_dec(K e, Codec<K> c)
{
    using S = signed_of<K>;
    e ^= c.inv;
    K fill = (K)((S)(~e) >> (8 * sizeof(K) - 1));
    return e ^ ((fill & c.fmask) | c.flip);
}

// Inverse of key_enc_ck (for encoded-input kinds: the decoding of their
// codec, since those keys arrive encoded).
template <int CK, class K>
__device__ __forceinline__ K key_dec_ck(K e, Codec<K> c)
{
    constexpr K top = (K)1 << (8 * sizeof(K) - 1);
    if constexpr (CK == CODEC_IDENTITY) {
        (void)c;
        return e;
    } else if constexpr (CK == CODEC_SIGNED || CK == CODEC_ENCODED_SIGNED) {
        (void)c;
        return e ^ top;
    } else if constexpr (CK == CODEC_FLOAT || CK == CODEC_ENCODED_FLOAT) {
        (void)c;
        using S = signed_of<K>;
        return e ^ ((K)((S)(~e) >> (8 * sizeof(K) - 1)) | top);
    } else {
        return key_dec(e, c);
    }
}

// A key as it leaves a tile whose outputs are gathered from the staged
// input: unchanged, except for encoded-input kinds, which decode it.
template <int CK, class K>
__device__ __forceinline__ K key_out_ck(K x, Codec<K> c)
{
    if constexpr (codec_encoded_input<CK>())
        return key_dec_ck<CK>(x, c);
    else
        return x;
}

// ---------------------------------------------------------------------------
// 128-bit global and shared memory access.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 ld_global_nc_v4(const void* p)
{
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

__device__ __forceinline__ void st_global_cs_v4(void* p, uint4 v)
{
    asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

template <class E>
__device__ __forceinline__ E ld_global_nc(const E* p)
{
    if constexpr (sizeof(E) == 16) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
        E e;
        memcpy(&e, &v, 16);
        return e;
    } else {
        return __ldg(p);
    }
}

__device__ __forceinline__ void st_shared_v4(void* p, uint4 v)
{
    *reinterpret_cast<uint4*>(p) = v;
}

// Number of leading elements of type E before the first 16-byte boundary at
// or after p (capped at n).
template <class E>
__device__ __forceinline__ int head_to_16(const E* p, int n)
{
    int h = (int)(((16u - ((uint32_t)(uintptr_t)p & 15u)) & 15u) / sizeof(E));
    return h < n ? h : n;
}

// Phase (in elements) of p within its 16-byte granule.
template <class E>
__device__ __forceinline__ int phase16(const E* p)
{
    return (int)(((uint32_t)(uintptr_t)p & 15u) / sizeof(E));
}

// ---------------------------------------------------------------------------
// Stage the two windows of one Merge Path segment into shared memory
// (Lemma 16 / Thm 17: a path segment of length L touches at most L
// consecutive elements of A and at most L of B).
//
// The shared destinations sA and sB must have the same 16-byte phase as the
// global sources gA and gB, so the aligned interior moves with one 128-bit
// load and one 128-bit shared store per vector; the ragged head and tail
// (< 16 bytes each) move as scalars.  load() issues every global load of the
// thread and store() writes them out, so a caller can issue the loads of
// several arrays (keys, values) before the first store and keep many loads
// in flight.  R = vectors per thread, enough for (la + lb) / V + 2.
// ---------------------------------------------------------------------------
template <class E, int NT, int R>
struct WindowStager {
    static constexpr int V = 16 / sizeof(E);
    uint4 r[R];
    E s;
    int hA, nvA, tA, hB, nvB, tB;
    bool have;

    __device__ __forceinline__ void load(const E* __restrict__ gA, int la,
                                         const E* __restrict__ gB, int lb)
    {
        const int tid = threadIdx.x;
        hA = head_to_16(gA, la);
        nvA = (la - hA) / V;
        tA = la - hA - nvA * V;
        hB = head_to_16(gB, lb);
        nvB = (lb - hB) / V;
        tB = lb - hB - nvB * V;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            int i = tid + j * NT;
            if (i < nvA)
                r[j] = ld_global_nc_v4(gA + hA + i * V);
            else if (i - nvA < nvB)
                r[j] = ld_global_nc_v4(gB + hB + (i - nvA) * V);
        }
        // Scalars: threads [0, V) take A's head, [V, 2V) A's tail, [2V, 3V)
        // B's head, [3V, 4V) B's tail.
        const int g = tid / V, l = tid % V;
        s = E(0);
        have = false;
        if (g == 0 && l < hA) { s = ld_global_nc(gA + l); have = true; }
        else if (g == 1 && l < tA) { s = ld_global_nc(gA + hA + nvA * V + l); have = true; }
        else if (g == 2 && l < hB) { s = ld_global_nc(gB + l); have = true; }
        else if (g == 3 && l < tB) { s = ld_global_nc(gB + hB + nvB * V + l); have = true; }
    }

    __device__ __forceinline__ void store(E* sA, E* sB) const
    {
        const int tid = threadIdx.x;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            int i = tid + j * NT;
            if (i < nvA)
                st_shared_v4(sA + hA + i * V, r[j]);
            else if (i - nvA < nvB)
                st_shared_v4(sB + hB + (i - nvA) * V, r[j]);
        }
        if (have) {
            const int g = tid / V, l = tid % V;
            if (g == 0) sA[l] = s;
            else if (g == 1) sA[hA + nvA * V + l] = s;
            else if (g == 2) sB[l] = s;
            else sB[hB + nvB * V + l] = s;
        }
    }
};

// ---------------------------------------------------------------------------
// Diagonal search (Alg. 2, in its one-sided form): the number of A elements
// among the first `diag` outputs of the stable merge of A[0..la) and
// B[0..lb).  It is the smallest a in [max(0, diag-lb), min(diag, la)] with
// a == min(diag, la) or A[a] > B[diag-1-a]; each probe reads one element of
// each array (Thm 14).  KeyAt(i) returns the encoded key.
// ---------------------------------------------------------------------------
template <class K, class FA, class FB>
__device__ __forceinline__ int64_t diagonal_search(FA keyA, int64_t la, FB keyB, int64_t lb,
                                                   int64_t diag)
{
    int64_t lo = diag - lb > 0 ? diag - lb : 0;
    int64_t hi = diag < la ? diag : la;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keyA(mid) > keyB(diag - 1 - mid))
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// Clamp a split point on diagonal d into the grid: [max(0, d-nb), min(d, na)].
__device__ __forceinline__ int64_t clamp_split(int64_t a, int64_t d, int64_t na, int64_t nb)
{
    const int64_t lo = d - nb > 0 ? d - nb : 0;
    const int64_t hi = d < na ? d : na;
    return a < lo ? lo : (a > hi ? hi : a);
}

// A tile's end split from its start split a0 (on diagonal d0, already in
// the grid) and a raw end split a1 on d1: in the grid on d1 and in
// [a0, a0 + (d1 - d0)], so that both windows, A[a0, a1) and
// B[d0 - a0, d1 - a1), stay inside their arrays whatever the split array
// holds (splits of unsorted input, or a caller's foreign ones, need not be
// monotone).  For valid splits nothing changes.
__device__ __forceinline__ int64_t clamp_end_split(int64_t a1, int64_t a0, int64_t d0, int64_t d1, int64_t na,
                                                   int64_t nb)
{
    a1 = clamp_split(a1, d1, na, nb);
    a1 = a1 < a0 ? a0 : a1;
    a1 = a1 > a0 + (d1 - d0) ? a0 + (d1 - d0) : a1;
    const int64_t lo1 = d1 - nb > 0 ? d1 - nb : 0;  // at most a0 + (d1 - d0), as a0 >= d0 - nb
    return a1 < lo1 ? lo1 : a1;
}

// 32-bit version for searches inside shared memory.
template <class K>
__device__ __forceinline__ int smem_diagonal_search(const K* sA, int la, const K* sB, int lb,
                                                    int diag, Codec<K> c)
{
    int lo = diag - lb > 0 ? diag - lb : 0;
    int hi = diag < la ? diag : la;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (key_enc(sA[mid], c) > key_enc(sB[diag - 1 - mid], c))
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// Same search on keys already encoded in shared memory.
template <class K>
__device__ __forceinline__ int smem_diagonal_search_enc(const K* sA, int la, const K* sB, int lb,
                                                        int diag)
{
    int lo = diag - lb > 0 ? diag - lb : 0;
    int hi = diag < la ? diag : la;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (sA[mid] > sB[diag - 1 - mid])
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Serial merge of VT outputs starting at split (ai, bi) (Alg. 1's Merge()):
// take A[ai] unless B is exhausted or A[ai] > B[bi] (ties take A: stable).
// Writes the source of each output as an index into the logical window
// [A | B] (A: 0..la-1, B: la..la+lb-1).  Each step reads the next element
// of the side it took, at most one past that side's end (sA[la], sB[lb]);
// the caller's shared buffers hold that slack, and a value read there is
// never used because the range checks come first.
// ---------------------------------------------------------------------------
template <class K, int VT>
__device__ __forceinline__ void serial_merge_indices(const K* sA, int la, const K* sB, int lb,
                                                     int ai, int bi, Codec<K> c,
                                                     uint32_t (&packed)[(VT + 1) / 2])
{
    K ka = key_enc(sA[ai], c);
    K kb = key_enc(sB[bi], c);
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        bool take_a = (bi >= lb) || (ai < la && !(ka > kb));
        uint32_t src = take_a ? (uint32_t)ai : (uint32_t)(la + bi);
        if (i & 1)
            packed[i / 2] |= src << 16;
        else
            packed[i / 2] = src;
        const K* nxt = take_a ? (sA + (ai < la ? ai + 1 : la)) : (sB + bi + 1);
        K kn = key_enc(*nxt, c);
        if (take_a) { ka = kn; ++ai; }
        else { kb = kn; ++bi; }
    }
}

// Same diagonal search with a compile-time codec kind.
template <int CK, class K>
__device__ __forceinline__ int smem_diagonal_search_ck(const K* sA, int la, const K* sB, int lb,
                                                       int diag, Codec<K> c)
{
    int lo = diag - lb > 0 ? diag - lb : 0;
    int hi = diag < la ? diag : la;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (key_enc_ck<CK>(sA[mid], c) > key_enc_ck<CK>(sB[diag - 1 - mid], c))
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// serial_merge_indices with a compile-time codec kind.
template <class K, int VT, int CK>
__device__ __forceinline__ void serial_merge_indices_ck(const K* sA, int la, const K* sB, int lb,
                                                        int ai, int bi, Codec<K> c,
                                                        uint32_t (&packed)[(VT + 1) / 2])
{
    K ka = key_enc_ck<CK>(sA[ai], c);
    K kb = key_enc_ck<CK>(sB[bi], c);
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        bool take_a = (bi >= lb) || (ai < la && !(ka > kb));
        uint32_t src = take_a ? (uint32_t)ai : (uint32_t)(la + bi);
        if (i & 1)
            packed[i / 2] |= src << 16;
        else
            packed[i / 2] = src;
        const K* nxt = take_a ? (sA + (ai < la ? ai + 1 : la)) : (sB + bi + 1);
        K kn = key_enc_ck<CK>(*nxt, c);
        if (take_a) { ka = kn; ++ai; }
        else { kb = kn; ++bi; }
    }
}

// The serial merge of serial_merge_indices_ck keeping the merged keys
// themselves in registers instead of their sources (decoded back to their
// stored form at the end): for tiles without values, whose outputs are then
// written back to shared memory in thread order and stored linearly.  Same
// reads, same decisions.
template <class K, int VT, int CK>
__device__ __forceinline__ void serial_merge_keys_ck(const K* sA, int la, const K* sB, int lb, int ai,
                                                     int bi, Codec<K> c, K (&out)[VT])
{
    K ka = key_enc_ck<CK>(sA[ai], c);
    K kb = key_enc_ck<CK>(sB[bi], c);
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        const bool take_a = (bi >= lb) || (ai < la && !(ka > kb));
        out[i] = take_a ? ka : kb;
        const K* nxt = take_a ? (sA + (ai < la ? ai + 1 : la)) : (sB + bi + 1);
        const K kn = key_enc_ck<CK>(*nxt, c);
        if (take_a) { ka = kn; ++ai; }
        else { kb = kn; ++bi; }
    }
#pragma unroll
    for (int i = 0; i < VT; ++i) out[i] = key_dec_ck<CK>(out[i], c);
}

// Serial merge on encoded keys carrying a 16-bit tag (block sort rounds).
template <class K, int VT>
__device__ __forceinline__ void serial_merge_regs(const K* sA, const uint16_t* tA, int la,
                                                  const K* sB, const uint16_t* tB, int lb,
                                                  int ai, int bi, K (&keys)[VT],
                                                  uint16_t (&tags)[VT])
{
    K ka = sA[ai < la ? ai : la - 1];
    K kb = sB[bi < lb ? bi : lb - 1];
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        bool take_a = (bi >= lb) || (ai < la && !(ka > kb));
        keys[i] = take_a ? ka : kb;
        tags[i] = take_a ? tA[ai < la ? ai : la - 1] : tB[bi < lb ? bi : lb - 1];
        if (take_a) {
            ++ai;
            ka = sA[ai < la ? ai : la - 1];
        } else {
            ++bi;
            kb = sB[bi < lb ? bi : lb - 1];
        }
    }
}

}  // namespace mp
