// mp_sort.cuh -- the block sort of one tile (first stage of the merge sort).
//
// Sec. I / Sec. III: each core first sorts its share on its own, then rounds
// of merges follow.  Here one CTA sorts one tile of T = NT * VT keys:
//   1. coalesced load into shared memory (keys encoded to unsigned order);
//   2. each thread sorts its VT keys in registers with Batcher's odd-even
//      merge network (stable: when values move, keys are compared together
//      with their source positions, which are distinct);
//   3. log2(NT) rounds of Merge Path inside shared memory: runs of width w
//      merge pairwise, each thread producing VT outputs of its pair after a
//      diagonal search (Alg. 2) in that pair;
//   4. coalesced store (keys decoded, or left encoded for the merge passes
//      that follow; values gathered by source position).
// With 4-byte keys alone each run pair is laid out bitonically: A ascending, then B
// descending, so that a walk that runs past the end of A reads B's largest
// key and one past the end of B reads A's largest.  Those act as sentinels:
// the serial merge needs no end tests, and where a sentinel ties the other
// side's head the key taken has the same value, which is all a keys-only
// sort can observe.
// With VT even, shared arrays are padded by one element per 128 bytes, so
// the thread-major accesses (thread t touching elements t*VT .. t*VT+VT-1)
// and the strided reads of the merge rounds spread over the banks; with VT
// odd the thread-major stride itself does, and the arrays are not padded.
#pragma once

#include "mp_device.cuh"
#include "mp_bulk.cuh"

namespace mp {

// Padded position of element i of a shared array of E-byte elements.
// log2 of the elements of size E in 128 bytes (E of 2, 4, 8 or 16 bytes).
template <class E>
constexpr int per128_log2()
{
    return sizeof(E) == 16 ? 3 : (sizeof(E) == 8 ? 4 : (sizeof(E) == 4 ? 5 : 6));
}

template <class E, bool PAD = true>
__device__ __forceinline__ int padded(int i)
{
    if constexpr (PAD)
        return i + (i >> per128_log2<E>());
    else
        return i;
}

template <class K, bool VALS, int NT, int VT>
struct SortSmem {
    static constexpr int T = NT * VT;
    static constexpr bool PAD = VT % 2 == 0;
    static constexpr int KEYS = T + (PAD ? (T >> per128_log2<K>()) : 0) + 1;
    static constexpr int TAGS = VALS ? T + (PAD ? T / 64 : 0) + 2 : 0;
    static constexpr size_t keys_bytes = ((size_t)KEYS * sizeof(K) + 15) / 16 * 16;
    static constexpr size_t tags_bytes = ((size_t)TAGS * 2 + 15) / 16 * 16;
    static constexpr size_t vals_bytes = VALS ? (size_t)T * 4 : 0;
    static constexpr size_t bytes = keys_bytes + tags_bytes + vals_bytes + 16;  // + mbarrier
};

// Compare-exchange of register slots a < b: order by key, then (with
// values) by source position, so the network is stable.
template <class K, bool VALS, int VT>
__device__ __forceinline__ void cmp_swap(K (&k)[VT], uint16_t (&g)[VT], int a, int b)
{
    const bool swap = VALS ? (k[a] > k[b] || (k[a] == k[b] && g[a] > g[b])) : (k[a] > k[b]);
    if (swap) {
        const K tk = k[a]; k[a] = k[b]; k[b] = tk;
        if constexpr (VALS) {
            const uint16_t tg = g[a]; g[a] = g[b]; g[b] = tg;
        }
    }
}

// Batcher's odd-even merge sort network on n elements, as a compile-time
// list of comparator pairs (a < b).  For n not a power of two it is the
// network of the next power of two with the comparators that reach past n
// left out (as if the missing inputs were +infinity).
constexpr int batcher_count(int n)
{
    int c = 0;
    for (int p = 1; p < n; p <<= 1)
        for (int s = p; s >= 1; s >>= 1)
            for (int j = s % p; j + s < n; j += 2 * s)
                for (int i = 0; i < s; ++i)
                    if (i + j + s < n && (i + j) / (2 * p) == (i + j + s) / (2 * p)) ++c;
    return c;
}

template <int VT>
struct BatcherNet {
    static constexpr int N = batcher_count(VT);
    int a[N > 0 ? N : 1];
    int b[N > 0 ? N : 1];
    constexpr BatcherNet() : a(), b()
    {
        int c = 0;
        for (int p = 1; p < VT; p <<= 1)
            for (int s = p; s >= 1; s >>= 1)
                for (int j = s % p; j + s < VT; j += 2 * s)
                    for (int i = 0; i < s; ++i)
                        if (i + j + s < VT && (i + j) / (2 * p) == (i + j + s) / (2 * p)) {
                            a[c] = i + j;
                            b[c] = i + j + s;
                            ++c;
                        }
    }
};

template <class K, bool VALS, int VT>
__device__ __forceinline__ void register_sort(K (&k)[VT], uint16_t (&g)[VT])
{
    constexpr BatcherNet<VT> net;
#pragma unroll
    for (int c = 0; c < BatcherNet<VT>::N; ++c) cmp_swap<K, VALS, VT>(k, g, net.a[c], net.b[c]);
}

// Keys-only merge round in the bitonic layout.  Thread tid's VT sorted keys
// belong to run tid >> r (runs of w = VT << r); threads of odd runs (the B
// side of their pair) store their block mirrored, so B reads descending.
template <class K, bool PAD, int VT>
__device__ __forceinline__ void bitonic_round_store(K* sk, int tid, int r, const K (&keys)[VT])
{
    const int w = VT << r;
    const bool is_b = (tid >> r) & 1;
    const int gs = ((tid >> (r + 1)) << (r + 1)) * VT;
    const int s = is_b ? gs + 2 * w - ((tid & ((1 << r) - 1)) + 1) * VT : tid * VT;
#pragma unroll
    for (int i = 0; i < VT; ++i) sk[padded<K, PAD>(s + i)] = is_b ? keys[VT - 1 - i] : keys[i];
}

// Diagonal search (Alg. 2) and serial merge of VT outputs in a bitonic run
// pair at gs: A[i] at gs + i, B[j] at gs + 2w - 1 - j.
template <class K, bool PAD, int VT>
__device__ __forceinline__ void bitonic_round_merge(const K* sk, int gs, int w, int diag, K (&keys)[VT])
{
    int lo = diag - w > 0 ? diag - w : 0;
    int hi = diag < w ? diag : w;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        // A[mid] against B[diag - 1 - mid]
        if (sk[padded<K, PAD>(gs + mid)] > sk[padded<K, PAD>(gs + 2 * w - diag + mid)])
            hi = mid;
        else
            lo = mid + 1;
    }
    int pa = gs + lo, pb = gs + 2 * w - 1 - (diag - lo);
    K ka = sk[padded<K, PAD>(pa)], kb = sk[padded<K, PAD>(pb)];
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        const bool take_a = !(ka > kb);  // ties take A
        keys[i] = take_a ? ka : kb;
        pa += take_a ? 1 : 0;
        pb -= take_a ? 0 : 1;
        const K nv = sk[padded<K, PAD>(take_a ? pa : pb)];
        ka = take_a ? nv : ka;
        kb = take_a ? kb : nv;
    }
}

// Sorts tile `tile` of in[0..n) into out (out may equal in: a CTA reads its
// whole tile before writing).  ENC_OUT leaves the keys encoded (unsigned
// order) for merge passes that compare them as they are.  TMA_LOAD (keys
// alone, unpadded layout): the tile arrives by one bulk copy on an mbarrier
// (bounded wait; on a timeout flag 1 of *err is set and the tile is left
// unwritten) instead of a loop of scalar loads, which with two CTAs per SM
// kept too few bytes in flight to reach the HBM rate.
template <class K, bool VALS, int NT, int VT, bool ENC_OUT = false, bool TMA_LOAD = false>
__device__ __forceinline__ void block_sort_body(const K* in, const uint32_t* vin, K* out,
                                                uint32_t* vout, int64_t n, Codec<K> c, int64_t tile,
                                                unsigned char* smem, unsigned int* err = nullptr)
{
    static_assert((NT & (NT - 1)) == 0, "NT must be a power of two");
    using SM = SortSmem<K, VALS, NT, VT>;
    constexpr bool PAD = SM::PAD;
    constexpr int T = SM::T;
    K* sk = reinterpret_cast<K*>(smem);
    uint16_t* stag = reinterpret_cast<uint16_t*>(smem + SM::keys_bytes);
    uint32_t* sv = reinterpret_cast<uint32_t*>(smem + SM::keys_bytes + SM::tags_bytes);

    const int tid = threadIdx.x;
    const int64_t base = tile * T;
    const int L = (int)(n - base < T ? n - base : T);
    const K pad = ~K(0);  // encoded maximum: sorts after every real key

    K keys[VT];
    uint16_t tags[VT];
    bool loaded = false;
    if constexpr (TMA_LOAD && !VALS && !PAD) {
        const K* src = in + base;
        if (((uintptr_t)src & 15) == 0) {  // the same for every thread of the CTA
            // 1. The tile's 16-byte-aligned body by one bulk copy, its
            //    ragged end (< 16 bytes) by threads; read back and encoded
            //    per thread, positions past the end taking the padding key.
            constexpr int EK = 16 / sizeof(K);
            constexpr uint32_t WAIT_LIMIT = 1u << 22;
            uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::bytes - 16);
            const int nmain = (L / EK) * EK;
            bulk_init(bar);
            __syncthreads();
            if (tid == 0) {
                mbar_arrive_expect_tx(bar, (uint32_t)(nmain * sizeof(K)));
                if (nmain) bulk_g2s(sk, src, (uint32_t)(nmain * sizeof(K)), bar);
            }
            if (tid < L - nmain) sk[nmain + tid] = src[nmain + tid];
            // err[1] is the staging-wait fault switch (see bulk_stage).
            const uint32_t first_limit = __ldcg(err + 1) ? 0u : WAIT_LIMIT;
            const bool ok = __syncthreads_and(mbar_wait_bounded(bar, 0, first_limit));
            if (!ok) {
                if (tid == 0) atomicOr(err, MP_KERR_MBAR_TIMEOUT);
                mbar_wait_bounded(bar, 0, WAIT_LIMIT);  // let copies in flight land
                return;
            }
#pragma unroll
            for (int i = 0; i < VT; ++i) {
                const int j = tid * VT + i;
                keys[i] = j < L ? key_enc(sk[j], c) : pad;
                tags[i] = (uint16_t)j;
            }
            loaded = true;
        }
    }
    if (!loaded) {
        // 1. Coalesced load; positions past the end hold the padding key.
#pragma unroll 4
        for (int j = tid; j < T; j += NT) {
            sk[padded<K, PAD>(j)] = j < L ? key_enc(in[base + j], c) : pad;
            if constexpr (VALS) {
                if (j < L) sv[j] = vin[base + j];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < VT; ++i) {
            keys[i] = sk[padded<K, PAD>(tid * VT + i)];
            tags[i] = (uint16_t)(tid * VT + i);
        }
    }

    // 2. Thread-local sort of VT keys.
    register_sort<K, VALS, VT>(keys, tags);

    // 3. Merge rounds: runs of width w = VT * 2^r merge pairwise; the pair
    //    of thread tid starts at run 2 * (tid >> (r + 1)).  While a pair's
    //    2^(r+1) threads lie inside one warp (r < 5) its data is the warp's
    //    own, and a warp barrier orders the writes and reads.
    if constexpr (!VALS && sizeof(K) == 4) {
        // Merge rounds on the bitonic layout (the pair of thread tid starts
        // at run 2 * (tid >> (r + 1)); warp barriers while it lies in one warp).
        for (int r = 0; (VT << r) < T; ++r) {
            const bool in_warp = (2 << r) <= 32;
            if (in_warp)
                __syncwarp();
            else
                __syncthreads();
            bitonic_round_store<K, PAD, VT>(sk, tid, r, keys);
            if (in_warp)
                __syncwarp();
            else
                __syncthreads();
            const int gs = ((tid >> (r + 1)) << (r + 1)) * VT;
            bitonic_round_merge<K, PAD, VT>(sk, gs, VT << r, tid * VT - gs, keys);
        }
    } else {
        for (int r = 0; (VT << r) < T; ++r) {
            const int w = VT << r;
            const bool in_warp = (2 << r) <= 32;
            if (in_warp)
                __syncwarp();
            else
                __syncthreads();
#pragma unroll
            for (int i = 0; i < VT; ++i) {
                sk[padded<K, PAD>(tid * VT + i)] = keys[i];
                if constexpr (VALS) stag[padded<uint16_t, PAD>(tid * VT + i)] = tags[i];
            }
            if (in_warp)
                __syncwarp();
            else
                __syncthreads();
            const int gs = ((tid >> (r + 1)) << (r + 1)) * VT;  // start of this thread's run pair
            const int diag = tid * VT - gs;
            // Diagonal search (Alg. 2) in the pair A = [gs, gs+w), B = [gs+w, gs+2w).
            int lo = diag - w > 0 ? diag - w : 0;
            int hi = diag < w ? diag : w;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sk[padded<K, PAD>(gs + mid)] > sk[padded<K, PAD>(gs + w + diag - 1 - mid)])
                    hi = mid;
                else
                    lo = mid + 1;
            }
            if constexpr (VALS) {
                // Serial merge of VT outputs (ties take A), on absolute positions:
                // A is [gs, gs + w), B is [gs + w, gs + 2w).  Each step reads the
                // next element of the side it took, at most one past that side's
                // end (B's start, the next pair's first element or the slack
                // element at T), never used because the end tests come first;
                // the tag follows the element taken.
                int ai = gs + lo, bi = gs + w + diag - lo;
                const int aend = gs + w, bend = gs + 2 * w;
                K ka = sk[padded<K, PAD>(ai)];
                K kb = sk[padded<K, PAD>(bi)];
#pragma unroll
                for (int i = 0; i < VT; ++i) {
                    const bool take_a = (bi >= bend) || (ai < aend && !(ka > kb));
                    const int src = take_a ? ai : bi;
                    keys[i] = take_a ? ka : kb;
                    tags[i] = stag[padded<uint16_t, PAD>(src)];
                    const int nxt = src + 1;
                    const K kn = sk[padded<K, PAD>(nxt)];
                    if (take_a) {
                        ai = nxt;
                        ka = kn;
                    } else {
                        bi = nxt;
                        kb = kn;
                    }
                }
            } else {
                // Wider keys alone: the same merge with the reads clamped
                // into each run (for 8- and 16-byte keys this measured faster
                // than the bitonic layout, whose mirrored stores and selects
                // cost more on wide keys: 2^27 int64 keys 7.08 against 7.47
                // ms, 2^25 128-bit keys 3.45 against 3.58 ms).
                int ai = lo, bi = diag - lo;
                K ka = sk[padded<K, PAD>(gs + (ai < w ? ai : w - 1))];
                K kb = sk[padded<K, PAD>(gs + w + (bi < w ? bi : w - 1))];
#pragma unroll
                for (int i = 0; i < VT; ++i) {
                    const bool take_a = (bi >= w) || (ai < w && !(ka > kb));
                    keys[i] = take_a ? ka : kb;
                    if (take_a) {
                        ++ai;
                        ka = sk[padded<K, PAD>(gs + (ai < w ? ai : w - 1))];
                    } else {
                        ++bi;
                        kb = sk[padded<K, PAD>(gs + w + (bi < w ? bi : w - 1))];
                    }
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        sk[padded<K, PAD>(tid * VT + i)] = keys[i];
        if constexpr (VALS) stag[padded<uint16_t, PAD>(tid * VT + i)] = tags[i];
    }
    __syncthreads();
    // 4. Coalesced store.
#pragma unroll 4
    for (int j = tid; j < L; j += NT) {
        out[base + j] = ENC_OUT ? sk[padded<K, PAD>(j)] : key_dec(sk[padded<K, PAD>(j)], c);
        if constexpr (VALS) vout[base + j] = sv[stag[padded<uint16_t, PAD>(j)]];
    }
}

}  // namespace mp
