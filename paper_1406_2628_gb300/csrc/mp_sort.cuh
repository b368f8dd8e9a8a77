// mp_sort.cuh -- the block sort of one tile (first stage of the merge sort).
#pragma once

#include "mp_device.cuh"

namespace mp {

template <class K, bool VALS, int NT, int VT>
struct SortSmem {
    static constexpr int T = NT * VT;
    static constexpr size_t keys_bytes = ((size_t)T * sizeof(K) + 15) / 16 * 16;
    static constexpr size_t tags_bytes = ((size_t)T * 2 + 15) / 16 * 16;
    static constexpr size_t vals_bytes = VALS ? (size_t)T * 4 : 0;
    static constexpr size_t bytes = keys_bytes + tags_bytes + vals_bytes;
};

// Sorts tile `tile` of in[0..n) into out (out may equal in: a CTA reads
// its whole tile before writing).  Keys are encoded once on load, compared
// as unsigned, and decoded on store; tags (tile-local source positions) ride
// along so values can be gathered at the end.
template <class K, bool VALS, int NT, int VT>
__device__ __forceinline__ void block_sort_body(const K* in, const uint32_t* vin, K* out,
                                                uint32_t* vout, int64_t n, Codec<K> c, int64_t tile,
                                                unsigned char* smem)
{
    using SM = SortSmem<K, VALS, NT, VT>;
    constexpr int T = SM::T;
    K* sk = reinterpret_cast<K*>(smem);
    uint16_t* stag = reinterpret_cast<uint16_t*>(smem + SM::keys_bytes);
    uint32_t* sv = reinterpret_cast<uint32_t*>(smem + SM::keys_bytes + SM::tags_bytes);

    const int tid = threadIdx.x;
    const int64_t base = tile * T;
    const int L = (int)(n - base < T ? n - base : T);
    const K pad = ~K(0);  // encoded maximum: sorts after every real key

    // Coalesced load; positions past the end hold the padding key.
#pragma unroll 4
    for (int j = tid; j < T; j += NT) {
        sk[j] = j < L ? key_enc(in[base + j], c) : pad;
        if constexpr (VALS) {
            if (j < L) sv[j] = vin[base + j];
        }
    }
    __syncthreads();

    K keys[VT];
    uint16_t tags[VT];
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        keys[i] = sk[tid * VT + i];
        tags[i] = (uint16_t)(tid * VT + i);
    }
    // Odd-even transposition sort of VT keys; swapping only strictly greater
    // neighbours keeps equal keys in order (stable).
#pragma unroll
    for (int r = 0; r < VT; ++r) {
#pragma unroll
        for (int i = r & 1; i + 1 < VT; i += 2) {
            if (keys[i] > keys[i + 1]) {
                K tk = keys[i]; keys[i] = keys[i + 1]; keys[i + 1] = tk;
                uint16_t tt = tags[i]; tags[i] = tags[i + 1]; tags[i + 1] = tt;
            }
        }
    }
    // Merge rounds: runs of width w merge pairwise, each thread producing VT
    // outputs of its pair at diagonal (tid*VT mod 2w).
    for (int w = VT; w < T; w *= 2) {
        __syncthreads();
#pragma unroll
        for (int i = 0; i < VT; ++i) {
            sk[tid * VT + i] = keys[i];
            stag[tid * VT + i] = tags[i];
        }
        __syncthreads();
        const int gs = (tid * VT) & ~(2 * w - 1);
        const int diag = tid * VT - gs;
        const K* sA = sk + gs;
        const K* sB = sk + gs + w;
        const int ai = smem_diagonal_search_enc(sA, w, sB, w, diag);
        serial_merge_regs<K, VT>(sA, stag + gs, w, sB, stag + gs + w, w, ai, diag - ai, keys, tags);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        sk[tid * VT + i] = keys[i];
        stag[tid * VT + i] = tags[i];
    }
    __syncthreads();
#pragma unroll 4
    for (int j = tid; j < L; j += NT) {
        out[base + j] = key_dec(sk[j], c);
        if constexpr (VALS) vout[base + j] = sv[stag[j]];
    }
}

}  // namespace mp
