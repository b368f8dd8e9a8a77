// mp_bulk.cuh -- merge tiles staged by TMA bulk copies.
//
// Same Merge Path tile as mp_tile.cuh (one CTA-tile = one path segment,
// Cor. 6; windows bounded by Lemma 16; per-thread splits by Thm 17), but the
// windows are moved by the Tensor Memory Accelerator: one thread issues a
// 1D bulk copy (cp.async.bulk) of each window's 16-byte-aligned interior,
// completion is tracked by an mbarrier, and the ragged edges (< 16 bytes per
// side) are loaded by a few threads.  No thread holds staged data in
// registers, so the tile needs fewer registers than the vector-staged one.
#pragma once

#include "mp_tile.cuh"

namespace mp {

// Bit set in the kernel error word when a bounded wait runs out.
#define MP_KERR_MBAR_TIMEOUT 1u

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t tx)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(tx)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the phase with the given parity, at most `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Where one tile's windows live in global and in shared memory.
template <class K>
struct TilePlace {
    const K* gA;
    const K* gB;
    const uint32_t* gvA;
    const uint32_t* gvB;
    int la, lb;
    int64_t d0;  // first output of the tile
};

template <class K>
__device__ __forceinline__ TilePlace<K> tile_place(const TileArgs<K>& p, int64_t tile, int T,
                                                   const int64_t* a_split)
{
    const int64_t d0 = tile * T;
    const int64_t d1 = d0 + T < p.total ? d0 + T : p.total;
    const Pair<K> q = pair_at(p, d0);
    const int64_t d0l = d0 - q.base, d1l = d1 - q.base;
    const int64_t a0 = clamp_split(a_split[tile], d0l, q.na, q.nb);
    const int64_t a1 = (d1l == q.na + q.nb) ? q.na : clamp_end_split(a_split[tile + 1], a0, d0l, d1l, q.na, q.nb);
    const int64_t b0 = d0l - a0, b1 = d1l - a1;
    TilePlace<K> t;
    t.gA = q.A + a0;
    t.gB = q.B + b0;
    t.gvA = q.AV ? q.AV + a0 : nullptr;
    t.gvB = q.BV ? q.BV + b0 : nullptr;
    t.la = (int)(a1 - a0);
    t.lb = (int)(b1 - b0);
    t.d0 = d0;
    return t;
}

// Shared-memory view of a tile placed in a stage (keys at their 16-byte phase).
template <class K, bool VALS, int NT, int VT>
__device__ __forceinline__ TileView<K, VALS, NT, VT> stage_view(const TilePlace<K>& t, K* sk,
                                                                uint32_t* sv, uint16_t* sidx)
{
    constexpr int EK = 16 / sizeof(K);
    TileView<K, VALS, NT, VT> v;
    v.la = t.la;
    v.lb = t.lb;
    v.sidx = sidx;
    v.sA = sk + phase16(t.gA);
    v.sB = sk + ((phase16(t.gA) + t.la + EK - 1) / EK) * EK + phase16(t.gB);
    if constexpr (VALS) {
        v.vA = sv + phase16(t.gvA);
        v.vB = sv + ((phase16(t.gvA) + t.la + 3) / 4) * 4 + phase16(t.gvB);
    } else {
        v.vA = v.vB = nullptr;
    }
    return v;
}

// Issue the bulk copies of a window pair's aligned interiors (one thread).
template <class E>
__device__ __forceinline__ uint32_t interior_bytes(const E* g, int n)
{
    const int h = head_to_16(g, n);
    return (uint32_t)(((n - h) * (int)sizeof(E)) & ~15);
}

template <class E>
__device__ __forceinline__ void issue_interior(E* s, const E* g, int n, uint64_t* bar)
{
    const int h = head_to_16(g, n);
    const uint32_t bytes = (uint32_t)(((n - h) * (int)sizeof(E)) & ~15);
    if (bytes) bulk_g2s(s + h, g + h, bytes, bar);
}

// Edge elements of one window pair (outside the aligned interiors): at most
// V-1 at each end of each window; thread slot j in [0, 4V) owns one.
template <class E>
struct EdgeLoad {
    E val;
    int dst;  // index relative to sA (j < 2V) or sB; -1 if none
    bool in_b;
};

template <class E>
__device__ __forceinline__ EdgeLoad<E> edge_load(int j, const E* gA, int la, const E* gB, int lb)
{
    constexpr int V = 16 / sizeof(E);
    EdgeLoad<E> e;
    e.dst = -1;
    e.in_b = j >= 2 * V;
    e.val = E(0);
    const E* g = e.in_b ? gB : gA;
    const int n = e.in_b ? lb : la;
    const int h = head_to_16(g, n);
    const int tail0 = h + ((n - h) / V) * V;
    const int jj = j % (2 * V);
    int idx = -1;
    if (jj < V) {
        if (jj < h) idx = jj;
    } else if (tail0 + (jj - V) < n) {
        idx = tail0 + (jj - V);
    }
    if (idx >= 0) {
        e.val = ld_global_nc(g + idx);
        e.dst = idx;
    }
    return e;
}

// Shared memory of a TMA-staged tile: keys, values (if VALS), the T source
// indices (if IDX) and the mbarrier.  SLACK: extra key slots after the
// windows, for walks that may read up to that far past them.
template <class K, bool VALS, int NT, int VT, bool IDX = true, int SLACK = 0>
struct BulkSmem {
    static constexpr int T = NT * VT;
    static constexpr int EK = 16 / sizeof(K);
    static constexpr size_t keys_bytes = ((size_t)(T + 3 * EK + SLACK) * sizeof(K) + 15) / 16 * 16;
    static constexpr size_t vals_bytes = VALS ? ((size_t)(T + 12) * 4 + 15) / 16 * 16 : 0;
    static constexpr size_t idx_bytes = IDX ? ((size_t)T * 2 + 15) / 16 * 16 : 0;
    static constexpr size_t bytes = keys_bytes + vals_bytes + idx_bytes + 16;  // + mbarrier
};

// Shared-memory regions of a TMA-staged tile (sidx is null without IDX).
template <class K, bool VALS, int NT, int VT, bool IDX = true, int SLACK = 0>
struct BulkLayout {
    K* sk;
    uint32_t* sv;
    uint16_t* sidx;
    uint64_t* bar;
    __device__ __forceinline__ explicit BulkLayout(unsigned char* smem)
    {
        using SM = BulkSmem<K, VALS, NT, VT, IDX, SLACK>;
        sk = reinterpret_cast<K*>(smem);
        sv = reinterpret_cast<uint32_t*>(smem + SM::keys_bytes);
        sidx = IDX ? reinterpret_cast<uint16_t*>(smem + SM::keys_bytes + SM::vals_bytes) : nullptr;
        bar = reinterpret_cast<uint64_t*>(smem + SM::keys_bytes + SM::vals_bytes + SM::idx_bytes);
    }
};

// Merge tiles of 4-byte keys alone with an odd number of outputs per thread
// keep the merged keys in registers and write them back over the windows
// (merge_tile_bulk_body), so they need no source indices.
template <class K, bool VALS, int VT>
constexpr bool merge_keys_direct()
{
    return !VALS && sizeof(K) == 4 && (VT & 1) != 0;
}

// Shared memory of merge_tile_bulk_body's tile.
template <class K, bool VALS, int NT, int VT>
using MergeBulkSmem = BulkSmem<K, VALS, NT, VT, !merge_keys_direct<K, VALS, VT>()>;

// Initialise the CTA's mbarrier (one thread); the caller then synchronises.
__device__ __forceinline__ void bulk_init(uint64_t* bar)
{
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
}

// Stage tile t into shared memory: thread 0 issues the bulk copies of the
// aligned interiors, threads [32, 32+4EK) and [64, 80) copy the ragged
// edges, every thread waits (bounded) for the mbarrier phase `parity`, and
// the block agrees on the outcome (the barrier also publishes the edges).
// Returns false, after recording MP_KERR_MBAR_TIMEOUT and giving copies in
// flight a bounded time to land, if the wait ran out.  err points at the
// kernel error word; err[1] is read as the fault switch described below.  The caller must have
// synchronised since the shared memory was last read.
template <class K, bool VALS, int NT, int VT>
__device__ __forceinline__ bool bulk_stage(const TilePlace<K>& t, const TileView<K, VALS, NT, VT>& v,
                                           uint64_t* bar, uint32_t parity, unsigned int* err)
{
    constexpr int EK = 16 / sizeof(K);
    constexpr uint32_t WAIT_LIMIT = 1u << 22;
    const int tid = threadIdx.x;
    if (tid == 0) {
        uint32_t tx = interior_bytes(t.gA, t.la) + interior_bytes(t.gB, t.lb);
        if constexpr (VALS) tx += interior_bytes(t.gvA, t.la) + interior_bytes(t.gvB, t.lb);
        mbar_arrive_expect_tx(bar, tx);
        issue_interior(v.sA, t.gA, t.la, bar);
        issue_interior(v.sB, t.gB, t.lb, bar);
        if constexpr (VALS) {
            issue_interior(v.vA, t.gvA, t.la, bar);
            issue_interior(v.vB, t.gvB, t.lb, bar);
        }
    }
    if (tid >= 32 && tid < 32 + 4 * EK) {
        const EdgeLoad<K> e = edge_load(tid - 32, t.gA, t.la, t.gB, t.lb);
        if (e.dst >= 0) (e.in_b ? v.sB : v.sA)[e.dst] = e.val;
    }
    if constexpr (VALS) {
        if (tid >= 64 && tid < 80) {
            const EdgeLoad<uint32_t> e = edge_load(tid - 64, t.gvA, t.la, t.gvB, t.lb);
            if (e.dst >= 0) (e.in_b ? v.vB : v.vA)[e.dst] = e.val;
        }
    }
    // err[1] is the staging-wait fault switch (a host-side test hook): when
    // set, the first wait gives up without polling, which exercises the
    // path below; the drain wait keeps its full bound, so the copies in
    // flight still land before the CTA returns.
    const uint32_t first_limit = __ldcg(err + 1) ? 0u : WAIT_LIMIT;
    const bool ok = __syncthreads_and(mbar_wait_bounded(bar, parity, first_limit));
    if (!ok) {
        if (tid == 0) atomicOr(err, MP_KERR_MBAR_TIMEOUT);
        mbar_wait_bounded(bar, parity, WAIT_LIMIT);
    }
    return ok;
}

// One tile of a merge problem (plain merge or sort pass) per CTA.
template <class K, bool VALS, int NT, int VT, int CK>
__device__ __forceinline__ void merge_tile_bulk_body(const TileArgs<K>& p, int64_t tile,
                                                     const int64_t* a_split, unsigned char* smem,
                                                     unsigned int* err)
{
    constexpr int T = NT * VT;
    constexpr bool DIRECT = merge_keys_direct<K, VALS, VT>();
    const int tid = threadIdx.x;
    const BulkLayout<K, VALS, NT, VT, !DIRECT> lay(smem);
    const TilePlace<K> t = tile_place(p, tile, T, a_split);
    const auto v = stage_view<K, VALS, NT, VT>(t, lay.sk, lay.sv, lay.sidx);
    bulk_init(lay.bar);
    __syncthreads();
    if (!bulk_stage<K, VALS, NT, VT>(t, v, lay.bar, 0, err)) return;
    const int L = t.la + t.lb;
    const int diag = tid * VT < L ? tid * VT : L;
    const int ai = smem_diagonal_search_ck<CK>(v.sA, t.la, v.sB, t.lb, diag, p.codec);
    if constexpr (DIRECT) {
        // 4-byte keys alone, odd VT: the merged keys stay in registers and
        // replace the windows in shared memory once every walk is done
        // (thread-major writes at an odd stride touch 32 different banks),
        // then leave with 128-bit loads and stores.  This skips the index
        // stores and the gather of the general path.
        K outk[VT];
        serial_merge_keys_ck<K, VT, CK>(v.sA, t.la, v.sB, t.lb, ai, diag - ai, p.codec, outk);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < VT; ++i) lay.sk[tid * VT + i] = outk[i];
        __syncthreads();
        store_linear<K, NT, VT>(lay.sk, L, p.out + t.d0);
    } else {
        uint32_t packed[(VT + 1) / 2];
        serial_merge_indices_ck<K, VT, CK>(v.sA, t.la, v.sB, t.lb, ai, diag - ai, p.codec, packed);
        put_indices<VT>(lay.sidx, packed);
        __syncthreads();
        store_tile<K, VALS, NT, VT, CK>(v, p.out + t.d0, VALS ? p.outv + t.d0 : nullptr, p.codec);
    }
}

// Order-sensitive fold of one merged output (key bits, value, position)
// into 64 bits; the checksum of a merge is the sum of these over all
// outputs (mod 2^64).
__device__ __forceinline__ uint64_t output_fold(uint64_t key, uint32_t val, bool vals, uint64_t pos)
{
    uint64_t h = key * 0x9E3779B97F4A7C15ull;
    if (vals) h ^= (uint64_t)val * 0xBF58476D1CE4E5B9ull;
    h ^= (pos + 1) * 0x94D049BB133111EBull;
    return h ^ (h >> 29);
}

// The merge with its results kept on chip: the tile is staged and merged as
// in merge_tile_bulk_body, but instead of being stored each output is folded
// into a per-thread sum, reduced over the CTA and written to partial[tile]
// (a second kernel adds the partials).  Global traffic is the read of A and
// B only (Sec. VI measures this variant to separate reading from writing).
template <class K, bool VALS, int NT, int VT, int CK>
__device__ __forceinline__ void merge_tile_checksum_body(const TileArgs<K>& p, int64_t tile,
                                                         const int64_t* a_split, unsigned char* smem,
                                                         unsigned int* err,
                                                         unsigned long long* partial)
{
    constexpr int T = NT * VT;
    const int tid = threadIdx.x;
    const BulkLayout<K, VALS, NT, VT> lay(smem);
    const TilePlace<K> t = tile_place(p, tile, T, a_split);
    const auto v = stage_view<K, VALS, NT, VT>(t, lay.sk, lay.sv, lay.sidx);
    bulk_init(lay.bar);
    __syncthreads();
    if (!bulk_stage<K, VALS, NT, VT>(t, v, lay.bar, 0, err)) return;
    const int L = t.la + t.lb;
    const int diag = tid * VT < L ? tid * VT : L;
    const int ai = smem_diagonal_search_ck<CK>(v.sA, t.la, v.sB, t.lb, diag, p.codec);
    uint32_t packed[(VT + 1) / 2];
    serial_merge_indices_ck<K, VT, CK>(v.sA, t.la, v.sB, t.lb, ai, diag - ai, p.codec, packed);
    uint64_t acc = 0;
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        if (diag + i < L) {
            const int src = (packed[i / 2] >> (16 * (i & 1))) & 0xFFFF;
            const K key = src < t.la ? v.sA[src] : v.sB[src - t.la];
            uint32_t val = 0;
            if constexpr (VALS) val = src < t.la ? v.vA[src] : v.vB[src - t.la];
            acc += output_fold((uint64_t)key, val, VALS, (uint64_t)(t.d0 + diag + i));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    __syncthreads();  // the index array is free again: reuse it for warp sums
    uint64_t* wsum = reinterpret_cast<uint64_t*>(lay.sidx);
    if ((tid & 31) == 0) wsum[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        uint64_t total = 0;
        for (int w = 0; w < NT / 32; ++w) total += wsum[w];
        partial[tile] = total;
    }
}



// ---------------------------------------------------------------------------
// Warp-cooperative tile (staging MP_STAGE_WARP).  After the TMA staging, each
// warp produces 32*VT consecutive outputs in steps of 32: it loads the next
// 32 elements of A and of B (consecutive shared addresses, no bank
// conflicts), ranks every candidate against the other side with warp
// shuffles (an A element's rank is its lane plus the number of B candidates
// strictly below it; a B element's is its lane plus the number of A
// candidates not above it, so ties take A), and writes the candidates whose
// rank is below 32 straight to their outputs.  By Lemma 16 the next 32
// outputs of the path lie among those 64 candidates.  Only the warp's first
// split is found by a diagonal search (Alg. 2), by one lane.
// ---------------------------------------------------------------------------
template <class K, bool VALS, int NT, int VT>
struct WarpSmem {
    static constexpr int T = NT * VT;
    static constexpr int EK = 16 / sizeof(K);
    static constexpr size_t keys_bytes = ((size_t)(T + 3 * EK) * sizeof(K) + 15) / 16 * 16;
    static constexpr size_t vals_bytes = VALS ? ((size_t)(T + 12) * 4 + 15) / 16 * 16 : 0;
    static constexpr size_t bytes = keys_bytes + vals_bytes + 16;  // + mbarrier
};

template <class K, bool VALS, int NT, int VT, int CK>
__device__ __forceinline__ void merge_tile_warp_body(const TileArgs<K>& p, int64_t tile,
                                                     const int64_t* a_split, unsigned char* smem,
                                                     unsigned int* err)
{
    using SM = WarpSmem<K, VALS, NT, VT>;
    constexpr int T = NT * VT;
    constexpr int W = 32 * VT;  // outputs per warp
    constexpr unsigned FULL = 0xFFFFFFFFu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    K* sk = reinterpret_cast<K*>(smem);
    uint32_t* sv = reinterpret_cast<uint32_t*>(smem + SM::keys_bytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::keys_bytes + SM::vals_bytes);

    const TilePlace<K> t = tile_place(p, tile, T, a_split);
    const auto v = stage_view<K, VALS, NT, VT>(t, sk, sv, nullptr);
    bulk_init(bar);
    __syncthreads();
    if (!bulk_stage<K, VALS, NT, VT>(t, v, bar, 0, err)) return;

    const int la = t.la, lb = t.lb, L = la + lb;
    const int p0 = warp * W;
    if (p0 >= L) return;
    const int pend = p0 + W < L ? p0 + W : L;
    int a = 0;
    if (lane == 0) a = smem_diagonal_search_ck<CK>(v.sA, la, v.sB, lb, p0, p.codec);
    a = __shfl_sync(FULL, a, 0);
    int b = p0 - a;
    K* gout = p.out + t.d0;
    uint32_t* gvout = VALS ? p.outv + t.d0 : nullptr;
    for (int pos = p0; pos < pend;) {
        const int n_out = pend - pos < 32 ? pend - pos : 32;
        const int nav = la - a < 32 ? la - a : 32;
        const int nbv = lb - b < 32 ? lb - b : 32;
        const bool va = lane < nav, vb = lane < nbv;
        const K ra = va ? v.sA[a + lane] : K(0);
        const K rb = vb ? v.sB[b + lane] : K(0);
        const K ka = key_enc_ck<CK>(ra, p.codec);
        const K kb = key_enc_ck<CK>(rb, p.codec);
        // cnt_b: B candidates strictly below ka; cnt_a: A candidates <= kb.
        int lo_b = 0, hi_b = nbv, lo_a = 0, hi_a = nav;
#pragma unroll
        for (int it = 0; it < 6; ++it) {
            const int mb = (lo_b + hi_b) >> 1;
            const int ma = (lo_a + hi_a) >> 1;
            const K kbm = __shfl_sync(FULL, kb, mb & 31);
            const K kam = __shfl_sync(FULL, ka, ma & 31);
            if (lo_b < hi_b) {
                if (kbm < ka) lo_b = mb + 1;
                else hi_b = mb;
            }
            if (lo_a < hi_a) {
                if (kam <= kb) lo_a = ma + 1;
                else hi_a = ma;
            }
        }
        const int r_a = lane + lo_b;
        const int r_b = lane + lo_a;
        const bool out_a = va && r_a < n_out;
        const bool out_b = vb && r_b < n_out;
        if (out_a) {
            gout[pos + r_a] = ra;
            if constexpr (VALS) gvout[pos + r_a] = v.vA[a + lane];
        }
        if (out_b) {
            gout[pos + r_b] = rb;
            if constexpr (VALS) gvout[pos + r_b] = v.vB[b + lane];
        }
        const int taken_a = __popc(__ballot_sync(FULL, out_a));
        a += taken_a;
        b += n_out - taken_a;
        pos += n_out;
    }
}

}  // namespace mp
