// setops.cu -- merge-based set operations on the Merge Path partitioning.
//
// Sec. I names joins of database query results and merges of adjacency
// lists as uses of merging.  Union, intersection, difference and symmetric
// difference of sorted A and B (multiset semantics: a key held m times by A
// and n times by B appears max(m,n), min(m,n), max(m-n,0) or |m-n| times;
// union keeps A's m copies and B's copies after the m-th, intersection A's
// first min(m,n), difference A's copies after the n-th, symmetric difference
// both of the latter) all emit a subsequence of the stable merge S of A and
// B.  Whether an element of S is emitted depends on its rank inside its run
// of equal keys on its own side and on the length of that key's run on the
// other side, so the method is the merge with a decision per output:
//   1. partition: Alg. 2 at every tile boundary (Cor. 6, as for the merge);
//   2. per tile (one CTA): stage the windows A[a0,a1), B[b0,b1) in shared
//      memory (TMA bulk copies, Lemma 16); each thread finds its split in
//      the windows (Thm 17), walks its VT outputs of S and decides each one.
//      Runs are measured inside the windows; a run that crosses a window
//      edge is completed with three galloping searches in global memory per
//      tile (the run ending at a0-1 in A, at b0-1 in B, the run starting at
//      b1 in B), done while the copies are in flight;
//   3. count-then-scatter: a count kernel walks every tile and stores the
//      number of outputs it keeps; a one-CTA scan turns the counts into
//      tile offsets (and the result length); an emit kernel walks every tile
//      again, places each kept output by a block scan of the kept counts and
//      writes them contiguously at the tile's offset.  The inputs are read
//      twice, but no CTA ever waits on another (a single-pass version with a
//      decoupled look-back across tiles spent most of its time in that wait).
#include <algorithm>

#include "mp_bulk.cuh"
#include "mp_device.cuh"
#include "mp_internal.h"
#include "mp_tile.cuh"

namespace mp {

// Bit set in the kernel error word when a set operation's output would pass
// the capacity (inputs not sorted).
#define MP_KERR_SETOP 2u

template <class K>
struct SetArgs {
    TileArgs<K> t;           // the merge problem (run == 0) and split points
    int op;                  // MP_SET_*
    int64_t ntiles;
    int64_t cap;             // output capacity (elements)
    uint32_t* counts;           // count kernel: kept outputs per tile
    const int64_t* offsets;     // emit kernel: exclusive prefix inside the scan block
    const int64_t* block_sums;  // emit kernel: total of each scan block
    int64_t* count;             // emit kernel (last tile): the result length
};

// Tiles per block of the offset scan.
constexpr int SET_SCAN_BLOCK = 1024;

// First index of the run of X[i]'s key that contains i (galloping down).
template <class K>
__device__ int64_t run_start(const K* X, int64_t i)
{
    const K v = X[i];
    int64_t hi = i, lo = -1, step = 1;
    while (true) {
        const int64_t probe = hi - step;
        if (probe < 0) break;
        if (X[probe] != v) {
            lo = probe;
            break;
        }
        hi = probe;
        step <<= 1;
    }
    while (hi - lo > 1) {  // X[lo] != v (or lo = -1), X[hi] == v
        const int64_t mid = lo + (hi - lo) / 2;
        if (X[mid] == v) hi = mid;
        else lo = mid;
    }
    return hi;
}

// One past the last index of the run of X[i]'s key that contains i.
template <class K>
__device__ int64_t run_end(const K* X, int64_t n, int64_t i)
{
    const K v = X[i];
    int64_t lo = i, hi = n, step = 1;
    while (true) {
        const int64_t probe = lo + step;
        if (probe >= n) break;
        if (X[probe] != v) {
            hi = probe;
            break;
        }
        lo = probe;
        step <<= 1;
    }
    while (hi - lo > 1) {  // X[lo] == v, X[hi] != v (or hi = n)
        const int64_t mid = lo + (hi - lo) / 2;
        if (X[mid] == v) lo = mid;
        else hi = mid;
    }
    return hi;
}

// Runs that cross the window edges (raw key bits: equal keys are equal bits).
template <class K>
struct SetCtx {
    K prev_a, prev_b, next_b;
    int64_t lb_prev_a, lb_prev_b, ub_next_b;
    int has_prev_a, has_prev_b, has_next_b;
};

template <class K, bool VALS, int NT, int VT>
struct SetSmem {
    using B = BulkSmem<K, VALS, NT, VT>;
    static constexpr size_t ctx_off = (B::bytes + 15) / 16 * 16;
    static constexpr size_t scan_off = ctx_off + (sizeof(SetCtx<K>) + 15) / 16 * 16;
    static constexpr size_t bytes = scan_off + (NT / 32 + 4) * 8;
};

// First index x in [lo, hi] with s[x] == v, given s[hi] == v (and the run
// of v is contiguous).
template <class K>
__device__ __forceinline__ int first_equal(const K* s, int lo, int hi, K v)
{
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s[mid] == v) hi = mid;
        else lo = mid + 1;
    }
    return hi;
}

// Decision for an output whose key v also occurs on the other side and
// repeats (or may repeat) beyond the immediate neighbours: measure the runs.
//   from A (window index ai, B pointer bi = start of v's run in B): keep for
//     intersection iff r_a < n, for difference / symmetric iff r_a >= n,
//     where r_a = rank of this copy in A's run of v and n = length of v's
//     run in B;
//   from B (index bi, A pointer ai = one past v's run in A): keep for union /
//     symmetric iff r_b >= m, r_b = rank in B's run, m = length of A's run.
template <class K>
__device__ __noinline__ bool setop_slow(bool from_a, K v, int ai, int bi, const K* sA, int la, const K* sB,
                                        int lb, int op, const SetCtx<K>& x, int64_t a0, int64_t b0)
{
    if (from_a) {
        int64_t r_a = 0;
        if ((ai > 0 && sA[ai - 1] == v) || (ai == 0 && x.has_prev_a && x.prev_a == v)) {
            const int f = first_equal(sA, 0, ai, v);
            const int64_t start = (f == 0 && x.has_prev_a && x.prev_a == v) ? x.lb_prev_a : a0 + f;
            r_a = a0 + ai - start;
        }
        int64_t end;
        if (bi >= lb) {
            end = x.ub_next_b;
        } else {
            int lo = bi, hi = lb;  // sB[lo] == v; first index != v in (lo, lb]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (sB[mid] == v) lo = mid;
                else hi = mid;
            }
            end = (hi == lb && x.has_next_b && x.next_b == v) ? x.ub_next_b : b0 + hi;
        }
        const int64_t n = end - (b0 + bi);
        return op == MP_SET_INTERSECTION ? r_a < n : r_a >= n;
    }
    int64_t start;
    if (ai == 0) {
        start = x.lb_prev_a;
    } else {
        const int f = first_equal(sA, 0, ai - 1, v);
        start = (f == 0 && x.has_prev_a && x.prev_a == v) ? x.lb_prev_a : a0 + f;
    }
    const int64_t m = a0 + ai - start;
    int64_t r_b = 0;
    if ((bi > 0 && sB[bi - 1] == v) || (bi == 0 && x.has_prev_b && x.prev_b == v)) {
        const int f = first_equal(sB, 0, bi, v);
        const int64_t bs = (f == 0 && x.has_prev_b && x.prev_b == v) ? x.lb_prev_b : b0 + f;
        r_b = b0 + bi - bs;
    }
    return r_b >= m;
}

// Walk VT outputs of the tile's merge from split (ai, bi) and decide each:
// records sources (A: 0..la-1, B: la..; when SRC) and returns a bit mask of
// kept outputs.  Equal keys are equal bits.  The walk is the plain merge
// (Alg. 1's Merge) recording three bits per output: taken from A; its key
// is held by the other side (for an A output: B's pointer is at an equal
// key, ties taking A; for a B output: the last A taken is equal); its key
// repeats on its own side (the previous element of that side is equal).
// An output whose key is not repeated is the first copy of its run (rank
// 0), and rank 0 < n, rank 0 >= m hold or fail whatever the run lengths
// n, m >= 1 of the other side are, so the operation's rule reduces to bit
// operations:
//   union         A outputs, and B outputs without a partner;
//   intersection  A outputs with a partner;
//   difference    A outputs without a partner;
//   symmetric     outputs without a partner.
// Outputs that have a partner and repeat go to setop_slow (rare).
template <class K, int VT, int CK, bool SRC>
__device__ __forceinline__ uint32_t setop_walk(const K* sA, int la, const K* sB, int lb, int ai, int bi,
                                               int n_valid, int op, const SetCtx<K>& x, int64_t a0,
                                               int64_t b0, Codec<K> c, uint32_t (&packed)[(VT + 1) / 2])
{
    static_assert(VT <= 32, "one bit per output");
    const int ai0 = ai, bi0 = bi;
    K ra = sA[ai], rb = sB[bi];
    K ka = key_enc_ck<CK>(ra, c), kb = key_enc_ck<CK>(rb, c);
    bool last_a_ok = ai > 0 || x.has_prev_a;
    K last_a = ai > 0 ? sA[ai - 1] : x.prev_a;
    bool last_b_ok = bi > 0 || x.has_prev_b;
    K last_b = bi > 0 ? sB[bi - 1] : x.prev_b;
    uint32_t took_a = 0, partner = 0, repeat = 0;
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        const bool take_a = (bi >= lb) || (ai < la && !(ka > kb));
        const K v = take_a ? ra : rb;
        const bool a_last = last_a_ok && last_a == v;
        const bool match = take_a ? (bi < lb ? rb == v : (x.has_next_b && x.next_b == v)) : a_last;
        const bool dup = take_a ? a_last : (last_b_ok && last_b == v);
        took_a |= (uint32_t)take_a << i;
        partner |= (uint32_t)match << i;
        repeat |= (uint32_t)dup << i;
        if constexpr (SRC) {
            const uint32_t src = take_a ? (uint32_t)ai : (uint32_t)(la + bi);
            if (i & 1) packed[i / 2] |= src << 16;
            else packed[i / 2] = src;
        }
        const K* nxt = take_a ? (sA + (ai < la ? ai + 1 : la)) : (sB + bi + 1);
        const K rn = *nxt;
        const K kn = key_enc_ck<CK>(rn, c);
        if (take_a) {
            last_a = v;
            last_a_ok = true;
            ra = rn;
            ka = kn;
            ++ai;
        } else {
            last_b = v;
            last_b_ok = true;
            rb = rn;
            kb = kn;
            ++bi;
        }
    }
    const uint32_t all = VT == 32 ? 0xFFFFFFFFu : ((1u << VT) - 1);
    const uint32_t valid = n_valid >= VT ? all : (n_valid > 0 ? (1u << n_valid) - 1 : 0u);
    uint32_t keep, slow_sides;
    switch (op) {
    case MP_SET_UNION:
        keep = took_a | ~partner;
        slow_sides = ~took_a;
        break;
    case MP_SET_INTERSECTION:
        keep = took_a & partner;
        slow_sides = took_a;
        break;
    case MP_SET_DIFFERENCE:
        keep = took_a & ~partner;
        slow_sides = took_a;
        break;
    default:
        keep = ~partner;
        slow_sides = all;
        break;
    }
    uint32_t slow = partner & repeat & slow_sides & valid;
    while (slow) {
        const int i = __ffs(slow) - 1;
        slow &= slow - 1;
        const int na = __popc(took_a & ((1u << i) - 1));
        const bool take_a = (took_a >> i) & 1;
        const int ai_i = ai0 + na, bi_i = bi0 + (i - na);
        const K v = take_a ? sA[ai_i] : sB[bi_i];
        const bool kp = setop_slow(take_a, v, ai_i, bi_i, sA, la, sB, lb, op, x, a0, b0);
        keep = (keep & ~(1u << i)) | ((uint32_t)kp << i);
    }
    return keep & valid;
}

// Stage tile `tile`, find the runs crossing the window edges, and walk this
// thread's VT outputs.  Returns false (all threads) if the staging wait ran
// out.
template <class K, bool VALS, int NT, int VT, int CK, bool SRC>
__device__ __forceinline__ bool setop_tile_walk(const SetArgs<K>& p, int64_t tile, unsigned char* smem,
                                                unsigned int* err, TilePlace<K>& t,
                                                TileView<K, VALS, NT, VT>& v, uint32_t (&packed)[(VT + 1) / 2],
                                                uint32_t& keep, unsigned long long* place = nullptr)
{
    using SM = SetSmem<K, VALS, NT, VT>;
    constexpr int T = NT * VT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const BulkLayout<K, VALS, NT, VT> lay(smem);
    SetCtx<K>& x = *reinterpret_cast<SetCtx<K>*>(smem + SM::ctx_off);
    const TileArgs<K>& ta = p.t;
    t = tile_place(ta, tile, T, ta.a_split);
    v = stage_view<K, VALS, NT, VT>(t, lay.sk, lay.sv, lay.sidx);
    const int64_t a0 = t.gA - ta.a, b0 = t.gB - ta.b;
    const int64_t b1 = b0 + t.lb;
    bulk_init(lay.bar);
    __syncthreads();
    if (place && warp == 2) {
        // The tile's place in the result: its offset inside its scan block
        // plus the totals of the earlier blocks (while the copies fly).
        const int64_t blk = tile / SET_SCAN_BLOCK;
        unsigned long long sum = 0;
        for (int64_t j = lane; j < blk; j += 32) sum += (unsigned long long)p.block_sums[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
        if (lane == 0) *place = sum + (unsigned long long)p.offsets[tile];
    }
    if (warp == 3) {  // the keys just outside the windows, while the copies fly
        if (lane == 0) {
            x.has_prev_a = a0 > 0;
            if (a0 > 0) x.prev_a = ld_global_nc(ta.a + a0 - 1);
        } else if (lane == 1) {
            x.has_prev_b = b0 > 0;
            if (b0 > 0) x.prev_b = ld_global_nc(ta.b + b0 - 1);
        } else if (lane == 2) {
            x.has_next_b = b1 < ta.nb;
            if (b1 < ta.nb) x.next_b = ld_global_nc(ta.b + b1);
        }
    }
    // The staging barrier also publishes x.
    if (!bulk_stage<K, VALS, NT, VT>(t, v, lay.bar, 0, err)) return false;
    // Run lengths are consulted only for outputs whose key repeats on its own
    // side and occurs on the other (setop_slow).  A run crossing a window
    // edge is then measured in global memory, once per tile (the condition
    // is the same on every thread): the run ending at a0-1 in A when A's
    // window starts inside it, or when B's window starts with its key and
    // that key repeats in B; the run ending at b0-1 in B when B's window
    // starts inside it; the run starting at b1 in B when B's window ends
    // inside it, or when A's window ends with its key and that key repeats
    // in A.  Duplicate-free inputs never need them.
    const int la = t.la, lb = t.lb;
    const bool b0_rep = lb > 0 && ((lb > 1 && v.sB[1] == v.sB[0]) || (x.has_prev_b && x.prev_b == v.sB[0]));
    const bool a_end_rep =
        la > 0 && ((la > 1 && v.sA[la - 2] == v.sA[la - 1]) || (la == 1 && x.has_prev_a && x.prev_a == v.sA[0]));
    const bool need_a = x.has_prev_a && ((la > 0 && v.sA[0] == x.prev_a) || (b0_rep && v.sB[0] == x.prev_a));
    const bool need_b = x.has_prev_b && lb > 0 && v.sB[0] == x.prev_b;
    const bool need_n = x.has_next_b &&
                        ((lb > 0 && v.sB[lb - 1] == x.next_b) || (a_end_rep && v.sA[la - 1] == x.next_b));
    if (need_a || need_b || need_n) {
        if (warp == 3) {
            if (lane == 0 && need_a) x.lb_prev_a = run_start(ta.a, a0 - 1);
            if (lane == 1 && need_b) x.lb_prev_b = run_start(ta.b, b0 - 1);
            if (lane == 2 && need_n) x.ub_next_b = run_end(ta.b, ta.nb, b1);
        }
        __syncthreads();
    }
    const int L = t.la + t.lb;
    const int diag = tid * VT < L ? tid * VT : L;
    const int ai = smem_diagonal_search_ck<CK>(v.sA, t.la, v.sB, t.lb, diag, ta.codec);
    keep = setop_walk<K, VT, CK, SRC>(v.sA, t.la, v.sB, t.lb, ai, diag - ai, L - diag, p.op, x, a0, b0,
                                      ta.codec, packed);
    return true;
}

// Pass 1: kept outputs per tile.
template <class K, bool VALS, int NT, int VT, int CK>
__global__ void __launch_bounds__(NT, sizeof(K) == 4 ? 4 : 2) setop_count_kernel(SetArgs<K> p, unsigned int* err)
{
    using SM = SetSmem<K, VALS, NT, VT>;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* scan = reinterpret_cast<unsigned long long*>(smem + SM::scan_off);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    TilePlace<K> t;
    TileView<K, VALS, NT, VT> v;
    uint32_t packed[(VT + 1) / 2];
    uint32_t keep = 0;
    if (!setop_tile_walk<K, VALS, NT, VT, CK, false>(p, blockIdx.x, smem, err, t, v, packed, keep, nullptr))
        return;
    int c = __popc(keep);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane == 0) scan[warp] = (unsigned long long)c;
    __syncthreads();
    if (tid == 0) {
        unsigned long long total = 0;
        for (int w = 0; w < NW; ++w) total += scan[w];
        p.counts[blockIdx.x] = (uint32_t)total;
    }
}

// Pass 2: exclusive scan of the counts inside blocks of NT tiles:
// offsets[t] = counts of the earlier tiles of t's block, block_sums[b] = the
// block's total.  The emit kernel adds the block sums of earlier blocks.
template <int NT>
__global__ void __launch_bounds__(NT) setop_scan_kernel(const uint32_t* counts, int64_t ntiles,
                                                        int64_t* offsets, int64_t* block_sums)
{
    __shared__ unsigned long long wsum[NT / 32];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = (int64_t)blockIdx.x * NT + tid;
    const unsigned long long c = i < ntiles ? counts[i] : 0;
    unsigned long long incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = lane < NT / 32 ? wsum[lane] : 0;
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < NT / 32) wsum[lane] = wi - w;
        if (lane == 31) block_sums[blockIdx.x] = (int64_t)wi;
    }
    __syncthreads();
    if (i < ntiles) offsets[i] = (int64_t)(wsum[warp] + incl - c);
}

// Pass 3: walk again, place the kept outputs, write them at the tile's offset.
template <class K, bool VALS, int NT, int VT, int CK>
__global__ void __launch_bounds__(NT, sizeof(K) == 4 ? 4 : 2) setop_emit_kernel(SetArgs<K> p, unsigned int* err)
{
    using SM = SetSmem<K, VALS, NT, VT>;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* scan = reinterpret_cast<unsigned long long*>(smem + SM::scan_off);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    TilePlace<K> t;
    TileView<K, VALS, NT, VT> v;
    uint32_t packed[(VT + 1) / 2];
    uint32_t keep = 0;
    if (!setop_tile_walk<K, VALS, NT, VT, CK, true>(p, blockIdx.x, smem, err, t, v, packed, keep, &scan[NW + 1]))
        return;
    const int c = __popc(keep);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) scan[warp] = (unsigned long long)incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = lane < NW ? scan[lane] : 0;
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < NW) scan[lane] = wi - w;  // exclusive warp offsets
        if (lane == 31) scan[NW] = wi;       // tile total
    }
    __syncthreads();
    const int64_t g = (int64_t)scan[NW + 1];
    const int n_out = (int)scan[NW];
    if (g < 0 || g + n_out > p.cap) {
        if (tid == 0) atomicOr(err, MP_KERR_SETOP);
        return;
    }
    // Compact the kept sources into the index array (the staged windows stay
    // where they are; only indices move).
    uint16_t* sidx = v.sidx;
    int pos = (int)scan[warp] + incl - c;
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        if (keep & (1u << i)) sidx[pos++] = (uint16_t)((packed[i / 2] >> (16 * (i & 1))) & 0xFFFF);
    }
    __syncthreads();
    const TileArgs<K>& ta = p.t;
    K* gout = ta.out + g;
    for (int j = tid; j < n_out; j += NT) {
        const int s = sidx[j];
        gout[j] = s < t.la ? v.sA[s] : v.sB[s - t.la];
    }
    if constexpr (VALS) {
        uint32_t* gvout = ta.outv + g;
        for (int j = tid; j < n_out; j += NT) {
            const int s = sidx[j];
            gvout[j] = s < t.la ? v.vA[s] : v.vB[s - t.la];
        }
    }
    if (tid == 0 && blockIdx.x == p.ntiles - 1) *p.count = g + n_out;
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
constexpr int SET_NT = 256;
// Items per thread (one bit each in the walk's masks, so at most 32).  An
// odd count starts the threads' walks in different shared-memory banks and
// spreads each thread's search over more outputs (two sets of 2^27 keys:
// uint32 union 1.50 -> 1.25 ms at 31, int64 union 1.47 -> 1.06 ms at 15;
// with values 27 beats 31).  16-byte keys keep 8.
constexpr int set_vt(int key_bytes, bool vals)
{
    return key_bytes == 4 ? (vals ? 27 : 31) : (key_bytes == 8 ? 15 : 8);
}

int64_t setop_tile(int key_bytes, bool vals) { return (int64_t)SET_NT * set_vt(key_bytes, vals); }

static cudaError_t pdl_launch_cfg(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, unsigned grid,
                                  unsigned block, size_t smem, cudaStream_t stream)
{
    cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaSuccess;
}

template <class K, bool VALS, int CK>
static cudaError_t launch_setop_ck(const MergeProblem& mp_, int op, const int64_t* splits, uint32_t* counts,
                                   int64_t* offsets, int64_t* block_sums, int64_t cap, int64_t* count,
                                   cudaStream_t stream)
{
    constexpr int VT = set_vt((int)sizeof(K), VALS);
    using SM = SetSmem<K, VALS, SET_NT, VT>;
    using SMK = SetSmem<K, false, SET_NT, VT>;  // the count pass stages keys only
    auto kcount = setop_count_kernel<K, false, SET_NT, VT, CK>;
    auto kemit = setop_emit_kernel<K, VALS, SET_NT, VT, CK>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kcount, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMK::bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kemit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    unsigned int* err = kernel_error_word();
    if (!err) return cudaErrorInvalidSymbol;
    SetArgs<K> a;
    TileArgs<K>& t = a.t;
    t.a = static_cast<const K*>(mp_.a);
    t.b = static_cast<const K*>(mp_.b);
    t.av = mp_.av;
    t.bv = mp_.bv;
    t.out = static_cast<K*>(mp_.out);
    t.outv = mp_.outv;
    t.na = mp_.na;
    t.nb = mp_.nb;
    t.run = 0;
    t.total = mp_.na + mp_.nb;
    t.a_split = splits;
    t.codec = make_codec<K>(mp_.kind.flip, mp_.kind.fmask, mp_.kind.inv);
    a.op = op;
    a.ntiles = ceil_div(t.total, setop_tile((int)sizeof(K), VALS));
    a.cap = cap;
    a.counts = counts;
    a.offsets = offsets;
    a.block_sums = block_sums;
    a.count = count;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    // The count pass reads keys only: same arguments, no values.
    SetArgs<K> ak = a;
    ak.t.av = ak.t.bv = nullptr;
    ak.t.outv = nullptr;
    pdl_launch_cfg(cfg, attr, (unsigned)a.ntiles, SET_NT, SMK::bytes, stream);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kcount, ak, err);
    if (e != cudaSuccess) return e;
    const int64_t nblk = ceil_div(a.ntiles, (int64_t)SET_SCAN_BLOCK);
    pdl_launch_cfg(cfg, attr, (unsigned)nblk, SET_SCAN_BLOCK, 0, stream);
    e = cudaLaunchKernelEx(&cfg, setop_scan_kernel<SET_SCAN_BLOCK>, (const uint32_t*)counts, a.ntiles, offsets,
                           block_sums);
    if (e != cudaSuccess) return e;
    pdl_launch_cfg(cfg, attr, (unsigned)a.ntiles, SET_NT, SM::bytes, stream);
    return cudaLaunchKernelEx(&cfg, kemit, a, err);
}

template <class K, bool VALS>
static cudaError_t launch_setop_t(const MergeProblem& p, int op, const int64_t* splits, uint32_t* counts,
                                  int64_t* offsets, int64_t cap, int64_t* count, cudaStream_t stream)
{
    // Block sums follow the offsets (one per SET_SCAN_BLOCK tiles).
    const int64_t ntiles = ceil_div(p.na + p.nb, setop_tile(p.kind.bytes, VALS));
    int64_t* block_sums = offsets + ntiles;
    if (p.kind.identity())
        return launch_setop_ck<K, VALS, CODEC_IDENTITY>(p, op, splits, counts, offsets, block_sums, cap, count,
                                                        stream);
    if (p.kind.signed_int())
        return launch_setop_ck<K, VALS, CODEC_SIGNED>(p, op, splits, counts, offsets, block_sums, cap, count,
                                                      stream);
    return launch_setop_ck<K, VALS, CODEC_RUNTIME>(p, op, splits, counts, offsets, block_sums, cap, count, stream);
}

cudaError_t launch_setop(const MergeProblem& p, int op, const int64_t* splits, uint32_t* counts,
                         int64_t* offsets, int64_t cap, int64_t* count, cudaStream_t stream)
{
    if (p.kind.bytes == 4)
        return p.vals ? launch_setop_t<uint32_t, true>(p, op, splits, counts, offsets, cap, count, stream)
                      : launch_setop_t<uint32_t, false>(p, op, splits, counts, offsets, cap, count, stream);
    if (p.kind.bytes == 16)
        return p.vals ? launch_setop_t<u128, true>(p, op, splits, counts, offsets, cap, count, stream)
                      : launch_setop_t<u128, false>(p, op, splits, counts, offsets, cap, count, stream);
    return p.vals ? launch_setop_t<uint64_t, true>(p, op, splits, counts, offsets, cap, count, stream)
                  : launch_setop_t<uint64_t, false>(p, op, splits, counts, offsets, cap, count, stream);
}

}  // namespace mp

using namespace mp;

extern "C" {

int64_t mp_set_capacity(mp_setop op, int64_t na, int64_t nb)
{
    if (na < 0 || nb < 0) return -1;
    switch (op) {
    case MP_SET_UNION:
    case MP_SET_SYMMETRIC_DIFFERENCE: return na + nb;
    case MP_SET_INTERSECTION: return na < nb ? na : nb;
    case MP_SET_DIFFERENCE: return na;
    }
    return -1;
}

mp_status mp_set_operation(mp_setop op, mp_dtype dtype, const void* a_keys, const uint32_t* a_vals, int64_t na,
                           const void* b_keys, const uint32_t* b_vals, int64_t nb, void* out_keys,
                           uint32_t* out_vals, int64_t* out_count, mp_stream_t stream)
{
    static const char* fn = "mp_set_operation";
    KeyKind k;
    if (!key_kind(dtype, &k)) return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_set_operation: unknown dtype");
    const int64_t cap = mp_set_capacity(op, na, nb);
    if (cap < 0) return fail(MP_ERR_INVALID_ARG, "mp_set_operation: unknown op or negative size");
    if (!out_count || ((uintptr_t)out_count & 7))
        return fail(MP_ERR_INVALID_ARG, "mp_set_operation: out_count NULL or not 8-byte aligned");
    const bool vals = a_vals || b_vals || out_vals;
    mp_status st = check_merge_args_ext(k, a_keys, a_vals, na, b_keys, b_vals, nb, out_keys, out_vals, vals, fn, cap);
    if (st != MP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (na + nb == 0) {
        cudaError_t e = cudaMemsetAsync(out_count, 0, sizeof(int64_t), s);
        return e == cudaSuccess ? MP_OK : cuda_fail(e, fn);
    }
    MergeProblem p;
    p.kind = k;
    p.vals = vals;
    p.a = a_keys;
    p.b = b_keys;
    p.av = a_vals;
    p.bv = b_vals;
    p.out = out_keys;
    p.outv = out_vals;
    p.na = na;
    p.nb = nb;
    p.run = 0;
    const int64_t T = setop_tile(k.bytes, vals);
    const int64_t ntiles = ceil_div(na + nb, T);
    const size_t split_bytes = (size_t)(ntiles + 1) * 8;
    const size_t offset_bytes = (size_t)(ntiles + ceil_div(ntiles, (int64_t)SET_SCAN_BLOCK)) * 8;
    const size_t count_bytes = (size_t)ntiles * 4;
    unsigned char* scratch = nullptr;
    st = scratch_alloc((void**)&scratch, split_bytes + offset_bytes + count_bytes, s);
    if (st != MP_OK) return st;
    int64_t* splits = reinterpret_cast<int64_t*>(scratch);
    int64_t* offsets = reinterpret_cast<int64_t*>(scratch + split_bytes);
    uint32_t* counts = reinterpret_cast<uint32_t*>(scratch + split_bytes + offset_bytes);
    cudaError_t e = launch_partition(p, T, splits, s);
    if (e == cudaSuccess) e = launch_setop(p, (int)op, splits, counts, offsets, cap, out_count, s);
    scratch_free(scratch, s);
    return e == cudaSuccess ? MP_OK : cuda_fail(e, fn);
}

}  // extern "C"
