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
//   2. per tile: stage the windows A[a0,a1), B[b0,b1) in shared memory
//      (TMA bulk copies, Lemma 16); each thread finds its split in the
//      windows (Thm 17), walks its VT outputs of S and decides each one.
//      Runs are measured inside the windows; a run that crosses a window
//      edge is completed with three galloping searches in global memory per
//      tile (the run ending at a0-1 in A, at b0-1 in B, the run starting at
//      b1 in B);
//   3. placement: tiles are taken in order from a counter; each publishes
//      its kept count as soon as its walk is done and adds up the counts of
//      the tiles before it back to the nearest one that has published its
//      inclusive prefix (a decoupled look-back); its kept outputs are
//      compacted in shared memory and written at that offset.  One pass over
//      the inputs.  (A count pass + scan + emit pass, which reads the inputs
//      twice and walks every tile twice, measured slower: 0.89 ms against
//      0.82 ms for the union of two 2^27-key sets.)
// Tiles of keys alone run in a persistent kernel whose CTAs overlap the
// copies, walk, look-back and store of consecutive tiles (setop_keys_kernel:
// 0.81 -> 0.68 ms for that union); tiles with values run one per CTA
// (setop_kernel).
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
    TileArgs<K> t;                // the merge problem (run == 0) and split points
    int op;                       // MP_SET_*
    int64_t ntiles;
    int64_t cap;                  // output capacity (elements)
    unsigned long long* status;   // one look-back word per tile, zeroed
    unsigned int* tile_counter;   // zeroed
    int64_t* count;               // the last tile: the result length
};

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
    K prev_a, prev_b, next_a, next_b;
    int64_t lb_prev_a, lb_prev_b, ub_next_b;
    int has_prev_a, has_prev_b, has_next_a, has_next_b;
};

// Shared memory of a tile with values (setop_kernel): the staged windows with
// their source indices, the run context, the scan and the thread splits.
template <class K, bool VALS, int NT, int VT>
struct SetSmem {
    using B = BulkSmem<K, VALS, NT, VT, true>;
    static constexpr size_t ctx_off = (B::bytes + 15) / 16 * 16;
    static constexpr size_t scan_off = ctx_off + (sizeof(SetCtx<K>) + 15) / 16 * 16;
    static constexpr size_t bytes = scan_off + (NT / 32 + 4) * 8;
};

// Order test of two stored keys under a codec kind: unsigned keys compare
// as they are, signed integers as signed integers, others through the
// encoding.
template <int CK, class K>
__device__ __forceinline__ bool key_gt_ck(K x, K y, Codec<K> c)
{
    if constexpr (CK == CODEC_IDENTITY)
        return x > y;
    else if constexpr (CK == CODEC_SIGNED)
        return (signed_of<K>)x > (signed_of<K>)y;
    else
        return key_enc_ck<CK>(x, c) > key_enc_ck<CK>(y, c);
}

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
// records sources (A: 0..la-1, B: la..) and returns a bit mask of
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
template <class K, int VT, int CK>
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
        const uint32_t src = take_a ? (uint32_t)ai : (uint32_t)(la + bi);
        if (i & 1) packed[i / 2] |= src << 16;
        else packed[i / 2] = src;
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

// The decision of one output from scratch (the outputs the neighbour rule
// below leaves open): whether its key occurs on the other side, then, if it
// does, its rank and the other side's run length (setop_slow).
template <class K>
__device__ __noinline__ bool setop_exact(bool from_a, K v, int ai, int bi, const K* sA, int la, const K* sB,
                                         int lb, int op, const SetCtx<K>& x, int64_t a0, int64_t b0)
{
    bool partner;
    if (from_a)  // B's pointer is at the first B key not below v
        partner = bi < lb ? sB[bi] == v : (x.has_next_b && x.next_b == v);
    else         // A's pointer is one past the last A key not above v
        partner = ai > 0 ? sA[ai - 1] == v : (x.has_prev_a && x.prev_a == v);
    if (partner) return setop_slow(from_a, v, ai, bi, sA, la, sB, lb, op, x, a0, b0);
    // No copy on the other side: every copy of this side is kept, by every
    // operation that emits this side.
    return from_a ? op != MP_SET_INTERSECTION : true;
}

// The walk for tiles without values: the merged keys stay in registers
// (as stored, out[]) with one bit per output for its side, and each output is
// decided from its neighbours in the merge.  In the stable merge the copies
// of a key form one run, A's copies first, so:
//   an A output whose next output is B's copy of the same key has a partner
//   (and is the last A copy), one whose next output has another key has
//   none; a B output whose previous output is A's copy of the same key has
//   a partner and is B's first copy, one whose previous output has another
//   key has none and is B's first copy.
// The first copy of a run decides by the partner bit alone (see setop_walk);
// A copies after the first with no partner keep or drop as the first does.
// What is left -- an A output followed by another A copy, an A copy after
// the first with a partner, a B copy after the first -- occurs only with
// repeated keys and is decided exactly (setop_exact).  The outputs just
// before and after the thread's share come from the windows or, at the
// tile's edges, from the keys next to the windows.
template <class K, int VT, int CK>
__device__ __forceinline__ uint32_t setop_walk_keys(const K* sA, int la, const K* sB, int lb, int ai, int bi,
                                                    int n_valid, bool inside, int op, const SetCtx<K>& x,
                                                    int64_t a0, int64_t b0, Codec<K> c,
                                                    K (&out)[VT])
{
    static_assert(VT <= 32, "one bit per output");
    const int ai0 = ai, bi0 = bi;
    // The output before the share: the later (in merge order) of A[ai-1]
    // and B[bi-1]; A's comes first on equal keys.
    const bool has_pa = ai > 0 || x.has_prev_a, has_pb = bi > 0 || x.has_prev_b;
    const K pa = ai > 0 ? sA[ai - 1] : x.prev_a;
    const K pb = bi > 0 ? sB[bi - 1] : x.prev_b;
    const bool prev_is_a = has_pa && (!has_pb || key_gt_ck<CK>(pa, pb, c));
    const bool has_prev = has_pa || has_pb;
    const K prev = prev_is_a ? pa : pb;
    K ka = sA[ai], kb = sB[bi];
    uint32_t took = 0, eqp = 0;  // output i from A; output i equals output i - 1
    K last = prev;
    if (inside) {
        // The share ends inside both windows: every head read is a real
        // element, so the steps need no end tests.
#pragma unroll
        for (int i = 0; i < VT; ++i) {
            const bool take_a = !key_gt_ck<CK>(ka, kb, c);
            const K v = take_a ? ka : kb;
            out[i] = v;
            took |= (uint32_t)take_a << i;
            eqp |= (uint32_t)(v == last) << i;
            last = v;
            const K kn = take_a ? sA[ai + 1] : sB[bi + 1];
            if (take_a) { ka = kn; ++ai; }
            else { kb = kn; ++bi; }
        }
    } else {
#pragma unroll
        for (int i = 0; i < VT; ++i) {
            const bool take_a = (bi >= lb) || (ai < la && !key_gt_ck<CK>(ka, kb, c));
            const K v = take_a ? ka : kb;
            out[i] = v;
            took |= (uint32_t)take_a << i;
            eqp |= (uint32_t)(v == last) << i;
            last = v;
            const K kn = take_a ? sA[ai < la ? ai + 1 : la] : sB[bi + 1];
            if (take_a) { ka = kn; ++ai; }
            else { kb = kn; ++bi; }
        }
    }
    const uint32_t all = VT == 32 ? 0xFFFFFFFFu : ((1u << VT) - 1);
    const uint32_t valid = n_valid >= VT ? all : (n_valid > 0 ? (1u << n_valid) - 1 : 0u);
    // The output after the share (only when the share is full: a partial
    // share is the end of the whole merge).
    bool next_is_a = false, has_next = false;
    K next = K(0);
    if (n_valid >= VT) {
        const bool has_na = ai < la || x.has_next_a, has_nb = bi < lb || x.has_next_b;
        const K na = ai < la ? ka : x.next_a;
        const K nb = bi < lb ? kb : x.next_b;
        next_is_a = has_na && (!has_nb || !key_gt_ck<CK>(na, nb, c));
        has_next = has_na || has_nb;
        next = next_is_a ? na : nb;
    }
    // last = output VT - 1.  eqn: output i equals output i + 1 (bits past
    // the valid outputs cleared).
    if (!has_prev) eqp &= ~1u;
    uint32_t eqn = (eqp >> 1) | ((uint32_t)(has_next && last == next) << (VT - 1));
    eqn &= valid >> 1 | (n_valid >= VT ? 1u << (VT - 1) : 0u);
    eqp = ((eqn << 1) | (eqp & 1u)) & all;
    const uint32_t ta_n = (took >> 1) | ((uint32_t)next_is_a << (VT - 1));
    const uint32_t ta_p = ((took << 1) | (uint32_t)prev_is_a) & all;
    const uint32_t partner_a = eqn & ~ta_n, slow_a = took & eqn & (ta_n | eqp);
    const uint32_t partner_b = eqp & ta_p, slow_b = ~took & eqp & ~ta_p & all;
    uint32_t keep, slow;
    switch (op) {
    case MP_SET_UNION:
        keep = took | ~partner_b;
        slow = slow_b;
        break;
    case MP_SET_INTERSECTION:
        keep = took & partner_a;
        slow = slow_a;
        break;
    case MP_SET_DIFFERENCE:
        keep = took & ~partner_a;
        slow = slow_a;
        break;
    default:
        keep = (took & ~partner_a) | (~took & ~partner_b);
        slow = slow_a | slow_b;
        break;
    }
    slow &= valid;
    while (slow) {
        const int i = __ffs(slow) - 1;
        slow &= slow - 1;
        const int na_i = __popc(took & ((1u << i) - 1));
        const bool from_a = (took >> i) & 1;
        const int ai_i = ai0 + na_i, bi_i = bi0 + (i - na_i);
        const K v = from_a ? sA[ai_i] : sB[bi_i];
        const bool kp = setop_exact(from_a, v, ai_i, bi_i, sA, la, sB, lb, op, x, a0, b0);
        keep = (keep & ~(1u << i)) | ((uint32_t)kp << i);
    }
    return keep & valid;
}

// Stage, split and walk with source indices (tiles with values).  Returns
// false (all threads) if the staging wait ran out.
template <class K, bool VALS, int NT, int VT, int CK>
__device__ __forceinline__ bool setop_tile_walk(const SetArgs<K>& p, int64_t tile, unsigned char* smem,
                                                unsigned int* err, TilePlace<K>& t,
                                                TileView<K, VALS, NT, VT>& v, uint32_t (&packed)[(VT + 1) / 2],
                                                uint32_t& keep)
{
    using SM = SetSmem<K, VALS, NT, VT>;
    constexpr int T = NT * VT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const BulkLayout<K, VALS, NT, VT, true> lay(smem);
    SetCtx<K>& x = *reinterpret_cast<SetCtx<K>*>(smem + SM::ctx_off);
    const TileArgs<K>& ta = p.t;
    t = tile_place(ta, tile, T, ta.a_split);
    v = stage_view<K, VALS, NT, VT>(t, lay.sk, lay.sv, lay.sidx);
    const int64_t a0 = t.gA - ta.a, b0 = t.gB - ta.b;
    const int64_t b1 = b0 + t.lb;
    bulk_init(lay.bar);
    __syncthreads();
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
        } else if (lane == 3) {
            const int64_t a1 = a0 + t.la;
            x.has_next_a = a1 < ta.na;
            if (a1 < ta.na) x.next_a = ld_global_nc(ta.a + a1);
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
    keep = setop_walk<K, VT, CK>(v.sA, t.la, v.sB, t.lb, ai, diag - ai, L - diag, p.op, x, a0, b0,
                                      ta.codec, packed);
    return true;
}

// ---------------------------------------------------------------------------
// Single pass: each tile's place in the result by a decoupled look-back over
// the tiles before it.  Tiles are taken in order from a counter (so every
// tile a CTA waits for has a CTA running it), each publishes its kept count
// as soon as it is known, then adds up its predecessors' published counts
// back to the nearest one that already holds its inclusive prefix, and
// publishes its own.  One 64-bit status word per tile: flag in the top two
// bits, count below.
// ---------------------------------------------------------------------------
#define MP_KERR_LOOKBACK 4u
constexpr unsigned long long LB_AGG = 1ull << 62, LB_INC = 2ull << 62, LB_VAL = (1ull << 62) - 1;
constexpr uint32_t LB_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Warp 0: the number of kept outputs in tiles [0, tile).  Each round reads
// the 32 nearest unread predecessors (lane l: tile base - l), waits until
// all of them have published, and adds them up back to the nearest
// inclusive prefix.  (Reading 128 per round measured slower.)  A wait that
// runs out (a predecessor never published: only after an earlier CTA
// stopped on a failed staging wait) sets MP_KERR_LOOKBACK and counts that
// tile as 0.
__device__ __forceinline__ unsigned long long lookback(unsigned long long* status, int64_t tile, int lane,
                                                       unsigned int* err)
{
    unsigned long long prefix = 0;
    int64_t base = tile - 1;
    while (base >= 0) {
        const int64_t idx = base - lane;
        unsigned long long v = idx >= 0 ? ld_relaxed_u64(status + idx) : LB_INC;  // before tile 0: 0
        uint32_t spins = 0;
        while (__any_sync(0xFFFFFFFFu, (v >> 62) == 0)) {
            if (++spins > LB_SPIN_LIMIT) {
                if (lane == 0) atomicOr(err, MP_KERR_LOOKBACK);
                if ((v >> 62) == 0) v = LB_AGG;  // counted as an empty tile
                break;
            }
            if ((v >> 62) == 0) v = ld_relaxed_u64(status + idx);
        }
        const uint32_t inc = __ballot_sync(0xFFFFFFFFu, (v >> 62) == 2);
        // Lanes up to the nearest inclusive prefix (lane 0 is the nearest tile).
        const int stop = inc ? __ffs(inc) - 1 : 31;
        unsigned long long x = (lane <= stop && idx >= 0) ? (v & LB_VAL) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
        prefix += x;
        if (inc) break;
        base -= 32;
    }
    return prefix;
}

// The set-operation tile kernel for tiles with values (one tile per CTA):
// take the next tile in order, stage it, walk and decide its outputs,
// publish its kept count and look back for its place, write the kept
// outputs and their values there.
template <class K, bool VALS, int NT, int VT, int CK>
__global__ void __launch_bounds__(NT, (sizeof(K) == 4 ? 1024 : 512) / NT)
    setop_kernel(SetArgs<K> p, unsigned int* err)
{
    using SM = SetSmem<K, VALS, NT, VT>;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long* scan = reinterpret_cast<unsigned long long*>(smem + SM::scan_off);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) scan[NW + 2] = atomicAdd(p.tile_counter, 1u);
    __syncthreads();
    const int64_t tile = (int64_t)scan[NW + 2];
    TilePlace<K> t;
    TileView<K, VALS, NT, VT> v;
    uint32_t keep = 0;
    static_assert(VALS, "tiles of keys alone run in setop_keys_kernel");
    uint32_t packed[(VT + 1) / 2];  // the outputs' sources
    if (!setop_tile_walk<K, VALS, NT, VT, CK>(p, tile, smem, err, t, v, packed, keep)) {
        // The tile stopped on a failed staging wait: publish it as empty so
        // that later tiles do not wait for it.
        if (tid == 0) st_relaxed_u64(p.status + tile, (tile == 0 ? LB_INC : LB_AGG));
        return;
    }
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
        wi = __shfl_sync(0xFFFFFFFFu, wi, 31);  // the tile's kept count
        if (lane == 0) {
            scan[NW] = wi;
            st_relaxed_u64(p.status + tile, (tile == 0 ? LB_INC : LB_AGG) | wi);
        }
        const unsigned long long pre = tile > 0 ? lookback(p.status, tile, lane, err) : 0ull;
        if (lane == 0) {
            if (tile > 0) st_relaxed_u64(p.status + tile, LB_INC | (pre + wi));
            scan[NW + 1] = pre;
        }
    }
    __syncthreads();
    const int64_t g = (int64_t)scan[NW + 1];
    const int n_out = (int)scan[NW];
    if (g < 0 || g + n_out > p.cap) {
        if (tid == 0) atomicOr(err, MP_KERR_SETOP);
        return;
    }
    const TileArgs<K>& ta = p.t;
    // Compact the kept sources into the index array (the staged windows
    // stay where they are; only indices move).
    uint16_t* sidx = v.sidx;
    int pos = (int)scan[warp] + incl - c;
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        if (keep & (1u << i)) sidx[pos++] = (uint16_t)((packed[i / 2] >> (16 * (i & 1))) & 0xFFFF);
    }
    __syncthreads();
    K* gout = ta.out + g;
    for (int j = tid; j < n_out; j += NT) {
        const int s = sidx[j];
        gout[j] = s < t.la ? v.sA[s] : v.sB[s - t.la];
    }
    uint32_t* gvout = ta.outv + g;
    for (int j = tid; j < n_out; j += NT) {
        const int s = sidx[j];
        gvout[j] = s < t.la ? v.vA[s] : v.vB[s - t.la];
    }
    if (tid == 0 && tile == p.ntiles - 1) *p.count = g + n_out;
}

// ---------------------------------------------------------------------------
// Persistent set-operation kernel for keys alone.  Each CTA runs tiles of
// the single pass through a ring of three shared-memory buffers, with three
// warp roles working on different tiles at once:
//   stager  (one warp): takes the next tile from the counter, and once a
//           buffer is free starts the TMA copies of the tile's windows into
//           it and loads the keys next to the windows;
//   walkers (NT threads): wait for a staged tile, split it (Thm 17), walk
//           and decide its outputs, publish its kept count, compact the kept
//           keys over the windows of the same buffer (which the walk no
//           longer needs), then write the previous tile's compacted keys to
//           the offset the look-back warp has found meanwhile, and free
//           that buffer;
//   look-back (one warp): for each walked tile, adds up the published
//           counts of the tiles before it (decoupled look-back) and
//           publishes its inclusive prefix.
// So the copies of later tiles and the look-back of the last one overlap the
// walk, where a CTA per tile waited for each in turn.  Hand-offs are
// mbarriers, one set per buffer (the k-th tile uses buffer k % 3 and waits
// for phase parity (k / 3) & 1); every wait is bounded.  Walkers synchronise
// among themselves with named barrier 1 only.
// ---------------------------------------------------------------------------
template <class K>
struct __align__(16) PSetInfo {
    TilePlace<K> t;
    SetCtx<K> x;
    int64_t tile;  // -1: no more tiles
};

constexpr int PSET_NB = 3;  // buffers in the ring

template <class K, int NT, int VT>
struct PSetSmem {
    static constexpr int T = NT * VT;
    static constexpr int EK = 16 / sizeof(K);
    // Windows (at their 16-byte phases), then spare slots: the end-test-free
    // walk reads up to VT + 1 past its start.  The compacted output (<= T
    // keys) later takes the buffer from its start; its store reads up to two
    // words past its end.
    static constexpr int SLACK = VT + 1;
    static constexpr size_t buf_bytes = ((size_t)(T + 3 * EK + SLACK) * sizeof(K) + 15) / 16 * 16;
    static constexpr size_t info_off = PSET_NB * buf_bytes;
    static constexpr size_t info_bytes = (sizeof(PSetInfo<K>) + 15) / 16 * 16;
    static constexpr size_t scan_off = info_off + PSET_NB * info_bytes;
    static constexpr size_t split_off = scan_off + (NT / 32) * 8;
    static constexpr size_t slot_off = split_off + NT * 4;  // per buffer: {tile, kept, prefix}
    static constexpr size_t bar_off = slot_off + PSET_NB * 24;
    static constexpr size_t bytes = bar_off + 4 * PSET_NB * 8;  // full, walked, placed, freed [NB]
};

constexpr uint32_t PSET_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t tx)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(tx)
                 : "memory");
}

// Named barrier 1 over the NT walker threads.
template <int NT>
__device__ __forceinline__ void walker_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

template <int NT>
__device__ __forceinline__ bool walker_sync_and(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred a, b;\n\t"
        "setp.ne.u32 a, %1, 0;\n\t"
        "bar.red.and.pred b, 1, %2, a;\n\t"
        "selp.u32 %0, 1, 0, b;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(NT)
        : "memory");
    return r != 0;
}

// Copies nw 32-bit words from shared memory (16-byte aligned) to global
// memory at any 4-byte phase: whole 16-byte vectors assembled from two
// aligned shared vectors, the partial vectors at both ends word by word.
// Reads up to two words past nw.
template <int NT>
__device__ __forceinline__ void store_words_shifted(const uint32_t* so, int nw, uint32_t* gw, int tid)
{
    const int pw = (int)(((uintptr_t)gw >> 2) & 3);
    uint32_t* gbase = gw - pw;  // 16-byte aligned
    const int end = pw + nw;
    const int q0 = pw ? 1 : 0, q1 = end >> 2;  // whole vectors [q0, q1) of gbase
    if (pw == 0) {
        for (int q = tid; q < q1; q += NT)
            st_global_cs_v4(gbase + 4 * q, *reinterpret_cast<const uint4*>(so + 4 * q));
    } else {
        for (int q = q0 + tid; q < q1; q += NT) {
            // Global word 4q is local word 4q - pw.
            const uint4 a = *reinterpret_cast<const uint4*>(so + 4 * q - 4);
            const uint4 c = *reinterpret_cast<const uint4*>(so + 4 * q);
            uint4 r;
            if (pw == 1) r = make_uint4(a.w, c.x, c.y, c.z);
            else if (pw == 2) r = make_uint4(a.z, a.w, c.x, c.y);
            else r = make_uint4(a.y, a.z, a.w, c.x);
            st_global_cs_v4(gbase + 4 * q, r);
        }
    }
    const int head_end = 4 * q0 < end ? 4 * q0 : end;
    if (tid < head_end - pw) gbase[pw + tid] = so[tid];
    const int tail0 = 4 * q1 > head_end ? 4 * q1 : head_end;
    if (tid < end - tail0) gbase[tail0 + tid] = so[tail0 - pw + tid];
}

template <class K, int NT, int VT>
struct PSetView {
    unsigned char* smem;
    __device__ __forceinline__ K* buf(int b) const
    {
        return reinterpret_cast<K*>(smem + b * PSetSmem<K, NT, VT>::buf_bytes);
    }
    __device__ __forceinline__ PSetInfo<K>& info(int b) const
    {
        return *reinterpret_cast<PSetInfo<K>*>(smem + PSetSmem<K, NT, VT>::info_off +
                                                b * PSetSmem<K, NT, VT>::info_bytes);
    }
    // set 0 full (stager -> walkers), 1 walked (walkers -> look-back),
    // 2 placed (look-back -> walkers), 3 freed (walkers -> stager)
    __device__ __forceinline__ uint64_t* bar(int set, int b) const
    {
        return reinterpret_cast<uint64_t*>(smem + PSetSmem<K, NT, VT>::bar_off) + set * PSET_NB + b;
    }
    __device__ __forceinline__ int64_t* slot(int b) const
    {
        return reinterpret_cast<int64_t*>(smem + PSetSmem<K, NT, VT>::slot_off) + 3 * b;
    }
};

// Stager: the ring position k's tile (taken before its buffer is free, so
// its split points are loaded while waiting).
template <class K, int NT, int VT>
__device__ __forceinline__ void pset_stager(const SetArgs<K>& p, unsigned char* smem, unsigned int* err)
{
    using SM = PSetSmem<K, NT, VT>;
    constexpr int EK = 16 / sizeof(K);
    const PSetView<K, NT, VT> sv{smem};
    const int lane = threadIdx.x & 31;
    const TileArgs<K>& ta = p.t;
    for (int k = 0;; ++k) {
        const int b = k % PSET_NB;
        unsigned int tk = 0;
        if (lane == 0) tk = atomicAdd(p.tile_counter, 1u);
        const int64_t tile = (int64_t)__shfl_sync(0xFFFFFFFFu, tk, 0);
        const bool last = tile >= p.ntiles;
        TilePlace<K> t;
        if (!last) t = tile_place(ta, tile, SM::T, ta.a_split);
        if (k >= PSET_NB &&
            !mbar_wait_bounded(sv.bar(3, b), ((k - PSET_NB) / PSET_NB) & 1, PSET_WAIT_LIMIT)) {
            // The buffer was never freed: stop staging.
            if (lane == 0) atomicOr(err, MP_KERR_MBAR_TIMEOUT);
            return;
        }
        PSetInfo<K>& in = sv.info(b);
        uint64_t* full = sv.bar(0, b);
        if (last) {
            if (lane == 0) in.tile = -1;
            mbar_arrive(full);
            return;
        }
        const auto v = stage_view<K, false, NT, VT>(t, sv.buf(b), nullptr, nullptr);
        if (lane == 0) {
            in.tile = tile;
            in.t = t;
            mbar_expect_tx(full, interior_bytes(t.gA, t.la) + interior_bytes(t.gB, t.lb));
            issue_interior(v.sA, t.gA, t.la, full);
            issue_interior(v.sB, t.gB, t.lb, full);
        }
        if (lane < 4 * EK) {
            const EdgeLoad<K> e = edge_load(lane, t.gA, t.la, t.gB, t.lb);
            if (e.dst >= 0) (e.in_b ? v.sB : v.sA)[e.dst] = e.val;
        }
        // The keys just outside the windows.
        const int64_t a0 = t.gA - ta.a, b0 = t.gB - ta.b, a1 = a0 + t.la, b1 = b0 + t.lb;
        SetCtx<K>& x = in.x;
        if (lane == 28) {
            x.has_prev_a = a0 > 0;
            if (a0 > 0) x.prev_a = ld_global_nc(ta.a + a0 - 1);
        } else if (lane == 29) {
            x.has_prev_b = b0 > 0;
            if (b0 > 0) x.prev_b = ld_global_nc(ta.b + b0 - 1);
        } else if (lane == 30) {
            x.has_next_b = b1 < ta.nb;
            if (b1 < ta.nb) x.next_b = ld_global_nc(ta.b + b1);
        } else if (lane == 31) {
            x.has_next_a = a1 < ta.na;
            if (a1 < ta.na) x.next_a = ld_global_nc(ta.a + a1);
        }
        mbar_arrive(full);  // every lane: its writes are released with the phase
    }
}

// Look-back warp: the place of each walked tile.
template <class K, int NT, int VT>
__device__ __forceinline__ void pset_lookback(const SetArgs<K>& p, unsigned char* smem, unsigned int* err)
{
    const PSetView<K, NT, VT> sv{smem};
    const int lane = threadIdx.x & 31;
    for (int k = 0;; ++k) {
        const int b = k % PSET_NB;
        if (!mbar_wait_bounded(sv.bar(1, b), (k / PSET_NB) & 1, PSET_WAIT_LIMIT)) {
            if (lane == 0) atomicOr(err, MP_KERR_MBAR_TIMEOUT);
            return;
        }
        const int64_t tile = sv.slot(b)[0], n = sv.slot(b)[1];
        if (tile < 0) return;
        const unsigned long long pre = tile > 0 ? lookback(p.status, tile, lane, err) : 0ull;
        if (lane == 0) {
            if (tile > 0) st_relaxed_u64(p.status + tile, LB_INC | (pre + (unsigned long long)n));
            if (tile == p.ntiles - 1) *p.count = (int64_t)pre + n;
            sv.slot(b)[2] = (int64_t)pre;
            mbar_arrive(sv.bar(2, b));
        }
        __syncwarp();
    }
}

// Walkers: tile j's compacted keys leave for their place (once the
// look-back warp has found it) and its buffer is freed.
template <class K, int NT, int VT>
__device__ __forceinline__ void pset_place(const SetArgs<K>& p, const PSetView<K, NT, VT>& sv, int j,
                                           unsigned int* err, int tid)
{
    constexpr int WPK = (int)sizeof(K) / 4;  // 32-bit words per key
    const int b = j % PSET_NB;
    if (walker_sync_and<NT>(mbar_wait_bounded(sv.bar(2, b), (j / PSET_NB) & 1, PSET_WAIT_LIMIT))) {
        const int64_t g = sv.slot(b)[2], n = sv.slot(b)[1];
        if (g + n > p.cap) {
            if (tid == 0) atomicOr(err, MP_KERR_SETOP);
        } else {
            store_words_shifted<NT>(reinterpret_cast<const uint32_t*>(sv.buf(b)), (int)n * WPK,
                                    reinterpret_cast<uint32_t*>(p.t.out + g), tid);
        }
    } else if (tid == 0) {
        atomicOr(err, MP_KERR_LOOKBACK);
    }
    mbar_arrive(sv.bar(3, b));  // every walker, after its reads of the buffer
}

template <class K, int NT, int VT, int CK>
__device__ __forceinline__ void pset_walkers(const SetArgs<K>& p, unsigned char* smem, unsigned int* err)
{
    using SM = PSetSmem<K, NT, VT>;
    constexpr int NW = NT / 32;
    const PSetView<K, NT, VT> sv{smem};
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long* scan = reinterpret_cast<unsigned long long*>(smem + SM::scan_off);
    int* split = reinterpret_cast<int*>(smem + SM::split_off);
    const TileArgs<K>& ta = p.t;
    // err[1]: the staging-wait fault switch (see bulk_stage).
    const uint32_t first_limit = __ldcg(err + 1) ? 0u : PSET_WAIT_LIMIT;
    int k = 0;
    for (;; ++k) {
        const int b = k % PSET_NB;
        const uint32_t par = (k / PSET_NB) & 1;
        const bool ok = walker_sync_and<NT>(mbar_wait_bounded(sv.bar(0, b), par, first_limit));
        if (!ok) {
            if (tid == 0) atomicOr(err, MP_KERR_MBAR_TIMEOUT);
            // Give copies in flight a bounded time to land; if they do not,
            // stop here (the tile, if any, is never published).
            if (!walker_sync_and<NT>(mbar_wait_bounded(sv.bar(0, b), par, PSET_WAIT_LIMIT))) break;
        }
        PSetInfo<K>& in = sv.info(b);
        const int64_t tile = in.tile;
        if (tile < 0) break;
        const TilePlace<K> t = in.t;
        SetCtx<K>& x = in.x;
        K keys[VT];
        uint32_t keep = 0;
        if (ok) {  // a tile whose staging wait failed is published as empty
            const auto v = stage_view<K, false, NT, VT>(t, sv.buf(b), nullptr, nullptr);
            const int64_t a0 = t.gA - ta.a, b0 = t.gB - ta.b, b1 = b0 + t.lb;
            const int la = t.la, lb = t.lb, L = la + lb;
            // Runs crossing a window edge (as in setop_tile_walk).
            const bool b0_rep =
                lb > 0 && ((lb > 1 && v.sB[1] == v.sB[0]) || (x.has_prev_b && x.prev_b == v.sB[0]));
            const bool a_end_rep = la > 0 && ((la > 1 && v.sA[la - 2] == v.sA[la - 1]) ||
                                              (la == 1 && x.has_prev_a && x.prev_a == v.sA[0]));
            const bool need_a =
                x.has_prev_a && ((la > 0 && v.sA[0] == x.prev_a) || (b0_rep && v.sB[0] == x.prev_a));
            const bool need_b = x.has_prev_b && lb > 0 && v.sB[0] == x.prev_b;
            const bool need_n = x.has_next_b &&
                                ((lb > 0 && v.sB[lb - 1] == x.next_b) || (a_end_rep && v.sA[la - 1] == x.next_b));
            if (need_a || need_b || need_n) {
                if (warp == 3) {
                    if (lane == 0 && need_a) x.lb_prev_a = run_start(ta.a, a0 - 1);
                    if (lane == 1 && need_b) x.lb_prev_b = run_start(ta.b, b0 - 1);
                    if (lane == 2 && need_n) x.ub_next_b = run_end(ta.b, ta.nb, b1);
                }
                walker_sync<NT>();
            }
            const int diag = tid * VT < L ? tid * VT : L;
            const int ai = smem_diagonal_search_ck<CK>(v.sA, la, v.sB, lb, diag, ta.codec);
            split[tid] = ai;
            walker_sync<NT>();
            const int dend = diag + VT;
            const int ai_end = tid + 1 < NT ? split[tid + 1] : la;
            const bool inside = dend < L && ai_end < la && dend - ai_end < lb;
            keep = setop_walk_keys<K, VT, CK>(v.sA, la, v.sB, lb, ai, diag - ai, L - diag, inside, p.op,
                                                     x, a0, b0, ta.codec, keys);
        }
        const int c = __popc(keep);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) scan[warp] = (unsigned long long)incl;
        walker_sync<NT>();  // every walk is done (the windows are dead); warp totals visible
        // Every warp scans the warp totals itself.
        const unsigned long long w = lane < NW ? scan[lane] : 0;
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        const unsigned long long total = __shfl_sync(0xFFFFFFFFu, wi, NW - 1);
        const int base = (int)__shfl_sync(0xFFFFFFFFu, wi - w, warp);
        if (tid == 0) {
            st_relaxed_u64(p.status + tile, (tile == 0 ? LB_INC : LB_AGG) | total);
            sv.slot(b)[0] = tile;
            sv.slot(b)[1] = (int64_t)total;
            mbar_arrive(sv.bar(1, b));
        }
        // The kept keys replace the windows, from the buffer's start.
        K* so = sv.buf(b);
        int pos = base + incl - c;
#pragma unroll
        for (int i = 0; i < VT; ++i) {
            if (keep & (1u << i)) so[pos++] = keys[i];
        }
        if (k > 0) pset_place<K, NT, VT>(p, sv, k - 1, err, tid);
    }
    // No more tiles (or a failed copy): release the look-back warp, place
    // the last tile.
    if (tid == 0) {
        sv.slot(k % PSET_NB)[0] = -1;
        mbar_arrive(sv.bar(1, k % PSET_NB));
    }
    if (k > 0) pset_place<K, NT, VT>(p, sv, k - 1, err, tid);
}

template <class K, int NT, int VT, int CK, int MINB>
__global__ void __launch_bounds__(NT + 64, MINB) setop_keys_kernel(SetArgs<K> p, unsigned int* err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    if (threadIdx.x == 0) {
        const PSetView<K, NT, VT> sv{smem};
        for (int b = 0; b < PSET_NB; ++b) {
            mbar_init(sv.bar(0, b), 32);  // full: the stager's lanes (+ the copies' bytes)
            mbar_init(sv.bar(1, b), 1);   // walked: walker 0, with the tile's kept count
            mbar_init(sv.bar(2, b), 1);   // placed: look-back lane 0, with the prefix
            mbar_init(sv.bar(3, b), NT);  // freed: every walker, after the store
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int warp = threadIdx.x >> 5;
    if (warp < NT / 32)
        pset_walkers<K, NT, VT, CK>(p, smem, err);
    else if (warp == NT / 32)
        pset_stager<K, NT, VT>(p, smem, err);
    else
        pset_lookback<K, NT, VT>(p, smem, err);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
// Tile shape per mode.  Items per thread: one bit each in the walk's masks,
// so at most 32; an odd count starts the threads' walks in different
// shared-memory banks.  Tiles with values (one per CTA): 256 threads x 27
// outputs for 4-byte keys (1.28 ms for the union of two 2^27-key sets
// against 1.57 with 512 threads), 15 for 8-byte keys, 8 for 16-byte keys.
// Keys alone (the persistent kernel; its three buffers of a tile each, two
// CTAs per SM, bound the tile): 320 walkers x 27 for 4-byte keys (uint32
// union 0.661 ms; 352 x 25: 0.669; 384 x 23: 0.676; 416 x 21, spilling:
// 0.772; 256 x 31: 0.687; 512 x 31 with one CTA per SM: 0.710), 256 x 15
// for 8-byte and 256 x 8 for 16-byte keys.
constexpr int set_vt(int key_bytes, bool /* vals: the same counts with and without */)
{
    return key_bytes == 4 ? 27 : (key_bytes == 8 ? 15 : 8);
}

constexpr int set_nt(int key_bytes, bool vals) { return vals ? 256 : (key_bytes == 4 ? 320 : 256); }
constexpr int PSET_MINB = 2;  // persistent keys-alone kernel: CTAs per SM

int64_t setop_tile(int key_bytes, bool vals) { return (int64_t)set_nt(key_bytes, vals) * set_vt(key_bytes, vals); }

template <class K, bool VALS, int CK>
static cudaError_t launch_setop_ck(const MergeProblem& mp_, int op, const int64_t* splits,
                                   unsigned long long* status, unsigned int* tile_counter, int64_t cap,
                                   int64_t* count, cudaStream_t stream)
{
    constexpr int VT = set_vt((int)sizeof(K), VALS);
    constexpr int NT = set_nt((int)sizeof(K), VALS);
    constexpr size_t smem_bytes = VALS ? SetSmem<K, VALS, NT, VT>::bytes : PSetSmem<K, NT, VT>::bytes;
    void (*kern)(SetArgs<K>, unsigned int*);
    if constexpr (VALS)
        kern = setop_kernel<K, VALS, NT, VT, CK>;
    else
        kern = setop_keys_kernel<K, NT, VT, CK, PSET_MINB>;
    static int resident = 0;  // CTAs per SM x SMs (persistent kernel)
    if (!resident) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, VALS ? NT : NT + 64, smem_bytes);
        if (e != cudaSuccess) return e;
        resident = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
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
    a.status = status;
    a.tile_counter = tile_counter;
    a.count = count;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(VALS ? a.ntiles : std::min<int64_t>(a.ntiles, resident)));
    cfg.blockDim = dim3(VALS ? NT : NT + 64);
    cfg.dynamicSmemBytes = smem_bytes;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, err);
}

template <class K, bool VALS>
static cudaError_t launch_setop_t(const MergeProblem& p, int op, const int64_t* splits,
                                  unsigned long long* status, unsigned int* tile_counter, int64_t cap,
                                  int64_t* count, cudaStream_t stream)
{
    if (p.kind.identity())
        return launch_setop_ck<K, VALS, CODEC_IDENTITY>(p, op, splits, status, tile_counter, cap, count, stream);
    if (p.kind.signed_int())
        return launch_setop_ck<K, VALS, CODEC_SIGNED>(p, op, splits, status, tile_counter, cap, count, stream);
    return launch_setop_ck<K, VALS, CODEC_RUNTIME>(p, op, splits, status, tile_counter, cap, count, stream);
}

cudaError_t launch_setop(const MergeProblem& p, int op, const int64_t* splits, unsigned long long* status,
                         unsigned int* tile_counter, int64_t cap, int64_t* count, cudaStream_t stream)
{
    if (p.kind.bytes == 4)
        return p.vals ? launch_setop_t<uint32_t, true>(p, op, splits, status, tile_counter, cap, count, stream)
                      : launch_setop_t<uint32_t, false>(p, op, splits, status, tile_counter, cap, count, stream);
    if (p.kind.bytes == 16)
        return p.vals ? launch_setop_t<u128, true>(p, op, splits, status, tile_counter, cap, count, stream)
                      : launch_setop_t<u128, false>(p, op, splits, status, tile_counter, cap, count, stream);
    return p.vals ? launch_setop_t<uint64_t, true>(p, op, splits, status, tile_counter, cap, count, stream)
                  : launch_setop_t<uint64_t, false>(p, op, splits, status, tile_counter, cap, count, stream);
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
    MP_RANGE("mp_set_operation");
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
    const size_t status_bytes = (size_t)ntiles * 8;
    unsigned char* scratch = nullptr;
    st = scratch_alloc((void**)&scratch, split_bytes + status_bytes + 16, s);
    if (st != MP_OK) return st;
    int64_t* splits = reinterpret_cast<int64_t*>(scratch);
    unsigned long long* status = reinterpret_cast<unsigned long long*>(scratch + split_bytes);
    unsigned int* tile_counter = reinterpret_cast<unsigned int*>(scratch + split_bytes + status_bytes);
    // The look-back words and the tile counter start at zero.
    cudaError_t e = cudaMemsetAsync(status, 0, status_bytes + 16, s);
    if (e == cudaSuccess) e = launch_partition(p, T, splits, s);
    if (e == cudaSuccess) e = launch_setop(p, (int)op, splits, status, tile_counter, cap, out_count, s);
    scratch_free(scratch, s);
    return e == cudaSuccess ? MP_OK : cuda_fail(e, fn);
}

}  // extern "C"
