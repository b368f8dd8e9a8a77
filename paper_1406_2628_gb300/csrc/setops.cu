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
//   3. count-then-scatter in one pass: a block scan of the kept counts gives
//      each output its place in the tile, a decoupled look-back over the
//      tiles' published counts gives the tile's place in the result, and the
//      kept outputs are gathered and written contiguously.
// Tiles take their index from an atomic counter, so every tile a CTA looks
// back on is already held by a running CTA; the look-back waits are bounded.
#include <algorithm>

#include "mp_bulk.cuh"
#include "mp_device.cuh"
#include "mp_internal.h"
#include "mp_tile.cuh"

namespace mp {

// Bit set in the kernel error word when a set operation's look-back gave up
// or its output would pass the capacity (inputs not sorted).
#define MP_KERR_SETOP 2u

template <class K>
struct SetArgs {
    TileArgs<K> t;               // the merge problem (run == 0) and split points
    int op;                      // MP_SET_*
    int64_t ntiles;
    int64_t cap;                 // output capacity (elements)
    unsigned long long* status;  // per tile: flag (top 2 bits) | count
    unsigned int* tile_counter;  // [0]: next tile, [1]: abort flag of this launch
    int64_t* count;              // result length (device)
};

constexpr unsigned long long ST_AGG = 1ull << 62;   // tile count published
constexpr unsigned long long ST_PRE = 2ull << 62;   // inclusive prefix published
constexpr unsigned long long ST_VAL = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

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

// Walk VT outputs of the tile's merge from split (ai, bi) and decide each:
// records sources (A: 0..la-1, B: la..) and a bit mask of kept outputs.
template <class K, int VT, int CK>
__device__ __forceinline__ uint32_t setop_walk(const K* sA, int la, const K* sB, int lb, int ai, int bi,
                                               int n_valid, int op, const SetCtx<K>& x, int64_t a0,
                                               int64_t b0, Codec<K> c, uint32_t (&packed)[VT / 2])
{
    const bool keep_a_alone = op != MP_SET_INTERSECTION;
    const bool keep_b_alone = op == MP_SET_UNION || op == MP_SET_SYMMETRIC_DIFFERENCE;
    K ra = sA[ai], rb = sB[bi];
    K ka = key_enc_ck<CK>(ra, c), kb = key_enc_ck<CK>(rb, c);
    bool last_a_ok = ai > 0 || x.has_prev_a;
    K last_a = ai > 0 ? sA[ai - 1] : x.prev_a;
    bool last_b_ok = bi > 0 || x.has_prev_b;
    K last_b = bi > 0 ? sB[bi - 1] : x.prev_b;
    uint32_t keep = 0;
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        const bool take_a = (bi >= lb) || (ai < la && !(ka > kb));
        bool kp = false;
        if (take_a) {
            const K v = ra;
            if (i < n_valid) {
                // The B pointer is where v's run in B starts (ties take A).
                const bool match_b = bi < lb ? rb == v : (x.has_next_b && x.next_b == v);
                if (!match_b || op == MP_SET_UNION) {
                    kp = keep_a_alone;
                } else {
                    // Rank of this copy in A's run of v.
                    int64_t r_a = 0;
                    if (last_a_ok && last_a == v) {
                        const int f = first_equal(sA, 0, ai, v);
                        const int64_t start = (f == 0 && x.has_prev_a && x.prev_a == v) ? x.lb_prev_a : a0 + f;
                        r_a = a0 + ai - start;
                    }
                    // Length of v's run in B (from b0 + bi).
                    int64_t end;
                    if (bi >= lb) {
                        end = x.ub_next_b;
                    } else if (bi + 1 < lb && sB[bi + 1] != v) {
                        end = b0 + bi + 1;
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
                    kp = op == MP_SET_INTERSECTION ? r_a < n : r_a >= n;
                }
            }
            const uint32_t src = (uint32_t)ai;
            if (i & 1) packed[i / 2] |= src << 16;
            else packed[i / 2] = src;
            last_a = v;
            last_a_ok = true;
            ++ai;
            ra = sA[ai < la ? ai : la];
            ka = key_enc_ck<CK>(ra, c);
        } else {
            const K v = rb;
            if (i < n_valid && keep_b_alone) {
                // The A pointer is one past v's run in A.
                const bool match_a = last_a_ok && last_a == v;
                if (!match_a) {
                    kp = true;
                } else {
                    int64_t start;
                    if (ai == 0) {
                        start = x.lb_prev_a;
                    } else if (ai >= 2 && sA[ai - 2] != v) {
                        start = a0 + ai - 1;
                    } else {
                        const int f = first_equal(sA, 0, ai - 1, v);
                        start = (f == 0 && x.has_prev_a && x.prev_a == v) ? x.lb_prev_a : a0 + f;
                    }
                    const int64_t m = a0 + ai - start;
                    int64_t r_b = 0;
                    if (last_b_ok && last_b == v) {
                        const int f = first_equal(sB, 0, bi, v);
                        const int64_t bs = (f == 0 && x.has_prev_b && x.prev_b == v) ? x.lb_prev_b : b0 + f;
                        r_b = b0 + bi - bs;
                    }
                    kp = r_b >= m;
                }
            }
            const uint32_t src = (uint32_t)(la + bi);
            if (i & 1) packed[i / 2] |= src << 16;
            else packed[i / 2] = src;
            last_b = v;
            last_b_ok = true;
            ++bi;
            rb = sB[bi];
            kb = key_enc_ck<CK>(rb, c);
        }
        if (kp) keep |= 1u << i;
    }
    return keep;
}

// Exclusive prefix of this tile's count over all earlier tiles (warp 0).
// Returns false if a wait ran out.
__device__ __forceinline__ bool look_back(unsigned long long* status, int64_t tile, unsigned long long count,
                                          const unsigned int* abort_flag, unsigned long long* excl_out)
{
    constexpr uint32_t SPIN_LIMIT = 1u << 20;
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_release_u64(&status[0], ST_PRE | count);
        *excl_out = 0;
        return true;
    }
    if (lane == 0) st_release_u64(&status[tile], ST_AGG | count);
    unsigned long long excl = 0;
    int64_t q = tile - 1;
    bool ok = true;
    while (true) {
        const int64_t idx = q - lane;
        unsigned long long w = ST_PRE;  // before tile 0: a zero prefix
        if (idx >= 0) {
            w = ld_acquire_u64(&status[idx]);
            uint32_t spins = 0;
            while ((w >> 62) == 0) {
                // Give up after the limit, or early once a CTA of this
                // launch has failed (a failed tile never publishes).
                if (++spins > SPIN_LIMIT || (spins % 1024 == 0 && *(volatile const unsigned int*)abort_flag != 0))
                    break;
                __nanosleep(64);
                w = ld_acquire_u64(&status[idx]);
            }
        }
        if (__any_sync(0xFFFFFFFFu, (w >> 62) == 0)) {
            ok = false;
            break;
        }
        const unsigned pre = __ballot_sync(0xFFFFFFFFu, (w >> 62) == 2);
        const int first = pre ? __ffs(pre) - 1 : 31;  // nearest published prefix
        unsigned long long v = lane <= first ? (w & ST_VAL) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        excl += v;
        if (pre) break;
        q -= 32;
    }
    if (ok && lane == 0) st_release_u64(&status[tile], ST_PRE | (excl + count));
    *excl_out = excl;
    return ok;
}

template <class K, bool VALS, int NT, int VT, int CK>
__global__ void __launch_bounds__(NT, 2) setop_kernel(SetArgs<K> p, unsigned int* err)
{
    using SM = SetSmem<K, VALS, NT, VT>;
    constexpr int T = NT * VT;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    const BulkLayout<K, VALS, NT, VT> lay(smem);
    SetCtx<K>& x = *reinterpret_cast<SetCtx<K>*>(smem + SM::ctx_off);
    unsigned long long* scan = reinterpret_cast<unsigned long long*>(smem + SM::scan_off);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (tid == 0) scan[NW + 2] = atomicAdd(p.tile_counter, 1u);
    bulk_init(lay.bar);
    __syncthreads();
    const int64_t tile = (int64_t)scan[NW + 2];
    if (tile >= p.ntiles) return;  // uniform

    const TileArgs<K>& ta = p.t;
    const TilePlace<K> t = tile_place(ta, tile, T, ta.a_split);
    const auto v = stage_view<K, VALS, NT, VT>(t, lay.sk, lay.sv, lay.sidx);
    const int64_t a0 = t.gA - ta.a, b0 = t.gB - ta.b;
    const int64_t b1 = b0 + t.lb;
    if (warp == 3) {  // edge runs, in global memory, while the copies fly
        if (lane == 0) {
            x.has_prev_a = a0 > 0;
            if (a0 > 0) {
                x.prev_a = ta.a[a0 - 1];
                x.lb_prev_a = run_start(ta.a, a0 - 1);
            }
        } else if (lane == 1) {
            x.has_prev_b = b0 > 0;
            if (b0 > 0) {
                x.prev_b = ta.b[b0 - 1];
                x.lb_prev_b = run_start(ta.b, b0 - 1);
            }
        } else if (lane == 2) {
            x.has_next_b = b1 < ta.nb;
            if (b1 < ta.nb) {
                x.next_b = ta.b[b1];
                x.ub_next_b = run_end(ta.b, ta.nb, b1);
            }
        }
    }
    if (!bulk_stage<K, VALS, NT, VT>(t, v, lay.bar, 0, err)) {  // (the barrier also publishes x)
        if (tid == 0) atomicExch(p.tile_counter + 1, 1u);
        return;
    }

    // Merge walk with decisions.
    const int L = t.la + t.lb;
    const int diag = tid * VT < L ? tid * VT : L;
    const int ai = smem_diagonal_search_ck<CK>(v.sA, t.la, v.sB, t.lb, diag, ta.codec);
    uint32_t packed[VT / 2];
    const uint32_t keep = setop_walk<K, VT, CK>(v.sA, t.la, v.sB, t.lb, ai, diag - ai, L - diag, p.op, x, a0,
                                                b0, ta.codec, packed);

    // Block scan of the kept counts.
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
        unsigned long long w = lane < NW ? scan[lane] : 0;
        unsigned long long wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += y;
        }
        const unsigned long long total = __shfl_sync(0xFFFFFFFFu, wi, 31);
        unsigned long long g = 0;
        const bool ok = look_back(p.status, tile, total, p.tile_counter + 1, &g);
        if (lane < NW) scan[lane] = wi - w;  // exclusive warp offsets
        if (lane == 0) {
            scan[NW] = total;
            scan[NW + 1] = ok ? g : ~0ull;
        }
    }
    __syncthreads();
    const unsigned long long total = scan[NW];
    const unsigned long long g = scan[NW + 1];
    if (g == ~0ull || g + total > (unsigned long long)p.cap) {
        if (tid == 0) {
            atomicOr(err, MP_KERR_SETOP);
            atomicExch(p.tile_counter + 1, 1u);
        }
        return;
    }
    // Compact the kept sources into the index array (positions in the tile's
    // share of the result).
    int pos = (int)scan[warp] + incl - c;
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        if (keep & (1u << i)) lay.sidx[pos++] = (uint16_t)((packed[i / 2] >> (16 * (i & 1))) & 0xFFFF);
    }
    __syncthreads();
    const int n_out = (int)total;
    K* gout = ta.out + g;
    for (int j = tid; j < n_out; j += NT) {
        const int s = lay.sidx[j];
        gout[j] = s < t.la ? v.sA[s] : v.sB[s - t.la];
    }
    if constexpr (VALS) {
        uint32_t* gvout = ta.outv + g;
        for (int j = tid; j < n_out; j += NT) {
            const int s = lay.sidx[j];
            gvout[j] = s < t.la ? v.vA[s] : v.vB[s - t.la];
        }
    }
    if (tile == p.ntiles - 1 && tid == 0) *p.count = (int64_t)(g + total);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
constexpr int SET_NT = 256;
constexpr int SET_VT = 8;

int64_t setop_tile() { return (int64_t)SET_NT * SET_VT; }

template <class K, bool VALS, int CK>
static cudaError_t launch_setop_ck(const MergeProblem& mp_, int op, const int64_t* splits,
                                   unsigned long long* status, unsigned int* counter, int64_t cap,
                                   int64_t* count, cudaStream_t stream)
{
    using SM = SetSmem<K, VALS, SET_NT, SET_VT>;
    auto kern = setop_kernel<K, VALS, SET_NT, SET_VT, CK>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
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
    t.codec.flip = (K)mp_.kind.flip;
    t.codec.fmask = (K)mp_.kind.fmask;
    t.codec.inv = (K)mp_.kind.inv;
    a.op = op;
    a.ntiles = ceil_div(t.total, setop_tile());
    a.cap = cap;
    a.status = status;
    a.tile_counter = counter;
    a.count = count;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.ntiles);
    cfg.blockDim = dim3(SET_NT);
    cfg.dynamicSmemBytes = SM::bytes;
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
                                  unsigned long long* status, unsigned int* counter, int64_t cap, int64_t* count,
                                  cudaStream_t stream)
{
    if (p.kind.identity())
        return launch_setop_ck<K, VALS, CODEC_IDENTITY>(p, op, splits, status, counter, cap, count, stream);
    return launch_setop_ck<K, VALS, CODEC_RUNTIME>(p, op, splits, status, counter, cap, count, stream);
}

cudaError_t launch_setop(const MergeProblem& p, int op, const int64_t* splits, unsigned long long* status,
                         unsigned int* counter, int64_t cap, int64_t* count, cudaStream_t stream)
{
    if (p.kind.bytes == 4)
        return p.vals ? launch_setop_t<uint32_t, true>(p, op, splits, status, counter, cap, count, stream)
                      : launch_setop_t<uint32_t, false>(p, op, splits, status, counter, cap, count, stream);
    return p.vals ? launch_setop_t<uint64_t, true>(p, op, splits, status, counter, cap, count, stream)
                  : launch_setop_t<uint64_t, false>(p, op, splits, status, counter, cap, count, stream);
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
    const int64_t T = setop_tile();
    const int64_t ntiles = ceil_div(na + nb, T);
    const size_t split_bytes = (size_t)(ntiles + 1) * 8;
    const size_t status_bytes = (size_t)ntiles * 8;
    unsigned char* scratch = nullptr;
    st = scratch_alloc((void**)&scratch, split_bytes + status_bytes + 16, s);
    if (st != MP_OK) return st;
    int64_t* splits = reinterpret_cast<int64_t*>(scratch);
    unsigned long long* status = reinterpret_cast<unsigned long long*>(scratch + split_bytes);
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + split_bytes + status_bytes);
    cudaError_t e = cudaMemsetAsync(status, 0, status_bytes + 16, s);
    if (e == cudaSuccess) e = launch_partition(p, T, splits, s);
    if (e == cudaSuccess) e = launch_setop(p, (int)op, splits, status, counter, cap, out_count, s);
    scratch_free(scratch, s);
    return e == cudaSuccess ? MP_OK : cuda_fail(e, fn);
}

}  // extern "C"
