// batched.cu -- many independent merges in one launch.
//
// Segment s merges A_s = a[a_off[s]..a_off[s+1]) with B_s = b[b_off[s]..
// b_off[s+1]) into out at c(s) = a_off[s] + b_off[s].  Concatenated, the
// segments' outputs form one merge of the concatenated A and B ordered by
// (segment, key) with ties to A (Cor. 6 applied to the segments), so Merge
// Path runs over the whole concatenated output: tiles of equal length
// whatever the segment sizes (Cor. 7), a tile may straddle segments.
//
//   partition  for each tile boundary d: the segment s holding output d
//              (upper bound of d in c(.)), then Alg. 2 inside that segment.
//   merge      one CTA per tile (TMA staging; register staging loops over a
//              resident grid); each stages its contiguous
//              A and B windows, each thread finds its segment (upper bound
//              in c over the tile's few segments) and its split inside the
//              window, then merges VT outputs, stepping to the next segment
//              when both sides of the current one are used up.
#include <algorithm>
#include <vector>

#include "mp_device.cuh"
#include "mp_internal.h"
#include "mp_tile.cuh"
#include "mp_bulk.cuh"

namespace mp {

template <class K>
struct BatchArgs {
    const K* a;
    const K* b;
    const uint32_t* av;
    const uint32_t* bv;
    K* out;
    uint32_t* outv;
    const int64_t* a_off;
    const int64_t* b_off;
    int64_t nseg;
    int64_t na, nb, total;
    int64_t ntiles;
    const int64_t* a_split;    // ntiles + 1
    const int64_t* seg_split;  // ntiles + 1: segment holding output t*T
    Codec<K> codec;
};

__device__ __forceinline__ int64_t seg_start(const int64_t* a_off, const int64_t* b_off, int64_t s)
{
    return __ldg(a_off + s) + __ldg(b_off + s);
}

// Largest s in [lo, hi] with c(s) <= d (c(lo) <= d must hold).
__device__ __forceinline__ int64_t segment_of(const int64_t* a_off, const int64_t* b_off, int64_t lo,
                                              int64_t hi, int64_t d)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (seg_start(a_off, b_off, mid) <= d)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <class K>
__global__ void __launch_bounds__(256) batched_partition_kernel(BatchArgs<K> p, int64_t spacing,
                                                                int64_t n_bounds, int64_t* a_split,
                                                                int64_t* seg_split)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_bounds) return;
    const int64_t d = t * spacing < p.total ? t * spacing : p.total;
    if (d == p.total) {
        a_split[t] = p.na;
        seg_split[t] = p.nseg - 1;
    } else {
        const int64_t s = segment_of(p.a_off, p.b_off, 0, p.nseg - 1, d);
        const int64_t aS = __ldg(p.a_off + s), aE = __ldg(p.a_off + s + 1);
        const int64_t bS = __ldg(p.b_off + s), bE = __ldg(p.b_off + s + 1);
        const K* A = p.a + aS;
        const K* B = p.b + bS;
        const Codec<K> c = p.codec;
        const int64_t al = diagonal_search<K>([&](int64_t i) { return key_enc(__ldg(A + i), c); }, aE - aS,
                                              [&](int64_t i) { return key_enc(__ldg(B + i), c); }, bE - bS,
                                              d - aS - bS);
        a_split[t] = aS + al;
        seg_split[t] = s;
    }
    asm volatile("griddepcontrol.launch_dependents;");
}

// The tile's window bounds (split points clamped into the grid and made
// monotone, see merge_tile_body) and segment range.
struct BatchTile {
    int64_t d0, a0, a1, b0, b1, s0, s1;
    int la, lb;
};

template <class K>
__device__ __forceinline__ BatchTile batch_tile(const BatchArgs<K>& p, int64_t tile, int T)
{
    BatchTile t;
    t.d0 = tile * T;
    const int64_t d1 = t.d0 + T < p.total ? t.d0 + T : p.total;
    t.a0 = clamp_split(p.a_split[tile], t.d0, p.na, p.nb);
    t.a1 = clamp_end_split(p.a_split[tile + 1], t.a0, t.d0, d1, p.na, p.nb);
    t.b0 = t.d0 - t.a0;
    t.b1 = d1 - t.a1;
    int64_t s0 = p.seg_split[tile], s1 = p.seg_split[tile + 1];
    t.s0 = s0 < 0 ? 0 : (s0 > p.nseg - 1 ? p.nseg - 1 : s0);
    t.s1 = s1 < t.s0 ? t.s0 : (s1 > p.nseg - 1 ? p.nseg - 1 : s1);
    t.la = (int)(t.a1 - t.a0);
    t.lb = (int)(t.b1 - t.b0);
    return t;
}

// Per-thread part of a batched tile: find the thread's segment and its
// split inside the staged window, merge VT outputs (stepping to the next
// segment when both sides of the current one are used up) and record the
// outputs' sources in v.sidx, or (DIRECT) the merged keys themselves in
// outk.  Returns false for a thread with no outputs in the tile.
template <class K, bool VALS, int NT, int VT, int CK, bool DIRECT = false>
__device__ __forceinline__ bool batched_thread_merge(const BatchArgs<K>& p, const BatchTile& bt,
                                                     const TileView<K, VALS, NT, VT>& v,
                                                     K* outk = nullptr)
{
    const Codec<K> c = p.codec;
    const int tid = threadIdx.x;
    const int la = bt.la, lb = bt.lb, L = la + lb;
    const int64_t a0 = bt.a0, a1 = bt.a1, b0 = bt.b0, b1 = bt.b1;
    const int diag = tid * VT < L ? tid * VT : L;
    if (diag >= L) return false;
    uint32_t packed[(VT + 1) / 2];
    if (bt.s0 == bt.s1) {
        // The whole tile lies in one segment: a plain Merge Path tile.
        const int ai = smem_diagonal_search_ck<CK>(v.sA, la, v.sB, lb, diag, c);
        if constexpr (DIRECT) {
            K (&ok)[VT] = *reinterpret_cast<K(*)[VT]>(outk);
            serial_merge_keys_ck<K, VT, CK>(v.sA, la, v.sB, lb, ai, diag - ai, c, ok);
        } else {
            serial_merge_indices_ck<K, VT, CK>(v.sA, la, v.sB, lb, ai, diag - ai, c, packed);
            put_indices<VT>(v.sidx, packed);
        }
        return true;
    }
    const int64_t dg = bt.d0 + diag;
    int64_t s = segment_of(p.a_off, p.b_off, bt.s0, bt.s1, dg);
    const int64_t aS = __ldg(p.a_off + s), aE = __ldg(p.a_off + s + 1);
    const int64_t bS = __ldg(p.b_off + s), bE = __ldg(p.b_off + s + 1);
    const int64_t dl = dg - aS - bS;
    // Alg. 2 inside segment s, restricted to the staged window (the split at
    // dg lies between the tile's own splits).
    int64_t lo = dl - (bE - bS);
    lo = lo > 0 ? lo : 0;
    lo = lo > a0 - aS ? lo : a0 - aS;
    lo = lo > dl - (b1 - bS) ? lo : dl - (b1 - bS);
    int64_t hi = dl < aE - aS ? dl : aE - aS;
    hi = hi < a1 - aS ? hi : a1 - aS;
    hi = hi < dl - (b0 - bS) ? hi : dl - (b0 - bS);
    const K* sAs = v.sA + (aS - a0);  // segment s's A, window-relative
    const K* sBs = v.sB + (bS - b0);
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (key_enc_ck<CK>(sAs[mid], c) > key_enc_ck<CK>(sBs[dl - 1 - mid], c))
            hi = mid;
        else
            lo = mid + 1;
    }
    // Window-relative positions, kept inside the window even for malformed
    // offsets (no effect on valid input).
    auto clampi = [](int64_t x, int top) { return (int)(x < 0 ? 0 : (x > top ? top : x)); };
    int ai = clampi(aS + lo - a0, la);
    int bi = clampi(bS + dl - lo - b0, lb);
    int aEnd = clampi((aE < a1 ? aE : a1) - a0, la);
    int bEnd = clampi((bE < b1 ? bE : b1) - b0, lb);
    K ka = key_enc_ck<CK>(v.sA[ai], c);
    K kb = key_enc_ck<CK>(v.sB[bi], c);
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        uint32_t src = 0;
        K key = K(0);
        if (diag + i < L) {
            // Both sides of segment s used up: step to the next segment
            // (skipping empty ones); ai, bi already point at its first elements.
            while (ai >= aEnd && bi >= bEnd && s + 1 < p.nseg) {
                ++s;
                const int64_t na1 = __ldg(p.a_off + s + 1), nb1 = __ldg(p.b_off + s + 1);
                aEnd = clampi((na1 < a1 ? na1 : a1) - a0, la);
                bEnd = clampi((nb1 < b1 ? nb1 : b1) - b0, lb);
            }
            const bool take_a = ai < aEnd && (bi >= bEnd || !(ka > kb));
            src = take_a ? (uint32_t)ai : (uint32_t)(la + bi);
            key = take_a ? ka : kb;
            const K* nxt = take_a ? (v.sA + (ai < la ? ai + 1 : la)) : (v.sB + (bi < lb ? bi + 1 : lb));
            const K kn = key_enc_ck<CK>(*nxt, c);
            if (take_a) { ka = kn; ++ai; }
            else { kb = kn; ++bi; }
        }
        if constexpr (DIRECT) {
            outk[i] = key_dec_ck<CK>(key, c);
        } else {
            if (i & 1)
                packed[i / 2] |= src << 16;
            else
                packed[i / 2] = src;
        }
    }
    if constexpr (!DIRECT) put_indices<VT>(v.sidx, packed);
    return true;
}

template <class K, bool VALS, int NT, int VT>
__global__ void __launch_bounds__(NT) batched_merge_kernel(BatchArgs<K> p)
{
    static_assert(VT % 4 == 0, "VT must be a multiple of 4");
    constexpr int T = NT * VT;
    extern __shared__ __align__(16) unsigned char smem[];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int64_t tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
        const BatchTile bt = batch_tile(p, tile, T);
        const auto v = stage_tile<K, VALS, NT, VT>(smem, p.a + bt.a0, bt.la, p.b + bt.b0, bt.lb,
                                                   VALS ? p.av + bt.a0 : nullptr,
                                                   VALS ? p.bv + bt.b0 : nullptr);
        batched_thread_merge<K, VALS, NT, VT, CODEC_RUNTIME>(p, bt, v);
        __syncthreads();
        store_tile<K, VALS, NT, VT>(v, p.out + bt.d0, VALS ? p.outv + bt.d0 : nullptr);
        __syncthreads();
    }
}

// Same, with the windows staged by TMA bulk copies (no staging registers),
// compiled per key codec (CK).
template <class K, bool VALS, int NT, int VT, int CK>
__global__ void __launch_bounds__(NT, merge_keys_direct<K, VALS, VT>() ? 1024 / NT : 1)
    batched_merge_bulk_kernel(BatchArgs<K> p, unsigned int* err)
{
    constexpr int T = NT * VT;
    constexpr bool DIRECT = merge_keys_direct<K, VALS, VT>();
    extern __shared__ __align__(16) unsigned char smem[];
    const BulkLayout<K, VALS, NT, VT, !DIRECT> lay(smem);
    bulk_init(lay.bar);
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    uint32_t parity = 0;
    for (int64_t tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
        const BatchTile bt = batch_tile(p, tile, T);
        TilePlace<K> t;
        t.gA = p.a + bt.a0;
        t.gB = p.b + bt.b0;
        t.gvA = VALS ? p.av + bt.a0 : nullptr;
        t.gvB = VALS ? p.bv + bt.b0 : nullptr;
        t.la = bt.la;
        t.lb = bt.lb;
        t.d0 = bt.d0;
        const auto v = stage_view<K, VALS, NT, VT>(t, lay.sk, lay.sv, lay.sidx);
        if (!bulk_stage<K, VALS, NT, VT>(t, v, lay.bar, parity, err)) return;
        parity ^= 1;
        if constexpr (DIRECT) {
            // As in merge_tile_bulk_body: the merged keys replace the
            // windows in thread order and leave by 128-bit loads and stores.
            K outk[VT];
            const bool active = batched_thread_merge<K, VALS, NT, VT, CK, true>(p, bt, v, outk);
            __syncthreads();
            if (active) {
#pragma unroll
                for (int i = 0; i < VT; ++i) lay.sk[threadIdx.x * VT + i] = outk[i];
            }
            __syncthreads();
            store_linear<K, NT, VT>(lay.sk, bt.la + bt.lb, p.out + bt.d0);
            // Order these shared-memory accesses before the next tile's
            // bulk copies into the same bytes.
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        } else {
            batched_thread_merge<K, VALS, NT, VT, CK>(p, bt, v);
            __syncthreads();
            store_tile<K, VALS, NT, VT>(v, p.out + bt.d0, VALS ? p.outv + bt.d0 : nullptr);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
template <class K>
static BatchArgs<K> make_batch_args(const BatchedProblem& q, int64_t tile, const int64_t* a_split,
                                    const int64_t* seg_split)
{
    BatchArgs<K> p;
    p.a = static_cast<const K*>(q.a);
    p.b = static_cast<const K*>(q.b);
    p.av = q.av;
    p.bv = q.bv;
    p.out = static_cast<K*>(q.out);
    p.outv = q.outv;
    p.a_off = q.a_off;
    p.b_off = q.b_off;
    p.nseg = q.nseg;
    p.na = q.na;
    p.nb = q.nb;
    p.total = q.na + q.nb;
    p.ntiles = ceil_div(p.total, tile);
    p.a_split = a_split;
    p.seg_split = seg_split;
    p.codec.flip = (K)q.kind.flip;
    p.codec.fmask = (K)q.kind.fmask;
    p.codec.inv = (K)q.kind.inv;
    return p;
}

template <class K, bool VALS, int NT, int VT, bool BULK, int CK = CODEC_RUNTIME>
static cudaError_t launch_batched_t(const BatchedProblem& q, int64_t* a_split, int64_t* seg_split,
                                    cudaStream_t stream)
{
    using SM = typename std::conditional<BULK, MergeBulkSmem<K, VALS, NT, VT>, TileSmem<K, VALS, NT, VT>>::type;
    void (*kern)(BatchArgs<K>, unsigned int*) = nullptr;
    void (*kern_v)(BatchArgs<K>) = nullptr;
    if constexpr (BULK)
        kern = batched_merge_bulk_kernel<K, VALS, NT, VT, CK>;
    else
        kern_v = batched_merge_kernel<K, VALS, NT, VT>;
    static int blocks_per_sm = 0;
    static int num_sms = 0;
    if (blocks_per_sm == 0) {
        cudaError_t e = BULK ? cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes)
                             : cudaFuncSetAttribute(kern_v, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = BULK ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, NT, SM::bytes)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern_v, NT, SM::bytes);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    const int64_t T = (int64_t)NT * VT;
    BatchArgs<K> p = make_batch_args<K>(q, T, a_split, seg_split);
    const int64_t n_bounds = p.ntiles + 1;
    batched_partition_kernel<K><<<(unsigned)ceil_div(n_bounds, 256), 256, 0, stream>>>(
        p, T, n_bounds, a_split, seg_split);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // One launch over every segment.  TMA-staged tiles go one per CTA (the
    // hardware starts a CTA as soon as one retires, overlapping one tile's
    // copies with other tiles' merges); register-staged tiles loop over a
    // resident grid.
    const int64_t grid = BULK ? p.ntiles : std::min<int64_t>(p.ntiles, (int64_t)num_sms * blocks_per_sm);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = SM::bytes;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if constexpr (BULK) {
        unsigned int* err = kernel_error_word();
        if (!err) return cudaErrorInvalidSymbol;
        return cudaLaunchKernelEx(&cfg, kern, p, err);
    } else {
        return cudaLaunchKernelEx(&cfg, kern_v, p);
    }
}

// Tile shapes: register-staged and TMA-staged (MP_BATCHED_SHAPES), and
// TMA-staged only (MP_BATCHED_BULK_SHAPES: odd items per thread).
#define MP_BATCHED_SHAPES(X) X(128, 8) X(256, 8) X(128, 12) X(256, 12) X(128, 16) X(256, 16)
#define MP_BATCHED_BULK_SHAPES(X) X(128, 27) X(128, 33)

static bool batched_shape_supported(const Shape& s)
{
    if (s.staging != MP_STAGE_VECTOR && s.staging != MP_STAGE_BULK) return false;
#define X(NT_, VT_) if (s.nt == NT_ && s.vt == VT_) return true;
    MP_BATCHED_SHAPES(X)
    if (s.staging == MP_STAGE_BULK) {
        MP_BATCHED_BULK_SHAPES(X)
    }
#undef X
    return false;
}

// TMA-staged launch with the key codec fixed at compile time where it can
// be (unsigned keys, signed integers); other kinds use the runtime codec.
template <class K, bool VALS, int NT, int VT>
static cudaError_t launch_batched_bulk(const BatchedProblem& q, int64_t* a_split, int64_t* seg_split,
                                       cudaStream_t stream)
{
    if (q.kind.identity())
        return launch_batched_t<K, VALS, NT, VT, true, CODEC_IDENTITY>(q, a_split, seg_split, stream);
    if (q.kind.signed_int())
        return launch_batched_t<K, VALS, NT, VT, true, CODEC_SIGNED>(q, a_split, seg_split, stream);
    return launch_batched_t<K, VALS, NT, VT, true, CODEC_RUNTIME>(q, a_split, seg_split, stream);
}

static cudaError_t launch_batched(const BatchedProblem& q, const Shape& s, int64_t* a_split,
                                  int64_t* seg_split, cudaStream_t stream)
{
    const bool vals = q.vals;
    const bool bulk = s.staging == MP_STAGE_BULK;
#define X(NT_, VT_)                                                                                    \
    if (s.nt == NT_ && s.vt == VT_) {                                                                  \
        if (q.kind.bytes == 4) {                                                                       \
            if (bulk)                                                                                  \
                return vals ? launch_batched_bulk<uint32_t, true, NT_, VT_>(q, a_split, seg_split, stream)   \
                            : launch_batched_bulk<uint32_t, false, NT_, VT_>(q, a_split, seg_split, stream); \
            return vals ? launch_batched_t<uint32_t, true, NT_, VT_, false>(q, a_split, seg_split, stream)      \
                        : launch_batched_t<uint32_t, false, NT_, VT_, false>(q, a_split, seg_split, stream);    \
        }                                                                                              \
        if (bulk)                                                                                      \
            return vals ? launch_batched_bulk<uint64_t, true, NT_, VT_>(q, a_split, seg_split, stream)       \
                        : launch_batched_bulk<uint64_t, false, NT_, VT_>(q, a_split, seg_split, stream);     \
        return vals ? launch_batched_t<uint64_t, true, NT_, VT_, false>(q, a_split, seg_split, stream)          \
                    : launch_batched_t<uint64_t, false, NT_, VT_, false>(q, a_split, seg_split, stream);        \
    }
    MP_BATCHED_SHAPES(X)
#undef X
#define X(NT_, VT_)                                                                                    \
    if (bulk && s.nt == NT_ && s.vt == VT_) {                                                          \
        if (q.kind.bytes == 4)                                                                         \
            return vals ? launch_batched_bulk<uint32_t, true, NT_, VT_>(q, a_split, seg_split, stream)       \
                        : launch_batched_bulk<uint32_t, false, NT_, VT_>(q, a_split, seg_split, stream);     \
        return vals ? launch_batched_bulk<uint64_t, true, NT_, VT_>(q, a_split, seg_split, stream)           \
                    : launch_batched_bulk<uint64_t, false, NT_, VT_>(q, a_split, seg_split, stream);         \
    }
    MP_BATCHED_BULK_SHAPES(X)
#undef X
    return cudaErrorInvalidValue;
}

mp_status batched_prepare(mp_dtype dtype, const void* a, const int64_t* a_off, const void* b,
                          const int64_t* b_off, int64_t nseg, int64_t na_total, int64_t nb_total,
                          void* out, const uint32_t* a_vals, const uint32_t* b_vals,
                          uint32_t* out_vals, const mp_plan* plan, BatchedProblem* q, Shape* s)
{
    KeyKind k;
    if (!key_kind(dtype, &k) || k.bytes == 16)
        return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_merge_batched: unknown or 128-bit dtype");
    if (nseg < 0 || na_total < 0 || nb_total < 0)
        return fail(MP_ERR_INVALID_ARG, "mp_merge_batched: negative size");
    if (nseg == 0 && na_total + nb_total != 0)
        return fail(MP_ERR_INVALID_ARG, "mp_merge_batched: no segments but nonzero totals");
    if (nseg > 0 && (!a_off || !b_off))
        return fail(MP_ERR_INVALID_ARG, "mp_merge_batched: NULL offsets");
    if (((uintptr_t)a_off & 7) || ((uintptr_t)b_off & 7))
        return fail(MP_ERR_INVALID_ARG, "mp_merge_batched: offsets not 8-byte aligned");
    const bool vals = a_vals || b_vals || out_vals;
    if (vals && ((na_total > 0 && !a_vals) || (nb_total > 0 && !b_vals) || (na_total + nb_total > 0 && !out_vals)))
        return fail(MP_ERR_INVALID_ARG, "mp_merge_batched: NULL value array for a non-empty side");
    if ((na_total > 0 && !a) || (nb_total > 0 && !b) || (na_total + nb_total > 0 && !out))
        return fail(MP_ERR_INVALID_ARG, "mp_merge_batched: NULL key pointer");
    if (((uintptr_t)a % k.bytes) || ((uintptr_t)b % k.bytes) || ((uintptr_t)out % k.bytes))
        return fail(MP_ERR_INVALID_ARG, "mp_merge_batched: key pointer not aligned to the key size");
    if (vals && (((uintptr_t)a_vals & 3) || ((uintptr_t)b_vals & 3) || ((uintptr_t)out_vals & 3)))
        return fail(MP_ERR_INVALID_ARG, "mp_merge_batched: value pointer not 4-byte aligned");

    if (!tuned_shape("batched", k.bytes, vals, na_total + nb_total, s)) {
        // Tiles of 128 x 33: the batched tile's walks (segment lookups and
        // the serial merge) are bound by the shared-memory pipe; an odd
        // number of outputs per thread starts the threads' walks in
        // different banks and spreads each thread's search over more
        // outputs (16,384 int32 segments: 1.11 ms, against 1.17 ms for
        // 128 x 12 and 1.63 ms for 256 x 16).
        s->nt = 128;
        s->vt = 33;
        s->staging = MP_STAGE_BULK;
    }
    if (plan) {
        if (plan->reserved) return fail(MP_ERR_INVALID_ARG, "plan.reserved must be 0");
        if (plan->block_threads) s->nt = plan->block_threads;
        if (plan->items_per_thread) s->vt = plan->items_per_thread;
        if (plan->staging) s->staging = plan->staging;
    }
    if (!batched_shape_supported(*s)) return fail(MP_ERR_INVALID_ARG, "mp_merge_batched: unsupported plan");

    q->kind = k;
    q->a = a;
    q->b = b;
    q->a_off = a_off;
    q->b_off = b_off;
    q->nseg = nseg;
    q->na = na_total;
    q->nb = nb_total;
    q->out = out;
    q->vals = vals;
    q->av = a_vals;
    q->bv = b_vals;
    q->outv = out_vals;
    return MP_OK;
}

size_t batched_scratch_bytes(const BatchedProblem& q, const Shape& s)
{
    return (size_t)(ceil_div(q.na + q.nb, s.tile()) + 1) * 16;
}

cudaError_t batched_launch(const BatchedProblem& q, const Shape& s, void* scratch, cudaStream_t stream)
{
    if (q.na + q.nb == 0) return cudaSuccess;
    const int64_t bounds = ceil_div(q.na + q.nb, s.tile()) + 1;
    int64_t* sp = static_cast<int64_t*>(scratch);
    return launch_batched(q, s, sp, sp + bounds, stream);
}

std::vector<Shape> batched_shapes()
{
    std::vector<Shape> v;
#define X(NT_, VT_) v.push_back(Shape{NT_, VT_, MP_STAGE_VECTOR}); v.push_back(Shape{NT_, VT_, MP_STAGE_BULK});
    MP_BATCHED_SHAPES(X)
#undef X
#define X(NT_, VT_) v.push_back(Shape{NT_, VT_, MP_STAGE_BULK});
    MP_BATCHED_BULK_SHAPES(X)
#undef X
    return v;
}

}  // namespace mp

using namespace mp;

extern "C" mp_status mp_merge_batched(mp_dtype dtype, const void* a, const int64_t* a_off,
                                      const void* b, const int64_t* b_off, int64_t nseg,
                                      int64_t na_total, int64_t nb_total, void* out,
                                      const uint32_t* a_vals, const uint32_t* b_vals,
                                      uint32_t* out_vals, const mp_plan* plan, mp_stream_t stream)
{
    MP_RANGE("mp_merge_batched");
    BatchedProblem q;
    Shape s;
    mp_status ms = batched_prepare(dtype, a, a_off, b, b_off, nseg, na_total, nb_total, out, a_vals,
                                   b_vals, out_vals, plan, &q, &s);
    if (ms != MP_OK || na_total + nb_total == 0) return ms;
    cudaStream_t st = (cudaStream_t)stream;
    void* scratch = nullptr;
    ms = scratch_alloc(&scratch, batched_scratch_bytes(q, s), st);
    if (ms != MP_OK) return ms;
    cudaError_t e = batched_launch(q, s, scratch, st);
    scratch_free(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "mp_merge_batched");
    return MP_OK;
}

extern "C" mp_status mp_autotune_batched(mp_dtype dtype, const void* a, const int64_t* a_off,
                                         const void* b, const int64_t* b_off, int64_t nseg,
                                         int64_t na_total, int64_t nb_total, void* out,
                                         const uint32_t* a_vals, const uint32_t* b_vals,
                                         uint32_t* out_vals, int reps, mp_plan* best,
                                         mp_stream_t stream)
{
    BatchedProblem q;
    Shape s;
    mp_status ms = batched_prepare(dtype, a, a_off, b, b_off, nseg, na_total, nb_total, out, a_vals,
                                   b_vals, out_vals, nullptr, &q, &s);
    if (ms != MP_OK) return ms;
    if (na_total + nb_total == 0) return fail(MP_ERR_INVALID_ARG, "mp_autotune_batched: empty problem");
    if (reps < 1) reps = 1;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(MP_ERR_CUDA, "mp_autotune_batched: events");
    Shape best_s = s;
    float best_ms = 1e30f;
    for (const Shape& cand : batched_shapes()) {
        void* scratch = nullptr;
        ms = scratch_alloc(&scratch, batched_scratch_bytes(q, cand), st);
        if (ms != MP_OK) break;
        cudaError_t e = batched_launch(q, cand, scratch, st);  // warm-up
        float cand_ms = 1e30f;
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            cudaEventRecord(e0, st);
            e = batched_launch(q, cand, scratch, st);
            cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0;
            if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess && t < cand_ms) cand_ms = t;
        }
        scratch_free(scratch, st);
        if (e != cudaSuccess) { ms = cuda_fail(e, "mp_autotune_batched"); break; }
        if (cand_ms < best_ms) { best_ms = cand_ms; best_s = cand; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms != MP_OK) return ms;
    record_shape("batched", q.kind.bytes, q.vals, na_total + nb_total, best_s);
    if (best) *best = mp_plan{best_s.nt, best_s.vt, best_s.staging, 0};
    return MP_OK;
}
