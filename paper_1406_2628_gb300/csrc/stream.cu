// stream.cu -- the partition-free streaming merge (Sec. V, Alg. 3).
//
// Alg. 3 lets each core walk its share of the output window after window,
// carrying its position on the Merge Path from one window to the next, so
// that only the start of the share needs a diagonal search.  Here each CTA
// owns R consecutive steps of T = NT*VT outputs.  It finds the split at the
// start and at the end of its share (Alg. 2, evaluated 32 probes at a time by
// one warp), then repeats:
//   * merge the next T outputs from the windows A[a, a+T) and B[b, b+T),
//     which by Lemma 16 hold every element those outputs can use: each
//     thread searches its diagonal inside the windows (Thm 17) and merges
//     VT outputs serially (ties take A);
//   * store them with coalesced 128-bit stores (gather by source index);
//   * advance (a, b) by the counts the merge consumed.
// The windows live in shared-memory ring buffers of C = (L+1)*T + 16
// elements per side.  At every step one thread issues TMA bulk copies that
// extend each ring to (L+1)*T elements past the current position, so the
// loads for step k+L are in flight while step k merges; every element of A
// and B crosses HBM once and no split-point array is read or written.
#include <algorithm>
#include <vector>

#include "mp_bulk.cuh"
#include "mp_device.cuh"
#include "mp_internal.h"
#include "mp_tile.cuh"

namespace mp {

template <class K>
struct StreamArgs {
    const K* a;
    const K* b;
    const uint32_t* av;
    const uint32_t* bv;
    K* out;
    uint32_t* outv;
    int64_t na, nb, total;
    int64_t steps_per_cta;  // R
    Codec<K> codec;
};

template <class K, bool VALS, int NT, int VT, int L>
struct StreamSmem {
    static constexpr int T = NT * VT;
    static constexpr int C = (L + 1) * T + 16;  // ring capacity, elements
    static constexpr size_t key_ring = ((size_t)C * sizeof(K) + 15) / 16 * 16;
    static constexpr size_t val_ring = VALS ? ((size_t)C * 4 + 15) / 16 * 16 : 0;
    static constexpr size_t idx_bytes = ((size_t)T * 2 + 15) / 16 * 16;
    static constexpr size_t ctl_bytes = ((size_t)(L + 1) * 8 + 32 + 15) / 16 * 16;  // mbarriers, splits
    static constexpr size_t bytes = 2 * key_ring + 2 * val_ring + idx_bytes + ctl_bytes;
};

// u + v with u, v < C, reduced mod C.
template <int C>
__device__ __forceinline__ uint32_t wrap(uint32_t u)
{
    const uint32_t v = u - (uint32_t)C;
    return u < v ? u : v;
}

// One side's ring: element j of the CTA's share (j counted from the share's
// first element g) lives in slot (j + ph) mod C, where ph is g's phase in
// its 16-byte granule, so a slot and its global element share their 16-byte
// phase and aligned runs can move by bulk copies.
template <class E>
struct Ring {
    E* s;
    const E* g;
    uint32_t ph;
};

template <int C>
__device__ __forceinline__ uint32_t slot_of(uint32_t j, uint32_t ph)
{
    return (j + ph) % (uint32_t)C;
}

// Aligned interior [h, t) of the range [f0, f1) of a ring.
template <class E>
__device__ __forceinline__ void ring_interior(const Ring<E>& r, uint32_t f0, uint32_t f1, uint32_t& h,
                                              uint32_t& t)
{
    constexpr uint32_t V = 16 / sizeof(E);
    const uint32_t m = (f0 + r.ph) % V;
    h = f0 + (m ? V - m : 0);
    if (h > f1) h = f1;
    t = h + ((f1 - h) / V) * V;
}

// Bulk copies of [h, t) into the ring (split where the ring wraps; both
// pieces start and end on 16-byte boundaries).
template <class E, int C>
__device__ __forceinline__ void ring_issue(const Ring<E>& r, uint32_t h, uint32_t t, uint64_t* bar)
{
    if (t == h) return;
    const uint32_t s0 = slot_of<C>(h, r.ph);
    const uint32_t n1 = (t - h) < (uint32_t)C - s0 ? (t - h) : (uint32_t)C - s0;
    bulk_g2s(r.s + s0, r.g + h, n1 * (uint32_t)sizeof(E), bar);
    if (t - h > n1) bulk_g2s(r.s, r.g + h + n1, (t - h - n1) * (uint32_t)sizeof(E), bar);
}

// Plain load of edge element j in [0, 2V) of [f0, f1): j < V: the head
// [f0, h); else the tail [t, f1).
template <class E, int C>
__device__ __forceinline__ void ring_edge(const Ring<E>& r, uint32_t f0, uint32_t f1, int j)
{
    constexpr int V = 16 / sizeof(E);
    if (j >= 2 * V) return;
    uint32_t h, t;
    ring_interior(r, f0, f1, h, t);
    const uint32_t idx = j < V ? f0 + j : t + (j - V);
    if (j < V ? idx < h : idx < f1) r.s[slot_of<C>(idx, r.ph)] = ld_global_nc(r.g + idx);
}

// Alg. 2 in global memory, one warp: the number of A elements among the
// first d outputs.  Each round the 32 lanes test 32 evenly spaced points of
// the remaining range [lo, hi) (the predicate A[m] > B[d-1-m] is false then
// true along the diagonal) and the range shrinks to the gap between the
// last false and the first true probe.  Returns the same value on every lane.
template <int CK, class K>
__device__ __forceinline__ int64_t warp_split(const K* A, int64_t na, const K* B, int64_t nb, int64_t d,
                                              Codec<K> c)
{
    const int lane = threadIdx.x & 31;
    int64_t lo = d - nb > 0 ? d - nb : 0;
    int64_t hi = d < na ? d : na;
    while (lo < hi) {
        const int64_t span = hi - lo;
        int64_t m;
        bool valid;
        if (span <= 32) {
            m = lo + lane;
            valid = lane < span;
        } else {
            m = lo + (span / 33) * (lane + 1) + ((span % 33) * (lane + 1)) / 33;
            valid = true;
        }
        bool pred = true;
        if (valid) pred = key_enc_ck<CK>(ld_global_nc(A + m), c) > key_enc_ck<CK>(ld_global_nc(B + (d - 1 - m)), c);
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, pred);
        const int f = ball ? __ffs(ball) - 1 : 32;
        const int64_t m_first = __shfl_sync(0xFFFFFFFFu, m, f & 31);
        const int64_t m_prev = __shfl_sync(0xFFFFFFFFu, m, (f + 31) & 31);
        if (f < 32 && (span > 32 || f < span)) hi = m_first;
        if (f > 0) lo = m_prev + 1;
    }
    return lo;
}

// Diagonal search (Alg. 2) inside the ring windows A' = ring A from slot bA
// (la elements) and B' likewise.
template <int CK, int C, class K>
__device__ __forceinline__ int ring_search(const K* sA, uint32_t bA, int la, const K* sB, uint32_t bB,
                                           int lb, int diag, Codec<K> c)
{
    int lo = diag - lb > 0 ? diag - lb : 0;
    int hi = diag < la ? diag : la;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key_enc_ck<CK>(sA[wrap<C>(bA + mid)], c) > key_enc_ck<CK>(sB[wrap<C>(bB + (diag - 1 - mid))], c))
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// Serial merge of VT outputs from split (ai, bi) of the ring windows (ties
// take A); records window-relative sources (A: 0..la-1, B: la..) and
// returns the A position after the last output.
template <class K, int VT, int CK, int C>
__device__ __forceinline__ int ring_merge_indices(const K* sA, uint32_t bA, int la, const K* sB,
                                                  uint32_t bB, int lb, int ai, int bi, Codec<K> c,
                                                  uint32_t (&packed)[(VT + 1) / 2])
{
    K ka = key_enc_ck<CK>(sA[wrap<C>(bA + ai)], c);
    K kb = key_enc_ck<CK>(sB[wrap<C>(bB + bi)], c);
#pragma unroll
    for (int i = 0; i < VT; ++i) {
        const bool take_a = (bi >= lb) || (ai < la && !(ka > kb));
        const uint32_t src = take_a ? (uint32_t)ai : (uint32_t)(la + bi);
        if (i & 1)
            packed[i / 2] |= src << 16;
        else
            packed[i / 2] = src;
        const K raw = take_a ? sA[wrap<C>(bA + (ai < la ? ai + 1 : la))] : sB[wrap<C>(bB + bi + 1)];
        const K kn = key_enc_ck<CK>(raw, c);
        if (take_a) {
            ka = kn;
            ++ai;
        } else {
            kb = kn;
            ++bi;
        }
    }
    return ai;
}

// Gather the step's L outputs by source index from the rings and write them
// (128-bit streaming stores when the destination is 16-byte aligned).
template <class K, bool VALS, int NT, int VT, int C>
__device__ __forceinline__ void ring_store(const K* sA, uint32_t kbA, const K* sB, uint32_t kbB,
                                           const uint32_t* vA, uint32_t vbA, const uint32_t* vB,
                                           uint32_t vbB, int la, int L, const uint16_t* sidx, K* gout,
                                           uint32_t* gvout)
{
    constexpr int EK = 16 / sizeof(K);
    const int tid = threadIdx.x;
    auto key_at = [&](int s) { return s < la ? sA[wrap<C>(kbA + s)] : sB[wrap<C>(kbB + (s - la))]; };
    int done = 0;
    if ((((uintptr_t)gout) & 15) == 0) {
        const int nvec = L / EK;
#pragma unroll
        for (int j = 0; j < VT / EK; ++j) {
            const int g = tid + j * NT;
            if (g < nvec) {
                K w[EK];
#pragma unroll
                for (int e = 0; e < EK; ++e) w[e] = key_at(sidx[g * EK + e]);
                st_global_cs_v4(gout + g * EK, *reinterpret_cast<uint4*>(w));
            }
        }
        done = nvec * EK;
    }
    for (int j = done + tid; j < L; j += NT) gout[j] = key_at(sidx[j]);
    if constexpr (VALS) {
        auto val_at = [&](int s) { return s < la ? vA[wrap<C>(vbA + s)] : vB[wrap<C>(vbB + (s - la))]; };
        int vdone = 0;
        if ((((uintptr_t)gvout) & 15) == 0) {
            const int nvec = L / 4;
#pragma unroll
            for (int j = 0; j < VT / 4; ++j) {
                const int g = tid + j * NT;
                if (g < nvec) {
                    const uint2 pk = *reinterpret_cast<const uint2*>(sidx + g * 4);
                    uint4 w;
                    w.x = val_at(pk.x & 0xFFFF);
                    w.y = val_at(pk.x >> 16);
                    w.z = val_at(pk.y & 0xFFFF);
                    w.w = val_at(pk.y >> 16);
                    st_global_cs_v4(gvout + g * 4, w);
                }
            }
            vdone = nvec * 4;
        }
        for (int j = vdone + tid; j < L; j += NT) gvout[j] = val_at(sidx[j]);
    }
}

template <class K, bool VALS, int NT, int VT, int L, int CK>
__global__ void __launch_bounds__(NT) merge_stream_kernel(StreamArgs<K> p, unsigned int* err)
{
    static_assert(VT % 4 == 0 && L >= 1, "stream shape");
    using SM = StreamSmem<K, VALS, NT, VT, L>;
    constexpr int T = NT * VT;
    constexpr int C = SM::C;
    constexpr int NB = L + 1;  // mbarriers: batch j uses bar[j % NB]
    constexpr uint32_t WAIT_LIMIT = 1u << 22;
    static_assert(2 * T <= 65535, "window indices are 16-bit");
    extern __shared__ __align__(16) unsigned char smem[];
    K* skA = reinterpret_cast<K*>(smem);
    K* skB = reinterpret_cast<K*>(smem + SM::key_ring);
    uint32_t* svA = reinterpret_cast<uint32_t*>(smem + 2 * SM::key_ring);
    uint32_t* svB = reinterpret_cast<uint32_t*>(smem + 2 * SM::key_ring + SM::val_ring);
    uint16_t* sidx = reinterpret_cast<uint16_t*>(smem + 2 * SM::key_ring + 2 * SM::val_ring);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * SM::key_ring + 2 * SM::val_ring + SM::idx_bytes);
    int64_t* ctl = reinterpret_cast<int64_t*>(bar + NB);  // [0] a at share start, [1] at end, [2] advance

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t d_start = (int64_t)blockIdx.x * p.steps_per_cta * T;
    if (d_start >= p.total) return;
    const int64_t d_end = d_start + p.steps_per_cta * T < p.total ? d_start + p.steps_per_cta * T : p.total;

    // Splits at both ends of the share (Alg. 2), warps 0 and 1 in parallel.
    if (warp < 2) {
        const int64_t d = warp == 0 ? d_start : d_end;
        const int64_t a = warp_split<CK>(p.a, p.na, p.b, p.nb, d, p.codec);
        if (lane == 0) ctl[warp] = a;
    }
    if (tid == 0) {
        for (int j = 0; j < NB; ++j) mbar_init(&bar[j], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // The end split kept consistent with the start (see clamp_end_split), so
    // that the share's windows lie inside A and B even for unsorted input.
    const int64_t a0 = ctl[0], b0 = d_start - a0;
    const int64_t a_end = clamp_end_split(ctl[1], a0, d_start, d_end, p.na, p.nb);
    const uint32_t nA = (uint32_t)(a_end - a0), nB = (uint32_t)((d_end - a_end) - b0);
    const Ring<K> rkA{skA, p.a + a0, (uint32_t)phase16(p.a + a0)};
    const Ring<K> rkB{skB, p.b + b0, (uint32_t)phase16(p.b + b0)};
    Ring<uint32_t> rvA{svA, nullptr, 0}, rvB{svB, nullptr, 0};
    if constexpr (VALS) {
        if (nA) rvA = Ring<uint32_t>{svA, p.av + a0, (uint32_t)phase16(p.av + a0)};
        if (nB) rvB = Ring<uint32_t>{svB, p.bv + b0, (uint32_t)phase16(p.bv + b0)};
    }

    const int nsteps = (int)((d_end - d_start + T - 1) / T);
    uint32_t a = 0, b = 0, fillA = 0, fillB = 0;
    int k = 0;
    bool ok = true;
    for (; k < nsteps; ++k) {
        // Batch k: extend both rings to (L+1)*T elements past (a, b).  The
        // slots it writes held elements before a (or b), consumed by step k-1.
        const uint32_t tA = nA - a < (uint32_t)((L + 1) * T) ? nA : a + (L + 1) * T;
        const uint32_t tB = nB - b < (uint32_t)((L + 1) * T) ? nB : b + (L + 1) * T;
        if (tid == 0) {
            uint32_t h[4], t[4];
            ring_interior(rkA, fillA, tA, h[0], t[0]);
            ring_interior(rkB, fillB, tB, h[1], t[1]);
            uint32_t tx = (t[0] - h[0] + t[1] - h[1]) * (uint32_t)sizeof(K);
            if constexpr (VALS) {
                ring_interior(rvA, fillA, tA, h[2], t[2]);
                ring_interior(rvB, fillB, tB, h[3], t[3]);
                tx += (t[2] - h[2] + t[3] - h[3]) * 4u;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_expect_tx(&bar[k % NB], tx);
            ring_issue<K, C>(rkA, h[0], t[0], &bar[k % NB]);
            ring_issue<K, C>(rkB, h[1], t[1], &bar[k % NB]);
            if constexpr (VALS) {
                ring_issue<uint32_t, C>(rvA, h[2], t[2], &bar[k % NB]);
                ring_issue<uint32_t, C>(rvB, h[3], t[3], &bar[k % NB]);
            }
        } else if (warp == 1) {
            // Ragged edges: lanes 0-7 key A, 8-15 key B, 16-23 value A, 24-31 value B.
            const int r = lane >> 3, j = lane & 7;
            if (r == 0) ring_edge<K, C>(rkA, fillA, tA, j);
            else if (r == 1) ring_edge<K, C>(rkB, fillB, tB, j);
            else if (VALS && r == 2) ring_edge<uint32_t, C>(rvA, fillA, tA, j);
            else if (VALS && r == 3) ring_edge<uint32_t, C>(rvB, fillB, tB, j);
        }
        fillA = tA;
        fillB = tB;

        // Step k reads A[a, a+T) and B[b, b+T): batch 0 covers them for
        // k <= L, batch k-L afterwards (earlier batches were waited before).
        bool ready = true;
        if (k == 0 || k > L) {
            const int j = k == 0 ? 0 : k - L;
            ready = mbar_wait_bounded(&bar[j % NB], (uint32_t)((j / NB) & 1), WAIT_LIMIT);
        }
        if (!__syncthreads_and(ready)) {
            ok = false;
            break;
        }

        const int64_t left = d_end - d_start - (int64_t)k * T;
        const int Lk = left < T ? (int)left : T;
        const int la = nA - a < (uint32_t)T ? (int)(nA - a) : T;
        const int lb = nB - b < (uint32_t)T ? (int)(nB - b) : T;
        const uint32_t kbA = slot_of<C>(a, rkA.ph), kbB = slot_of<C>(b, rkB.ph);
        {
            const int diag = tid * VT < Lk ? tid * VT : Lk;
            const int ai = ring_search<CK, C>(skA, kbA, la, skB, kbB, lb, diag, p.codec);
            uint32_t packed[(VT + 1) / 2];
            const int ae = ring_merge_indices<K, VT, CK, C>(skA, kbA, la, skB, kbB, lb, ai, diag - ai, p.codec,
                                                            packed);
            put_indices<VT>(sidx, packed);
            if (tid == NT - 1) ctl[2] = ae;  // A consumed by a full step
        }
        __syncthreads();
        uint32_t vbA = 0, vbB = 0;
        if constexpr (VALS) {
            vbA = slot_of<C>(a, rvA.ph);
            vbB = slot_of<C>(b, rvB.ph);
        }
        const int64_t d = d_start + (int64_t)k * T;
        ring_store<K, VALS, NT, VT, C>(skA, kbA, skB, kbB, svA, vbA, svB, vbB, la, Lk, sidx, p.out + d,
                                       VALS ? p.outv + d : nullptr);
        // A taken by this step; for sorted input exactly the path's, and
        // otherwise kept inside what remains of the share on each side (the
        // remainder holds at least T before the last step).
        uint32_t adv = (uint32_t)ctl[2];
        if ((uint32_t)T - adv > nB - b) adv = (uint32_t)T - (nB - b);
        if (adv > nA - a) adv = nA - a;
        a += adv;
        b += (uint32_t)T - adv;
        __syncthreads();  // rings and indices are free for the next batch and step
    }

    // Batches issued but not waited for (and, after a timeout, the one that
    // ran out) must land before the CTA's shared memory is released.
    if (tid == 0) {
        const int last = ok ? k - 1 : k;
        int first = ok ? last - L + 1 : 1;
        if (first < 1) first = 1;
        if (!ok) atomicOr(err, MP_KERR_MBAR_TIMEOUT);
        for (int j = first; j <= last; ++j) mbar_wait_bounded(&bar[j % NB], (uint32_t)((j / NB) & 1), WAIT_LIMIT);
    }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
// Compiled shapes (NT, VT, L): L = lookahead in steps; one L per (NT, VT).
#define MP_STREAM_SHAPES(X) X(128, 8, 1) X(256, 8, 1) X(256, 4, 1) X(128, 4, 2)

template <class K, bool VALS, int NT, int VT, int L, int CK>
static cudaError_t launch_stream_ck(const MergeProblem& p, cudaStream_t stream)
{
    using SM = StreamSmem<K, VALS, NT, VT, L>;
    constexpr int64_t T = NT * VT;
    auto kern = merge_stream_kernel<K, VALS, NT, VT, L, CK>;
    static int occ = 0;
    static int sms = 0;
    if (!occ) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
        if (e != cudaSuccess) return e;
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        int o = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, NT, SM::bytes)) != cudaSuccess) return e;
        if (o < 1) return cudaErrorInvalidConfiguration;
        occ = o;
    }
    unsigned int* err = kernel_error_word();
    if (!err) return cudaErrorInvalidSymbol;
    const int64_t total = p.na + p.nb;
    const int64_t tiles = ceil_div(total, T);
    // One resident wave when possible; a share stays below 2^30 elements so
    // share-relative indices fit 32 bits.
    int64_t steps = ceil_div(tiles, (int64_t)sms * occ);
    const int64_t max_steps = ((int64_t)1 << 30) / T;
    if (steps > max_steps) steps = max_steps;
    const int64_t grid = ceil_div(tiles, steps);
    StreamArgs<K> a;
    a.a = static_cast<const K*>(p.a);
    a.b = static_cast<const K*>(p.b);
    a.av = p.av;
    a.bv = p.bv;
    a.out = static_cast<K*>(p.out);
    a.outv = p.outv;
    a.na = p.na;
    a.nb = p.nb;
    a.total = total;
    a.steps_per_cta = steps;
    a.codec = make_codec<K>(p.kind.flip, p.kind.fmask, p.kind.inv);
    kern<<<(unsigned)grid, NT, SM::bytes, stream>>>(a, err);
    return cudaGetLastError();
}

template <class K, bool VALS, int NT, int VT, int L>
static cudaError_t launch_stream_t(const MergeProblem& p, cudaStream_t stream)
{
    if (p.kind.identity()) return launch_stream_ck<K, VALS, NT, VT, L, CODEC_IDENTITY>(p, stream);
    return launch_stream_ck<K, VALS, NT, VT, L, CODEC_RUNTIME>(p, stream);
}

bool stream_shape_supported(const Shape& s)
{
#define X(NT_, VT_, L_) \
    if (s.nt == NT_ && s.vt == VT_) return true;
    MP_STREAM_SHAPES(X)
#undef X
    return false;
}

std::vector<Shape> stream_shapes()
{
    std::vector<Shape> v;
#define X(NT_, VT_, L_) v.push_back(Shape{NT_, VT_, MP_STAGE_STREAM});
    MP_STREAM_SHAPES(X)
#undef X
    return v;
}

// Up to this many outputs the single streaming launch beats partition +
// tile kernels on GB300 (the saved launch and partition outweigh the lower
// occupancy of the ring buffers); above it the tile kernels win.  Measured
// crossover, L2 flushed: 4-byte keys alone between 2^22 and 2^23 outputs,
// 4-byte keys with values and 8-byte keys near 2^22.
int64_t stream_auto_limit(int key_bytes, bool with_values)
{
    if (key_bytes == 4 && !with_values) return (int64_t)1 << 22;
    return (int64_t)3 << 20;
}

Shape stream_default_shape(int key_bytes, bool with_values)
{
    if (key_bytes == 16 || (key_bytes == 8 && with_values)) return Shape{128, 8, MP_STAGE_STREAM};
    return Shape{256, 8, MP_STAGE_STREAM};
}

cudaError_t launch_merge_stream(const MergeProblem& p, const Shape& s, cudaStream_t stream)
{
    if (p.run != 0) return cudaErrorInvalidValue;
    if (p.na + p.nb == 0) return cudaSuccess;
    const bool vals = p.vals;
#define X(NT_, VT_, L_)                                                                          \
    if (s.nt == NT_ && s.vt == VT_) {                                                            \
        if (p.kind.bytes == 4)                                                                   \
            return vals ? launch_stream_t<uint32_t, true, NT_, VT_, L_>(p, stream)               \
                        : launch_stream_t<uint32_t, false, NT_, VT_, L_>(p, stream);             \
        if (p.kind.bytes == 16)                                                                  \
            return vals ? launch_stream_t<u128, true, NT_, VT_, L_>(p, stream)                   \
                        : launch_stream_t<u128, false, NT_, VT_, L_>(p, stream);                 \
        return vals ? launch_stream_t<uint64_t, true, NT_, VT_, L_>(p, stream)                   \
                    : launch_stream_t<uint64_t, false, NT_, VT_, L_>(p, stream);                 \
    }
    MP_STREAM_SHAPES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace mp
