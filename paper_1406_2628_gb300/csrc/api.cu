// api.cu -- the C ABI (include/mp.h): argument checks, scratch memory,
// dispatch to the kernels, status strings and the sortedness check.
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>
#include <string>

#include "mp_device.cuh"
#include "mp_internal.h"

namespace mp {

static thread_local std::string g_last_error;

mp_status fail(mp_status st, const std::string& detail)
{
    g_last_error = detail;
    return st;
}

mp_status cuda_fail(cudaError_t err, const char* where)
{
    std::string d = std::string(where) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
    if (err == cudaErrorMemoryAllocation) return fail(MP_ERR_NO_MEMORY, d);
    return fail(MP_ERR_CUDA, d);
}

bool key_kind(mp_dtype dtype, KeyKind* k)
{
    const int d = (int)dtype;
    if (d & ~(0xFF | MP_DESCENDING)) return false;
    switch (d & 0xFF) {
    case MP_I32: *k = {4, 0x80000000ull, 0, 0}; break;
    case MP_U32: *k = {4, 0, 0, 0}; break;
    case MP_F32: *k = {4, 0x80000000ull, 0xFFFFFFFFull, 0}; break;
    case MP_U64: *k = {8, 0, 0, 0}; break;
    case MP_I64: *k = {8, 0x8000000000000000ull, 0, 0}; break;
    // 128-bit keys: flip names the top bit of the top 64-bit word.
    case MP_U128: *k = {16, 0, 0, 0}; break;
    case MP_I128: *k = {16, 0x8000000000000000ull, 0, 0}; break;
    default: return false;
    }
    if (d & MP_DESCENDING) k->inv = k->bytes == 4 ? 0xFFFFFFFFull : ~0ull;
    return true;
}

// ---------------------------------------------------------------------------
// Scratch: one stream-ordered memory pool per device, owned by the library.
// Its release threshold keeps freed blocks for reuse, so repeated calls do
// not go back to the driver.
// ---------------------------------------------------------------------------
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64];
static bool g_pool_made[64];

static mp_status get_pool(cudaMemPool_t* pool)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(MP_ERR_INTERNAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_made[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&g_pools[dev], &props);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemPoolCreate");
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool_made[dev] = true;
    }
    *pool = g_pools[dev];
    return MP_OK;
}

// Host-side fault injection (mp_inject_fault): how many more scratch
// allocations and queue steps are to fail.
static std::atomic<int64_t> g_fault_count[4];

bool take_fault(int kind)
{
    if (kind <= 0 || kind >= 4) return false;
    int64_t c = g_fault_count[kind].load();
    while (c > 0)
        if (g_fault_count[kind].compare_exchange_weak(c, c - 1)) return true;
    return false;
}

mp_status scratch_alloc(void** ptr, size_t bytes, cudaStream_t stream)
{
    cudaMemPool_t pool = nullptr;
    mp_status st = get_pool(&pool);
    if (st != MP_OK) return st;
    if (take_fault(MP_FAULT_SCRATCH_ALLOC)) {
        *ptr = nullptr;
        return cuda_fail(cudaErrorMemoryAllocation, "scratch allocation (injected fault)");
    }
    cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes < 256 ? 256 : bytes, pool, stream);
    if (e != cudaSuccess) return cuda_fail(e, "scratch allocation");
    return MP_OK;
}

void scratch_free(void* ptr, cudaStream_t stream)
{
    if (ptr) cudaFreeAsync(ptr, stream);
}

// ---------------------------------------------------------------------------
// Argument checks.
// ---------------------------------------------------------------------------
static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

static bool overlaps(const void* p, size_t pb, const void* q, size_t qb)
{
    if (!p || !q || pb == 0 || qb == 0) return false;
    uintptr_t a = (uintptr_t)p, b = (uintptr_t)q;
    return a < b + qb && b < a + pb;
}

// out_n: the output length in elements (-1: na + nb).
static mp_status check_merge_args(const KeyKind& k, const void* a, const uint32_t* av, int64_t na,
                                  const void* b, const uint32_t* bv, int64_t nb, const void* out,
                                  const uint32_t* outv, bool vals, const char* fn, int64_t out_n = -1)
{
    std::string f(fn);
    if (na < 0 || nb < 0) return fail(MP_ERR_INVALID_ARG, f + ": negative size");
    if (na > ((int64_t)1 << 46) || nb > ((int64_t)1 << 46)) return fail(MP_ERR_INVALID_ARG, f + ": size too large");
    const int64_t on = out_n < 0 ? na + nb : out_n;
    if (vals && ((na > 0 && !av) || (nb > 0 && !bv) || (on > 0 && !outv)))
        return fail(MP_ERR_INVALID_ARG, f + ": NULL value array for a non-empty side");
    if ((na > 0 && !a) || (nb > 0 && !b) || (on > 0 && !out))
        return fail(MP_ERR_INVALID_ARG, f + ": NULL key pointer");
    if (!aligned(a, k.bytes) || !aligned(b, k.bytes) || !aligned(out, k.bytes))
        return fail(MP_ERR_INVALID_ARG, f + ": key pointer not aligned to the key size");
    if (vals && (!aligned(av, 4) || !aligned(bv, 4) || !aligned(outv, 4)))
        return fail(MP_ERR_INVALID_ARG, f + ": value pointer not 4-byte aligned");
    const size_t ob = (size_t)on * k.bytes;
    if (overlaps(out, ob, a, (size_t)na * k.bytes) || overlaps(out, ob, b, (size_t)nb * k.bytes))
        return fail(MP_ERR_INVALID_ARG, f + ": output overlaps an input");
    if (vals) {
        const size_t ovb = (size_t)on * 4;
        if (overlaps(outv, ovb, av, (size_t)na * 4) || overlaps(outv, ovb, bv, (size_t)nb * 4) ||
            overlaps(outv, ovb, out, ob) || overlaps(outv, ovb, a, (size_t)na * k.bytes) ||
            overlaps(outv, ovb, b, (size_t)nb * k.bytes) || overlaps(out, ob, av, (size_t)na * 4) ||
            overlaps(out, ob, bv, (size_t)nb * 4))
            return fail(MP_ERR_INVALID_ARG, f + ": value output overlaps another array");
    }
    return MP_OK;
}

mp_status check_merge_args_ext(const KeyKind& k, const void* a, const uint32_t* av, int64_t na,
                               const void* b, const uint32_t* bv, int64_t nb, const void* out,
                               const uint32_t* outv, bool vals, const char* fn, int64_t out_n)
{
    return check_merge_args(k, a, av, na, b, bv, nb, out, outv, vals, fn, out_n);
}

static bool plan_is_auto(const mp_plan* plan)
{
    return !plan || (!plan->block_threads && !plan->items_per_thread && !plan->staging && !plan->reserved);
}

// MP_FORCE_PLAN=NT,VT[,staging] (staging: vector, bulk, warp, stream or its
// MP_STAGE_* number) replaces every automatic merge plan, for experiments;
// read at each call.  Returns false when unset.
static bool forced_plan(mp_plan* out)
{
    const char* env = getenv("MP_FORCE_PLAN");
    if (!env || !*env) return false;
    int nt = 0, vt = 0;
    char stage[16] = {0};
    const int got = sscanf(env, "%d,%d,%15s", &nt, &vt, stage);
    if (got < 2) return false;
    int st = 0;
    if (got == 3) {
        if (!strcmp(stage, "vector")) st = MP_STAGE_VECTOR;
        else if (!strcmp(stage, "bulk")) st = MP_STAGE_BULK;
        else if (!strcmp(stage, "warp")) st = MP_STAGE_WARP;
        else if (!strcmp(stage, "stream")) st = MP_STAGE_STREAM;
        else st = atoi(stage);
    }
    *out = mp_plan{nt, vt, st, 0};
    return true;
}

// allow_stream: an automatic plan may pick the streaming merge (small
// merges, where it saves the partition launch); callers that supply split
// points pass false.
static mp_status resolve_shape(const KeyKind& k, bool vals, int64_t total, const mp_plan* plan, Shape* s,
                               bool allow_stream = true)
{
    mp_plan forced;
    if (plan_is_auto(plan) && forced_plan(&forced)) plan = &forced;
    if (plan_is_auto(plan)) {
        if (tuned_shape("merge", k.bytes, vals, total, s) && (allow_stream || s->staging != MP_STAGE_STREAM))
            return MP_OK;
        if (allow_stream && total <= stream_auto_limit(k.bytes, vals)) {
            *s = stream_default_shape(k.bytes, vals);
            return MP_OK;
        }
    }
    *s = default_merge_shape(k.bytes, vals, total);
    if (s->staging == MP_STAGE_STREAM) *s = builtin_merge_shape(k.bytes, vals);  // tuned, but splits are given
    if (plan && plan->staging == MP_STAGE_STREAM) *s = stream_default_shape(k.bytes, vals);
    if (plan) {
        if (plan->reserved != 0) return fail(MP_ERR_INVALID_ARG, "plan.reserved must be 0");
        if (plan->block_threads) s->nt = plan->block_threads;
        if (plan->items_per_thread) s->vt = plan->items_per_thread;
        if (plan->staging) {
            s->staging = plan->staging;
        } else if (!merge_shape_supported(k.bytes, vals, *s)) {
            // Automatic staging for a shape the default staging lacks.
            s->staging = MP_STAGE_VECTOR;
        }
    }
    const bool ok = s->staging == MP_STAGE_STREAM ? stream_shape_supported(*s)
                                                  : merge_shape_supported(k.bytes, vals, *s);
    if (!ok)
        return fail(MP_ERR_INVALID_ARG, plan == &forced
                                            ? "MP_FORCE_PLAN names an unsupported merge plan"
                                            : "unsupported merge plan (block_threads, items_per_thread, staging)");
    return MP_OK;
}

mp_status merge_prepare(mp_dtype dtype, const void* a, const uint32_t* av, int64_t na,
                        const void* b, const uint32_t* bv, int64_t nb, void* out, uint32_t* outv,
                        bool vals, const mp_plan* plan, const char* fn, MergeProblem* p, Shape* s,
                        bool allow_stream)
{
    KeyKind k;
    if (!key_kind(dtype, &k)) return fail(MP_ERR_UNSUPPORTED_DTYPE, std::string(fn) + ": unknown dtype");
    mp_status st = check_merge_args(k, a, av, na, b, bv, nb, out, outv, vals, fn);
    if (st != MP_OK) return st;
    st = resolve_shape(k, vals, na + nb, plan, s, allow_stream);
    if (st != MP_OK) return st;
    p->kind = k;
    p->vals = vals;
    p->a = a;
    p->b = b;
    p->av = av;
    p->bv = bv;
    p->out = out;
    p->outv = outv;
    p->na = na;
    p->nb = nb;
    p->run = 0;
    return MP_OK;
}

static mp_status merge_impl(mp_dtype dtype, const void* a, const uint32_t* av, int64_t na,
                            const void* b, const uint32_t* bv, int64_t nb, void* out,
                            uint32_t* outv, bool vals, const mp_plan* plan, cudaStream_t stream,
                            const char* fn, const int64_t* given_splits = nullptr)
{
    MergeProblem p;
    Shape s;
    mp_status st = merge_prepare(dtype, a, av, na, b, bv, nb, out, outv, vals, plan, fn, &p, &s,
                                 given_splits == nullptr);
    if (st != MP_OK) return st;
    if (s.staging == MP_STAGE_STREAM && given_splits)
        return fail(MP_ERR_INVALID_ARG, std::string(fn) + ": the streaming plan takes no split points");
    if (na + nb == 0) return MP_OK;
    if (s.staging == MP_STAGE_STREAM) {
        cudaError_t e = launch_merge_stream(p, s, stream);
        return e == cudaSuccess ? MP_OK : cuda_fail(e, fn);
    }
    if (given_splits) {
        if (((uintptr_t)given_splits & 7) != 0)
            return fail(MP_ERR_INVALID_ARG, std::string(fn) + ": a_split not 8-byte aligned");
        cudaError_t e = launch_merge_tiles(p, s, given_splits, stream);
        return e == cudaSuccess ? MP_OK : cuda_fail(e, fn);
    }
    const int64_t bounds = ceil_div(na + nb, s.tile()) + 1;
    int64_t* splits = nullptr;
    st = scratch_alloc((void**)&splits, (size_t)bounds * 8, stream);
    if (st != MP_OK) return st;
    cudaError_t e = launch_partition(p, s.tile(), splits, stream);
    if (e == cudaSuccess) e = launch_merge_tiles(p, s, splits, stream);
    scratch_free(splits, stream);
    if (e != cudaSuccess) return cuda_fail(e, fn);
    return MP_OK;
}

// ---------------------------------------------------------------------------
// Sortedness / NaN check.
// ---------------------------------------------------------------------------
template <class K>
__global__ void check_sorted_kernel(const K* x, int64_t n, Codec<K> c, bool is_f32, unsigned* flags)
{
    unsigned f = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const K v = x[i];
        if (is_f32 && ((uint32_t)v & 0x7FFFFFFFu) > 0x7F800000u) f |= 2u;
        if (i + 1 < n && key_enc(v, c) > key_enc(x[i + 1], c)) f |= 1u;
    }
    if (f) atomicOr(flags, f);
}

// ---------------------------------------------------------------------------
// End-to-end merge of host arrays, pipelined.  The inputs cross to the device
// in C chunks; after chunk i, A[0, X_i) and B[0, Y_i) have landed.  With
// x = X_i - 1 and y = Y_i - 1 (x = |A| once all of A has landed, likewise
// y), the prefix A[0, x) ∪ B[0, y) fixes the merged output up to
//   d_i = min(x + #{B[0, y) < A[x]},  y + #{A[0, x) <= B[y]})
// (the positions at which A[x] and B[y] would be emitted, ties taking A; a
// missing element counts as +inf; nothing is fixed while a nonempty side
// has no element landed), with a(d_i) = x when the first term is the
// smaller and d_i - y otherwise.  A one-thread cut kernel computes
// (d_i, a(d_i)); the outputs [d_{i-1}, d_i) are merged (Alg. 1 on that
// piece, Cor. 6) and copied back while later inputs are still arriving, so
// the input and output copies overlap.  Every copy starts and ends on a
// boundary of 1024 elements (but the last): copies that start off a 16-byte
// boundary ran the host link at 236 GB/s both ways together instead of 326.
// ---------------------------------------------------------------------------
template <class K>
__device__ int64_t count_less(const K* X, int64_t n, K v, Codec<K> c, bool or_equal)
{
    const K kv = key_enc(v, c);
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const K km = key_enc(X[mid], c);
        if (or_equal ? !(km > kv) : (km < kv))
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// xl, yl: elements of A and B landed so far.
template <class K>
__global__ void host_cut_kernel(const K* A, int64_t na, int64_t xl, const K* B, int64_t nb, int64_t yl,
                                Codec<K> c, int64_t* cut)
{
    constexpr int64_t INF = INT64_MAX;
    if ((xl == 0 && na > 0) || (yl == 0 && nb > 0)) {  // a side with nothing landed: nothing fixed
        cut[0] = 0;
        cut[1] = 0;
        __threadfence_system();
        return;
    }
    const int64_t x = xl < na ? xl - 1 : na, y = yl < nb ? yl - 1 : nb;
    const int64_t ra = x < na ? x + count_less(B, y, A[x], c, false) : INF;
    const int64_t rb = y < nb ? y + count_less(A, x, B[y], c, true) : INF;
    if (ra == INF && rb == INF) {
        cut[0] = na + nb;
        cut[1] = na;
    } else if (ra <= rb) {
        cut[0] = ra;
        cut[1] = x;
    } else {
        cut[0] = rb;
        cut[1] = rb - y;
    }
    __threadfence_system();  // cut may be host memory the host reads after the kernel
}

static cudaError_t launch_host_cut(const KeyKind& k, const void* A, int64_t na, int64_t x, const void* B,
                                   int64_t nb, int64_t y, int64_t* cut, cudaStream_t s)
{
    if (k.bytes == 4)
        host_cut_kernel<uint32_t><<<1, 1, 0, s>>>((const uint32_t*)A, na, x, (const uint32_t*)B, nb, y,
                                                  make_codec<uint32_t>(k.flip, k.fmask, k.inv), cut);
    else if (k.bytes == 8)
        host_cut_kernel<uint64_t><<<1, 1, 0, s>>>((const uint64_t*)A, na, x, (const uint64_t*)B, nb, y,
                                                  make_codec<uint64_t>(k.flip, k.fmask, k.inv), cut);
    else
        host_cut_kernel<u128><<<1, 1, 0, s>>>((const u128*)A, na, x, (const u128*)B, nb, y,
                                              make_codec<u128>(k.flip, k.fmask, k.inv), cut);
    return cudaGetLastError();
}

static mp_status host_merge_pipelined(mp_dtype dtype, const KeyKind& k, const void* a_keys,
                                      const uint32_t* a_vals, int64_t na, const void* b_keys,
                                      const uint32_t* b_vals, int64_t nb, void* out_keys, uint32_t* out_vals,
                                      bool vals, cudaStream_t s)
{
    static const char* fn = "mp_merge_pairs_host";
    const int64_t n = na + nb;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t kb = (size_t)k.bytes;
    const size_t row = kb + (vals ? 4 : 0);
    // Chunks of at least 64 MB of input (at most 32); small merges take one.
    const int nchunk = (int)std::min<int64_t>(32, std::max<int64_t>(1, (int64_t)((size_t)n * row >> 26)));
    const size_t off_b = al(na * kb), off_o = off_b + al(nb * kb), off_av = off_o + al(n * kb);
    const size_t off_bv = off_av + (vals ? al(na * 4) : 0), off_ov = off_bv + (vals ? al(nb * 4) : 0);
    const size_t total = off_ov + (vals ? al(n * 4) : 0);
    char* d = nullptr;
    mp_status st = scratch_alloc((void**)&d, total, s);
    if (st != MP_OK) return st;
    char* dA = d;
    char* dB = d + off_b;
    char* dO = d + off_o;
    uint32_t* dAV = vals ? (uint32_t*)(d + off_av) : nullptr;
    uint32_t* dBV = vals ? (uint32_t*)(d + off_bv) : nullptr;
    uint32_t* dOV = vals ? (uint32_t*)(d + off_ov) : nullptr;

    cudaStream_t s_in = nullptr, s_cut = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> ev_in(nchunk, nullptr), ev_cut(nchunk, nullptr), ev_merged(nchunk, nullptr);
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_cut, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming);
    for (int i = 0; i < nchunk && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&ev_in[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_cut[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_merged[i], cudaEventDisableTiming);
    }
    // Everything starts after the scratch allocation on the caller's stream.
    if (e == cudaSuccess) e = cudaEventRecord(ev_start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_in, ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ev_start, 0);

    // Input chunk i: A[X_{i-1}, X_i), B[Y_{i-1}, Y_i), boundaries on multiples
    // of ALIGN elements (the last at the end).
    constexpr int64_t ALIGN = 1024;
    auto bound = [&](int64_t len, int i) -> int64_t {
        if (i < 0) return 0;
        if (i == nchunk - 1) return len;
        return (int64_t)((double)len * (i + 1) / nchunk) / ALIGN * ALIGN;
    };
    auto xa = [&](int i) { return bound(na, i); };
    auto yb = [&](int i) { return bound(nb, i); };
    auto copy_in = [&](const void* src, char* dst, size_t esz, int64_t lo, int64_t hi) -> cudaError_t {
        if (hi <= lo) return cudaSuccess;
        return cudaMemcpyAsync(dst + lo * esz, (const char*)src + lo * esz, (size_t)(hi - lo) * esz,
                               cudaMemcpyHostToDevice, s_in);
    };
    // Per-thread landing place for the cuts: pinned host memory that the cut
    // kernel writes directly (mapped), so no cut waits behind a bulk copy on
    // the copy engines.
    static thread_local int64_t* h_cut = nullptr;
    static thread_local int64_t* h_cut_dev = nullptr;
    if (e == cudaSuccess && !h_cut) {
        e = cudaHostAlloc((void**)&h_cut, 32 * 16, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&h_cut_dev, h_cut, 0);
    }
    for (int i = 0; i < nchunk && e == cudaSuccess; ++i) {
        const int64_t a_lo = xa(i - 1), a_hi = xa(i);
        const int64_t b_lo = yb(i - 1), b_hi = yb(i);
        e = copy_in(a_keys, dA, kb, a_lo, a_hi);
        if (e == cudaSuccess) e = copy_in(b_keys, dB, kb, b_lo, b_hi);
        if (vals && e == cudaSuccess) e = copy_in(a_vals, (char*)dAV, 4, a_lo, a_hi);
        if (vals && e == cudaSuccess) e = copy_in(b_vals, (char*)dBV, 4, b_lo, b_hi);
        if (e == cudaSuccess) e = cudaEventRecord(ev_in[i], s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_cut, ev_in[i], 0);
        if (e == cudaSuccess) e = launch_host_cut(k, dA, na, xa(i), dB, nb, yb(i), h_cut_dev + 2 * i, s_cut);
        if (e == cudaSuccess) e = cudaEventRecord(ev_cut[i], s_cut);
    }
    // Merge and copy out each settled piece of the output as soon as its cut
    // is known (the host reads each cut; the copies keep running meanwhile).
    // The copy back stops at the last multiple of ALIGN merged so far (all
    // of the output after the last chunk).
    int64_t d_prev = 0, a_prev = 0, out_copied = 0;
    cudaEvent_t last_merge = nullptr;  // the latest merge issued (merges run in order on s)
    for (int i = 0; i < nchunk && e == cudaSuccess && st == MP_OK; ++i) {
        e = cudaEventSynchronize(ev_cut[i]);
        if (e != cudaSuccess) break;
        const int64_t d_i = h_cut[2 * i], a_i = h_cut[2 * i + 1];
        if (d_i < d_prev || a_i < a_prev || d_i > n || a_i > na || d_i - a_i > nb) {
            st = fail(MP_ERR_INTERNAL, "mp_merge_pairs_host: inconsistent chunk cut (inputs not sorted?)");
            break;
        }
        if (d_i > d_prev) {
            const int64_t b_prev = d_prev - a_prev, b_i = d_i - a_i;
            e = cudaStreamWaitEvent(s, ev_cut[i], 0);
            if (e != cudaSuccess) break;
            st = merge_impl(dtype, dA + a_prev * kb, vals ? dAV + a_prev : nullptr, a_i - a_prev,
                            dB + b_prev * kb, vals ? dBV + b_prev : nullptr, b_i - b_prev, dO + d_prev * kb,
                            vals ? dOV + d_prev : nullptr, vals, nullptr, s, fn);
            if (st != MP_OK) break;
            e = cudaEventRecord(ev_merged[i], s);
            if (e != cudaSuccess) break;
            last_merge = ev_merged[i];
        }
        const int64_t out_to = i == nchunk - 1 ? d_i : d_i / ALIGN * ALIGN;
        if (out_to > out_copied) {
            e = cudaStreamWaitEvent(s_out, last_merge, 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync((char*)out_keys + out_copied * kb, dO + out_copied * kb,
                                    (size_t)(out_to - out_copied) * kb, cudaMemcpyDeviceToHost, s_out);
            if (vals && e == cudaSuccess)
                e = cudaMemcpyAsync(out_vals + out_copied, dOV + out_copied, (size_t)(out_to - out_copied) * 4,
                                    cudaMemcpyDeviceToHost, s_out);
            out_copied = out_to;
        }
        d_prev = d_i;
        a_prev = a_i;
    }
    if (e == cudaSuccess && st == MP_OK && d_prev != n)
        st = fail(MP_ERR_INTERNAL, "mp_merge_pairs_host: chunks did not cover the output");
    // The scratch is freed on the caller's stream after every copy and cut.
    cudaError_t e2 = cudaEventRecord(ev_done, s_out);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, ev_done, 0);
    if (e2 == cudaSuccess) e2 = cudaEventRecord(ev_done, s_cut);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, ev_done, 0);
    if (e2 == cudaSuccess) e2 = cudaEventRecord(ev_done, s_in);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, ev_done, 0);
    scratch_free(d, s);
    const cudaError_t e3 = cudaStreamSynchronize(s);
    for (int i = 0; i < nchunk; ++i) {
        if (ev_in[i]) cudaEventDestroy(ev_in[i]);
        if (ev_cut[i]) cudaEventDestroy(ev_cut[i]);
        if (ev_merged[i]) cudaEventDestroy(ev_merged[i]);
    }
    if (ev_start) cudaEventDestroy(ev_start);
    if (ev_done) cudaEventDestroy(ev_done);
    if (s_in) cudaStreamDestroy(s_in);
    if (s_cut) cudaStreamDestroy(s_cut);
    if (s_out) cudaStreamDestroy(s_out);
    if (st != MP_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, fn);
    if (e2 != cudaSuccess) return cuda_fail(e2, fn);
    if (e3 != cudaSuccess) return cuda_fail(e3, fn);
    return MP_OK;
}

}  // namespace mp

using namespace mp;

extern "C" {

const char* mp_status_string(mp_status s)
{
    switch (s) {
    case MP_OK: return "MP_OK";
    case MP_ERR_INVALID_ARG: return "MP_ERR_INVALID_ARG: invalid argument";
    case MP_ERR_UNSUPPORTED_DTYPE: return "MP_ERR_UNSUPPORTED_DTYPE: unsupported key dtype";
    case MP_ERR_NOT_SORTED: return "MP_ERR_NOT_SORTED: input is not sorted ascending";
    case MP_ERR_NAN: return "MP_ERR_NAN: float key is NaN";
    case MP_ERR_NO_MEMORY: return "MP_ERR_NO_MEMORY: allocation failed";
    case MP_ERR_BUDGET: return "MP_ERR_BUDGET: request exceeds the memory budget";
    case MP_ERR_TIMEOUT: return "MP_ERR_TIMEOUT: wait timed out";
    case MP_ERR_CUDA: return "MP_ERR_CUDA: CUDA runtime error";
    case MP_ERR_INTERNAL: return "MP_ERR_INTERNAL: internal error";
    case MP_ERR_NOT_READY: return "MP_ERR_NOT_READY: result not ready";
    }
    return "unknown mp_status";
}

const char* mp_last_error(void) { return g_last_error.c_str(); }

size_t mp_dtype_size(mp_dtype dtype)
{
    KeyKind k;
    return key_kind(dtype, &k) ? (size_t)k.bytes : 0;
}

mp_status mp_merge_keys(mp_dtype dtype, const void* a, int64_t na, const void* b, int64_t nb,
                        void* out, mp_stream_t stream)
{
    MP_RANGE("mp_merge_keys");
    return merge_impl(dtype, a, nullptr, na, b, nullptr, nb, out, nullptr, false, nullptr,
                      (cudaStream_t)stream, "mp_merge_keys");
}

mp_status mp_merge_pairs(mp_dtype dtype, const void* a_keys, const uint32_t* a_vals, int64_t na,
                         const void* b_keys, const uint32_t* b_vals, int64_t nb, void* out_keys,
                         uint32_t* out_vals, mp_stream_t stream)
{
    MP_RANGE("mp_merge_pairs");
    return merge_impl(dtype, a_keys, a_vals, na, b_keys, b_vals, nb, out_keys, out_vals, true, nullptr,
                      (cudaStream_t)stream, "mp_merge_pairs");
}

mp_status mp_merge_plan(mp_dtype dtype, const void* a_keys, const uint32_t* a_vals, int64_t na,
                        const void* b_keys, const uint32_t* b_vals, int64_t nb, void* out_keys,
                        uint32_t* out_vals, const mp_plan* plan, mp_stream_t stream)
{
    MP_RANGE("mp_merge_plan");
    const bool vals = a_vals || b_vals || out_vals;
    return merge_impl(dtype, a_keys, a_vals, na, b_keys, b_vals, nb, out_keys, out_vals, vals, plan,
                      (cudaStream_t)stream, "mp_merge_plan");
}

int mp_plan_supported(const mp_plan* plan)
{
    if (!plan || plan->reserved) return 0;
    Shape s{plan->block_threads, plan->items_per_thread,
            plan->staging ? plan->staging : MP_STAGE_VECTOR};
    if (s.staging == MP_STAGE_STREAM) return stream_shape_supported(s) ? 1 : 0;
    return merge_shape_supported(4, false, s) ? 1 : 0;
}

mp_status mp_merge_resolve_plan(mp_dtype dtype, int with_values, int64_t total, const mp_plan* plan,
                                mp_plan* resolved)
{
    KeyKind k;
    if (!key_kind(dtype, &k)) return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_merge_resolve_plan: unknown dtype");
    if (!resolved) return fail(MP_ERR_INVALID_ARG, "mp_merge_resolve_plan: NULL result");
    Shape s;
    const mp_status st = resolve_shape(k, with_values != 0, total, plan, &s);
    if (st != MP_OK) return st;
    *resolved = mp_plan{s.nt, s.vt, s.staging, 0};
    return MP_OK;
}

int64_t mp_merge_tile_items(mp_dtype dtype, int with_values, int64_t total, const mp_plan* plan)
{
    KeyKind k;
    if (!key_kind(dtype, &k)) return 0;
    Shape s;
    if (resolve_shape(k, with_values != 0, total, plan, &s, false) != MP_OK) return 0;
    return s.tile();
}

mp_status mp_merge_partitioned(mp_dtype dtype, const void* a_keys, const uint32_t* a_vals, int64_t na,
                               const void* b_keys, const uint32_t* b_vals, int64_t nb, void* out_keys,
                               uint32_t* out_vals, const int64_t* a_split, const mp_plan* plan,
                               mp_stream_t stream)
{
    MP_RANGE("mp_merge_partitioned");
    if (na + nb > 0 && !a_split) return fail(MP_ERR_INVALID_ARG, "mp_merge_partitioned: NULL a_split");
    const bool vals = a_vals || b_vals || out_vals;
    return merge_impl(dtype, a_keys, a_vals, na, b_keys, b_vals, nb, out_keys, out_vals, vals, plan,
                      (cudaStream_t)stream, "mp_merge_partitioned", a_split);
}

mp_status mp_merge_pairs_host(mp_dtype dtype, const void* a_keys, const uint32_t* a_vals, int64_t na,
                              const void* b_keys, const uint32_t* b_vals, int64_t nb, void* out_keys,
                              uint32_t* out_vals, mp_stream_t stream)
{
    MP_RANGE("mp_merge_pairs_host");
    KeyKind k;
    if (!key_kind(dtype, &k)) return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_merge_pairs_host: unknown dtype");
    const bool vals = a_vals || b_vals || out_vals;
    mp_status st = check_merge_args(k, a_keys, a_vals, na, b_keys, b_vals, nb, out_keys, out_vals,
                                    vals, "mp_merge_pairs_host");
    if (st != MP_OK) return st;
    if (na + nb == 0) return MP_OK;
    return host_merge_pipelined(dtype, k, a_keys, a_vals, na, b_keys, b_vals, nb, out_keys, out_vals, vals,
                                (cudaStream_t)stream);
}

mp_status mp_merge_checksum(mp_dtype dtype, const void* a_keys, const uint32_t* a_vals, int64_t na,
                            const void* b_keys, const uint32_t* b_vals, int64_t nb, uint64_t* checksum,
                            mp_stream_t stream)
{
    MP_RANGE("mp_merge_checksum");
    KeyKind k;
    if (!key_kind(dtype, &k) || k.bytes == 16)
        return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_merge_checksum: unknown or 128-bit dtype");
    if (!checksum || ((uintptr_t)checksum & 7)) return fail(MP_ERR_INVALID_ARG, "mp_merge_checksum: checksum must be an aligned device pointer");
    const bool vals = a_vals || b_vals;
    if (na < 0 || nb < 0) return fail(MP_ERR_INVALID_ARG, "mp_merge_checksum: negative size");
    if ((na > 0 && !a_keys) || (nb > 0 && !b_keys))
        return fail(MP_ERR_INVALID_ARG, "mp_merge_checksum: NULL key pointer");
    if (!aligned(a_keys, k.bytes) || !aligned(b_keys, k.bytes))
        return fail(MP_ERR_INVALID_ARG, "mp_merge_checksum: key pointer not aligned to the key size");
    if (vals && ((na > 0 && !a_vals) || (nb > 0 && !b_vals)))
        return fail(MP_ERR_INVALID_ARG, "mp_merge_checksum: NULL value array for a non-empty side");
    if (vals && (!aligned(a_vals, 4) || !aligned(b_vals, 4)))
        return fail(MP_ERR_INVALID_ARG, "mp_merge_checksum: value pointer not 4-byte aligned");
    mp_status st = MP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(checksum, 0, 8, s);
    if (e != cudaSuccess) return cuda_fail(e, "mp_merge_checksum");
    if (na + nb == 0) return MP_OK;
    MergeProblem p = {};
    p.kind = k;
    p.vals = vals;
    p.a = a_keys;
    p.b = b_keys;
    p.av = a_vals;
    p.bv = b_vals;
    p.na = na;
    p.nb = nb;
    const int64_t T = checksum_tile(k.bytes, vals);
    const int64_t bounds = ceil_div(na + nb, T) + 1;
    int64_t* splits = nullptr;
    // Split points, then one partial digest per tile.
    st = scratch_alloc((void**)&splits, (size_t)bounds * 16, s);
    if (st != MP_OK) return st;
    e = launch_partition(p, T, splits, s);
    if (e == cudaSuccess)
        e = launch_merge_checksum(p, splits, (unsigned long long*)(splits + bounds),
                                  (unsigned long long*)checksum, s);
    scratch_free(splits, s);
    return e == cudaSuccess ? MP_OK : cuda_fail(e, "mp_merge_checksum");
}

mp_status mp_merge_path_partition(mp_dtype dtype, const void* a, int64_t na, const void* b,
                                  int64_t nb, int64_t spacing, int64_t* a_split, mp_stream_t stream)
{
    MP_RANGE("mp_merge_path_partition");
    KeyKind k;
    if (!key_kind(dtype, &k)) return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_merge_path_partition: unknown dtype");
    if (na < 0 || nb < 0 || spacing < 1) return fail(MP_ERR_INVALID_ARG, "mp_merge_path_partition: bad size or spacing");
    if ((na > 0 && !a) || (nb > 0 && !b) || !a_split)
        return fail(MP_ERR_INVALID_ARG, "mp_merge_path_partition: NULL pointer");
    if (!aligned(a, k.bytes) || !aligned(b, k.bytes) || !aligned(a_split, 8))
        return fail(MP_ERR_INVALID_ARG, "mp_merge_path_partition: misaligned pointer");
    if (na + nb == 0) {
        cudaError_t e = cudaMemsetAsync(a_split, 0, 8, (cudaStream_t)stream);
        return e == cudaSuccess ? MP_OK : cuda_fail(e, "mp_merge_path_partition");
    }
    MergeProblem p = {};
    p.kind = k;
    p.vals = false;
    p.a = a;
    p.b = b;
    p.na = na;
    p.nb = nb;
    cudaError_t e = launch_partition(p, spacing, a_split, (cudaStream_t)stream);
    return e == cudaSuccess ? MP_OK : cuda_fail(e, "mp_merge_path_partition");
}

size_t mp_sort_workspace_bytes(mp_dtype dtype, int64_t n, int with_values)
{
    KeyKind k;
    if (!key_kind(dtype, &k) || n < 0) return 0;
    return sort_workspace_bytes(k, n, with_values != 0);
}

mp_status mp_sort(mp_dtype dtype, void* keys, uint32_t* vals, int64_t n, void* workspace,
                  size_t workspace_bytes, mp_stream_t stream)
{
    MP_RANGE("mp_sort");
    KeyKind k;
    if (!key_kind(dtype, &k)) return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_sort: unknown dtype");
    if (n < 0) return fail(MP_ERR_INVALID_ARG, "mp_sort: negative size");
    if (n <= 1) return MP_OK;
    if (!keys) return fail(MP_ERR_INVALID_ARG, "mp_sort: NULL keys");
    if (!aligned(keys, k.bytes) || (vals && !aligned(vals, 4)))
        return fail(MP_ERR_INVALID_ARG, "mp_sort: misaligned pointer");
    const size_t kb = (size_t)n * k.bytes;
    if (vals && overlaps(keys, kb, vals, (size_t)n * 4))
        return fail(MP_ERR_INVALID_ARG, "mp_sort: keys and values overlap");
    if (overlaps(workspace, workspace_bytes, keys, kb) ||
        (vals && overlaps(workspace, workspace_bytes, vals, (size_t)n * 4)))
        return fail(MP_ERR_INVALID_ARG, "mp_sort: workspace overlaps the data");
    return sort_run(k, keys, vals, n, workspace, workspace_bytes, (cudaStream_t)stream);
}

mp_status mp_check_sorted(mp_dtype dtype, const void* keys, int64_t n, mp_stream_t stream)
{
    MP_RANGE("mp_check_sorted");
    KeyKind k;
    if (!key_kind(dtype, &k)) return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_check_sorted: unknown dtype");
    if (n < 0 || (n > 0 && !keys)) return fail(MP_ERR_INVALID_ARG, "mp_check_sorted: bad arguments");
    if (!aligned(keys, k.bytes)) return fail(MP_ERR_INVALID_ARG, "mp_check_sorted: misaligned pointer");
    if (n == 0) return MP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* flags = nullptr;
    mp_status st = scratch_alloc((void**)&flags, sizeof(unsigned), s);
    if (st != MP_OK) return st;
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(unsigned), s);
    const int threads = 256;
    int64_t blocks = ceil_div(n, threads);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (e == cudaSuccess) {
        if (k.bytes == 4)
            check_sorted_kernel<uint32_t><<<(unsigned)blocks, threads, 0, s>>>(
                (const uint32_t*)keys, n,
                Codec<uint32_t>{(uint32_t)k.flip, (uint32_t)k.fmask, (uint32_t)k.inv},
                ((int)dtype & 0xFF) == MP_F32, flags);
        else if (k.bytes == 8)
            check_sorted_kernel<uint64_t><<<(unsigned)blocks, threads, 0, s>>>(
                (const uint64_t*)keys, n, Codec<uint64_t>{k.flip, k.fmask, k.inv}, false, flags);
        else
            check_sorted_kernel<u128><<<(unsigned)blocks, threads, 0, s>>>(
                (const u128*)keys, n, make_codec<u128>(k.flip, k.fmask, k.inv), false, flags);
        e = cudaGetLastError();
    }
    unsigned host_flags = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_flags, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    scratch_free(flags, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "mp_check_sorted");
    if (host_flags & 2u) return fail(MP_ERR_NAN, "mp_check_sorted: NaN key");
    if (host_flags & 1u) return fail(MP_ERR_NOT_SORTED, "mp_check_sorted: keys out of order");
    return MP_OK;
}


mp_status mp_inject_fault(mp_fault kind, int64_t count)
{
    if (count < 0) return fail(MP_ERR_INVALID_ARG, "mp_inject_fault: negative count");
    switch (kind) {
    case MP_FAULT_SCRATCH_ALLOC:
    case MP_FAULT_QUEUE_STEP:
        g_fault_count[kind].store(count);
        return MP_OK;
    case MP_FAULT_STAGE_WAIT: {
        cudaError_t e = set_stage_wait_fault(count > 0);
        return e == cudaSuccess ? MP_OK : cuda_fail(e, "mp_inject_fault");
    }
    }
    return fail(MP_ERR_INVALID_ARG, "mp_inject_fault: unknown fault kind");
}

}  // extern "C"
