// merge.cu -- the partition kernel and the merge-tile kernel.
//
// Alg. 1 (Parallel Merge) on a GPU: the output is cut into tiles of
// T = NT * VT elements.  The partition kernel finds, for every tile
// boundary d = t*T, where the Merge Path crosses cross diagonal d (Alg. 2,
// Thm 9); the merge kernel then gives each tile to one CTA (Cor. 6: the
// tiles merge independently and concatenate), stages the tile's A and B
// windows in shared memory (Lemma 16), repeats the diagonal search inside
// the window for each thread's VT outputs (Thm 17), merges them serially in
// registers and writes the tile back with coalesced 128-bit stores.
#include <algorithm>
#include <vector>

#include "mp_device.cuh"
#include "mp_internal.h"
#include "mp_tile.cuh"
#include "mp_bulk.cuh"

namespace mp {

// Word 0: the kernel error flags (mp_kernel_error).  Word 1: the
// staging-wait fault switch (mp_inject_fault, MP_FAULT_STAGE_WAIT).
__device__ unsigned int g_mp_kernel_error[2] = {0, 0};

// ---------------------------------------------------------------------------
// Partition: one thread per tile boundary, binary search along the diagonal
// in global memory (Alg. 2; at most ceil(log2(min(|A|,|B|)+1)) probes, Thm 14).
//
// The search runs in two stages.  The split a(d) is the first a in
// [lo, hi) with A[a] > B[d-1-a] (else hi), and that test is monotone in a,
// so it can first be narrowed over the candidates a = jT only, then
// finished inside the one interval ((j-1)T, jT] left.  With d = tT (every
// tile boundary, also inside a sort pass's run pair) the first stage probes
// A[jT] and B[(t-j)T - 1]: every T-th element of each side, a set shared by
// all boundaries and held in L2, so only the second stage's probes (inside
// one T-wide window per side) go to DRAM.  The result is the same split.
// ---------------------------------------------------------------------------
template <class FA, class FB>
__device__ __forceinline__ int64_t diagonal_search_tiled(FA keyA, int64_t la, FB keyB, int64_t lb,
                                                         int64_t diag, int64_t T)
{
    int64_t lo = diag - lb > 0 ? diag - lb : 0;
    int64_t hi = diag < la ? diag : la;
    if (lo < hi && T > 1) {
        // Candidates jT in [lo, hi): j in [jlo, jhi].
        const int64_t jlo = (lo + T - 1) / T, jhi = (hi - 1) / T;
        int64_t a = jlo, b = jhi + 1;
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (keyA(m * T) > keyB(diag - 1 - m * T))
                b = m;
            else
                a = m + 1;
        }
        // The test holds at aT (if a <= jhi) and fails at (a-1)T (if a > jlo).
        if (a <= jhi) hi = a * T;
        if (a > jlo) lo = (a - 1) * T + 1;
    }
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keyA(mid) > keyB(diag - 1 - mid))
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

template <class K>
__device__ __forceinline__ int64_t partition_point_tiled(const TileArgs<K>& p, int64_t d, int64_t T)
{
    d = d < p.total ? d : p.total;
    const Pair<K> q = pair_at(p, d < p.total ? d : p.total - 1);
    const K* A = q.A;
    const K* B = q.B;
    const Codec<K> c = p.codec;
    return diagonal_search_tiled([&](int64_t i) { return key_enc(ld_global_nc(A + i), c); }, q.na,
                                 [&](int64_t i) { return key_enc(ld_global_nc(B + i), c); }, q.nb,
                                 d - q.base, T);
}

template <class K>
__global__ void __launch_bounds__(256) partition_kernel(TileArgs<K> p, int64_t spacing,
                                                        int64_t n_bounds, int64_t* a_split)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_bounds) a_split[t] = partition_point_tiled(p, t * spacing, spacing);
    // Let a dependent merge launch (programmatic dependent launch) start its
    // prologue; it waits on griddepcontrol.wait before reading a_split.
    asm volatile("griddepcontrol.launch_dependents;");
}

// ---------------------------------------------------------------------------
// Merge tile kernel: one CTA per tile of NT*VT outputs.
// ---------------------------------------------------------------------------
template <class K, bool VALS, int NT, int VT, int CK>
__global__ void __launch_bounds__(NT) merge_tile_kernel(TileArgs<K> p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // Wait for the partition kernel (programmatic dependent launch).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    merge_tile_body<K, VALS, NT, VT, CK>(p, blockIdx.x, p.a_split, smem);
}

// TMA-staged tile merged warp-cooperatively (MP_STAGE_WARP).
template <class K, bool VALS, int NT, int VT, int CK>
__global__ void __launch_bounds__(NT) merge_tile_warp_kernel(TileArgs<K> p, unsigned int* err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    merge_tile_warp_body<K, VALS, NT, VT, CK>(p, blockIdx.x, p.a_split, smem, err);
}

// Sum of n partial digests into *sum (one CTA).
__global__ void __launch_bounds__(1024) sum_partials_kernel(const unsigned long long* partial, int64_t n,
                                                            unsigned long long* sum)
{
    __shared__ unsigned long long ws[32];
    unsigned long long acc = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        *sum = t;
    }
}

template <class K, bool VALS, int NT, int VT, int CK>
__global__ void __launch_bounds__(NT) merge_tile_checksum_kernel(TileArgs<K> p, unsigned int* err,
                                                                 unsigned long long* partial)
{
    extern __shared__ __align__(16) unsigned char smem[];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    merge_tile_checksum_body<K, VALS, NT, VT, CK>(p, blockIdx.x, p.a_split, smem, err, partial);
}

// Device address of the kernel error word on the current device.
unsigned int* kernel_error_word()
{
    static unsigned int* addr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_mp_kernel_error) != cudaSuccess) return nullptr;
        addr[dev] = static_cast<unsigned int*>(p);
    }
    return addr[dev];
}

cudaError_t set_stage_wait_fault(bool on)
{
    const unsigned int v = on ? 1u : 0u;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(g_mp_kernel_error, &v, sizeof v, sizeof(unsigned int));
    return e;
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
cudaError_t launch_partition(const MergeProblem& p, int64_t spacing, int64_t* a_split,
                             cudaStream_t stream)
{
    const int64_t n_bounds = ceil_div(p.total(), spacing) + 1;
    const int threads = 256;
    const int64_t blocks = ceil_div(n_bounds, threads);
    if (p.kind.bytes == 4)
        partition_kernel<uint32_t><<<(unsigned)blocks, threads, 0, stream>>>(
            make_tile_args<uint32_t>(p, nullptr), spacing, n_bounds, a_split);
    else if (p.kind.bytes == 8)
        partition_kernel<uint64_t><<<(unsigned)blocks, threads, 0, stream>>>(
            make_tile_args<uint64_t>(p, nullptr), spacing, n_bounds, a_split);
    else
        partition_kernel<u128><<<(unsigned)blocks, threads, 0, stream>>>(
            make_tile_args<u128>(p, nullptr), spacing, n_bounds, a_split);
    return cudaGetLastError();
}

template <class K, bool VALS, int NT, int VT, int CK>
static cudaError_t launch_tiles_ck(const MergeProblem& p, const int64_t* a_split, cudaStream_t stream)
{
    using SM = TileSmem<K, VALS, NT, VT>;
    auto kern = merge_tile_kernel<K, VALS, NT, VT, CK>;
    static bool configured = false;  // attribute is per function, set once
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SM::bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int64_t tiles = ceil_div(p.total(), (int64_t)NT * VT);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)tiles);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = SM::bytes;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, make_tile_args<K>(p, a_split));
}

// Unsigned keys compare as they are; other dtypes go through the codec.
template <class K, bool VALS, int NT, int VT>
static cudaError_t launch_tiles_t(const MergeProblem& p, const int64_t* a_split, cudaStream_t stream)
{
    if (p.kind.identity())
        return launch_tiles_ck<K, VALS, NT, VT, CODEC_IDENTITY>(p, a_split, stream);
    return launch_tiles_ck<K, VALS, NT, VT, CODEC_RUNTIME>(p, a_split, stream);
}

template <class K, bool VALS, int NT, int VT, int CK>
static cudaError_t launch_warp_ck(const MergeProblem& p, const int64_t* a_split, cudaStream_t stream)
{
    using SM = WarpSmem<K, VALS, NT, VT>;
    auto kern = merge_tile_warp_kernel<K, VALS, NT, VT, CK>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    unsigned int* err = kernel_error_word();
    if (!err) return cudaErrorInvalidSymbol;
    const int64_t tiles = ceil_div(p.total(), (int64_t)NT * VT);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)tiles);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = SM::bytes;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, make_tile_args<K>(p, a_split), err);
}

template <class K, bool VALS, int NT, int VT>
static cudaError_t launch_warp_t(const MergeProblem& p, const int64_t* a_split, cudaStream_t stream)
{
    if (p.kind.identity()) return launch_warp_ck<K, VALS, NT, VT, CODEC_IDENTITY>(p, a_split, stream);
    return launch_warp_ck<K, VALS, NT, VT, CODEC_RUNTIME>(p, a_split, stream);
}

// Compiled tile shapes (NT, VT) of the register-staged and warp-cooperative
// tiles.  The TMA bulk shapes (MP_BULK_SHAPES, MP_WIDE_SHAPES) are listed in
// mp_internal.h; their kernels live in merge_bulk.cu.
#define MP_MERGE_SHAPES(X) X(128, 8) X(256, 8) X(128, 16) X(256, 16) X(512, 8)
#define MP_WARP_SHAPES(X) X(128, 8) X(256, 8) X(128, 16) X(256, 16)

bool merge_shape_supported(int key_bytes, bool with_values, const Shape& s)
{
    (void)with_values;
    if (key_bytes == 16) {
#define X(NT_, VT_) if (s.staging == MP_STAGE_BULK && s.nt == NT_ && s.vt == VT_) return true;
        MP_WIDE_SHAPES(X)
#undef X
        return false;
    }
    if (key_bytes != 4 && key_bytes != 8) return false;
#define X(NT_, VT_) if (s.nt == NT_ && s.vt == VT_) return true;
    if (s.staging == MP_STAGE_VECTOR) {
        MP_MERGE_SHAPES(X)
    } else if (s.staging == MP_STAGE_BULK) {
        MP_BULK_SHAPES(X)
    } else if (s.staging == MP_STAGE_WARP) {
        MP_WARP_SHAPES(X)
    }
#undef X
    return false;
}

std::vector<Shape> merge_shapes()
{
    std::vector<Shape> v;
#define X(NT_, VT_) v.push_back(Shape{NT_, VT_, MP_STAGE_VECTOR});
    MP_MERGE_SHAPES(X)
#undef X
#define X(NT_, VT_) v.push_back(Shape{NT_, VT_, MP_STAGE_BULK});
    MP_BULK_SHAPES(X)
#undef X
    // MP_STAGE_WARP is left out: on every workload measured it ran at less
    // than half the speed of the thread-serial TMA tile, so tuning it only
    // costs time.
    return v;
}

Shape default_merge_shape(int key_bytes, bool with_values, int64_t total)
{
    Shape s;
    if (tuned_shape("merge", key_bytes, with_values, total, &s)) return s;
    return builtin_merge_shape(key_bytes, with_values);
}

Shape builtin_merge_shape(int key_bytes, bool with_values)
{
    Shape s;
    // Shapes with the shortest partition + merge step on GB300 for large
    // merges (tile-shape sweep), all TMA-staged (no staging registers, so
    // more CTAs stay resident).  An odd number of outputs per thread starts
    // the threads' serial walks in different shared-memory banks and, with
    // more outputs per thread, spreads each thread's diagonal search over
    // more outputs: 4-byte keys alone take 128 x 33 (2 x 2^27 int32 keys:
    // 0.457 ms against 0.468 ms at 256 x 33), 8-byte keys alone 128 x 27.  Keys with values keep 12 per thread (256 x 12), where the
    // larger tile would leave fewer CTAs per SM.  mp_autotune_merge
    // overrides per size class.
    s.staging = MP_STAGE_BULK;
    if (key_bytes == 16) {
        s.nt = 128;
        s.vt = 12;
    } else if (with_values) {
        s.nt = 256;
        s.vt = 12;
    } else if (key_bytes == 8) {
        s.nt = 128;
        s.vt = 27;
    } else {
        s.nt = 128;
        s.vt = 33;
    }
    return s;
}

cudaError_t launch_merge_tiles(const MergeProblem& p, const Shape& s, const int64_t* a_split,
                               cudaStream_t stream)
{
    const bool vals = p.vals;
    if (p.kind.bytes == 16 || s.staging == MP_STAGE_BULK) return launch_merge_bulk(p, s, a_split, stream);
    if (s.staging == MP_STAGE_WARP) {
#define X(NT_, VT_)                                                                            \
        if (s.nt == NT_ && s.vt == VT_) {                                                      \
            if (p.kind.bytes == 4)                                                             \
                return vals ? launch_warp_t<uint32_t, true, NT_, VT_>(p, a_split, stream)      \
                            : launch_warp_t<uint32_t, false, NT_, VT_>(p, a_split, stream);    \
            return vals ? launch_warp_t<uint64_t, true, NT_, VT_>(p, a_split, stream)          \
                        : launch_warp_t<uint64_t, false, NT_, VT_>(p, a_split, stream);        \
        }
        MP_WARP_SHAPES(X)
#undef X
        return cudaErrorInvalidValue;
    }
#define X(NT_, VT_)                                                                            \
    if (s.nt == NT_ && s.vt == VT_) {                                                          \
        if (p.kind.bytes == 4)                                                                 \
            return vals ? launch_tiles_t<uint32_t, true, NT_, VT_>(p, a_split, stream)         \
                        : launch_tiles_t<uint32_t, false, NT_, VT_>(p, a_split, stream);       \
        return vals ? launch_tiles_t<uint64_t, true, NT_, VT_>(p, a_split, stream)             \
                    : launch_tiles_t<uint64_t, false, NT_, VT_>(p, a_split, stream);           \
    }
    MP_MERGE_SHAPES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace mp

extern "C" mp_status mp_kernel_error(unsigned int* code, int reset)
{
    unsigned int v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, mp::g_mp_kernel_error, sizeof v);
    if (e == cudaSuccess && reset) {
        unsigned int z = 0;
        e = cudaMemcpyToSymbol(mp::g_mp_kernel_error, &z, sizeof z);
    }
    if (e != cudaSuccess) return mp::cuda_fail(e, "mp_kernel_error");
    if (code) *code = v;
    return MP_OK;
}

extern "C" mp_status mp_kernel_status(mp_stream_t stream, int reset)
{
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, mp::g_mp_kernel_error, sizeof v, 0,
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && reset && v) {
        const unsigned int z = 0;
        e = cudaMemcpyToSymbolAsync(mp::g_mp_kernel_error, &z, sizeof z, 0, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return mp::cuda_fail(e, "mp_kernel_status");
    if (v & MP_KERR_MBAR_TIMEOUT)
        return mp::fail(MP_ERR_TIMEOUT, "mp_kernel_status: a kernel's bounded wait for its staged "
                                        "tile ran out; that tile's output was not written");
    if (v & 4u)
        return mp::fail(MP_ERR_TIMEOUT, "mp_kernel_status: a set operation's bounded wait for an "
                                        "earlier tile's count ran out; its output is misplaced");
    if (v & 2u)
        return mp::fail(MP_ERR_NOT_SORTED, "mp_kernel_status: a set operation's tile output "
                                           "passed the capacity (inputs not sorted)");
    return MP_OK;
}

namespace mp {

template <class K, bool VALS, int CK>
static cudaError_t launch_checksum_t(const MergeProblem& p, const int64_t* a_split,
                                     unsigned long long* partial, unsigned long long* sum,
                                     cudaStream_t stream)
{
    constexpr int NT = 256, VT = VALS ? 8 : 16;
    using SM = BulkSmem<K, VALS, NT, VT>;
    auto kern = merge_tile_checksum_kernel<K, VALS, NT, VT, CK>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    unsigned int* err = kernel_error_word();
    if (!err) return cudaErrorInvalidSymbol;
    const int64_t tiles = ceil_div(p.total(), (int64_t)NT * VT);
    kern<<<(unsigned)tiles, NT, SM::bytes, stream>>>(make_tile_args<K>(p, a_split), err, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_partials_kernel<<<1, 1024, 0, stream>>>(partial, tiles, sum);
    return cudaGetLastError();
}

int64_t checksum_tile(int key_bytes, bool vals)
{
    (void)key_bytes;
    return 256 * (vals ? 8 : 16);
}

cudaError_t launch_merge_checksum(const MergeProblem& p, const int64_t* a_split,
                                  unsigned long long* partial, unsigned long long* sum,
                                  cudaStream_t stream)
{
    const bool id = p.kind.identity();
    if (p.kind.bytes == 4) {
        if (p.vals) return id ? launch_checksum_t<uint32_t, true, CODEC_IDENTITY>(p, a_split, partial, sum, stream)
                              : launch_checksum_t<uint32_t, true, CODEC_RUNTIME>(p, a_split, partial, sum, stream);
        return id ? launch_checksum_t<uint32_t, false, CODEC_IDENTITY>(p, a_split, partial, sum, stream)
                  : launch_checksum_t<uint32_t, false, CODEC_RUNTIME>(p, a_split, partial, sum, stream);
    }
    if (p.vals) return id ? launch_checksum_t<uint64_t, true, CODEC_IDENTITY>(p, a_split, partial, sum, stream)
                          : launch_checksum_t<uint64_t, true, CODEC_RUNTIME>(p, a_split, partial, sum, stream);
    return id ? launch_checksum_t<uint64_t, false, CODEC_IDENTITY>(p, a_split, partial, sum, stream)
              : launch_checksum_t<uint64_t, false, CODEC_RUNTIME>(p, a_split, partial, sum, stream);
}

}  // namespace mp
