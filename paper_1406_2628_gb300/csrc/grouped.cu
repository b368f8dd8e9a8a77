// grouped.cu -- many independent merge / block-sort problems in one launch.
//
// A group is a list of problems, each with its own pointers, sizes and key
// codec (any dtypes of one key width).  Every problem is cut into tiles of
// T outputs (Alg. 1, Cor. 7); a problem's tiles never straddle problems, so
// each tile is an ordinary Merge Path segment of its own problem (Cor. 6).
// Tile t of the whole launch belongs to the problem whose tile range holds
// t (binary search over the problems' first tiles).  A merge problem may be
// a plain merge (run = 0) or one pass of a merge sort (run = width of the
// sorted runs being paired), so one launch can advance merges and sorts of
// many requests at once.
#include <algorithm>
#include <cstring>
#include <vector>

#include "mp_device.cuh"
#include "mp_internal.h"
#include "mp_sort.cuh"
#include "mp_tile.cuh"
#include "mp_bulk.cuh"

namespace mp {

// Index of the last problem whose first slot is <= x (first[0] == 0).
__device__ __forceinline__ int problem_of(const int64_t* first, int nprob, int64_t x)
{
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(first + mid) <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <class K>
__device__ __forceinline__ TileArgs<K> tile_args_of(const GroupMergeDesc& g)
{
    TileArgs<K> p;
    p.a = static_cast<const K*>(g.a);
    p.b = static_cast<const K*>(g.b);
    p.av = g.av;
    p.bv = g.bv;
    p.out = static_cast<K*>(g.out);
    p.outv = g.outv;
    p.na = g.na;
    p.nb = g.nb;
    p.run = g.run;
    p.total = g.run ? g.na : g.na + g.nb;
    p.a_split = nullptr;
    p.codec.flip = (K)g.flip;
    p.codec.fmask = (K)g.fmask;
    p.codec.inv = (K)g.inv;
    return p;
}

// One thread per (problem, boundary) slot; slot ranges per problem start at
// bound_first[p] = tile_first[p] + p.
template <class K>
__global__ void __launch_bounds__(256) grouped_partition_kernel(const GroupMergeDesc* descs,
                                                                const int64_t* bound_first,
                                                                int nprob, int64_t n_slots,
                                                                int64_t spacing, int64_t* splits)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n_slots) {
        const int p = problem_of(bound_first, nprob, g);
        const TileArgs<K> a = tile_args_of<K>(descs[p]);
        const int64_t t = g - __ldg(bound_first + p);
        splits[g] = a.total > 0 ? partition_point(a, t * spacing) : 0;
    }
    asm volatile("griddepcontrol.launch_dependents;");
}

// One tile of problem p per CTA, windows staged by TMA bulk copies.  CK is
// CODEC_IDENTITY when every problem of the launch has unsigned ascending
// keys, else the runtime codec (each problem carries its own).
template <class K, bool VALS, int NT, int VT, int CK>
__global__ void __launch_bounds__(NT) grouped_merge_bulk_kernel(const GroupMergeDesc* descs,
                                                                const int64_t* tile_first, int nprob,
                                                                const int64_t* splits, unsigned int* err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t tile = blockIdx.x;
    const int p = problem_of(tile_first, nprob, tile);
    const TileArgs<K> a = tile_args_of<K>(descs[p]);
    const int64_t first = __ldg(tile_first + p);
    merge_tile_bulk_body<K, VALS, NT, VT, CK>(a, tile - first, splits + first + p, smem, err);
}

template <class K, bool VALS, int NT, int VT>
__global__ void __launch_bounds__(NT) grouped_block_sort_kernel(const GroupSortDesc* descs,
                                                                const int64_t* tile_first, int nprob)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t tile = blockIdx.x;
    const int p = problem_of(tile_first, nprob, tile);
    const GroupSortDesc d = descs[p];
    Codec<K> c;
    c.flip = (K)d.flip;
    c.fmask = (K)d.fmask;
    c.inv = (K)d.inv;
    block_sort_body<K, VALS, NT, VT>(static_cast<const K*>(d.in), d.vin, static_cast<K*>(d.out),
                                     d.vout, d.n, c, tile - __ldg(tile_first + p), smem);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
template <class K, bool VALS, int NT, int VT, int CK>
static cudaError_t launch_grouped_merge_ck(const GroupMergeDesc* d_descs, const int64_t* d_tile_first,
                                           const int64_t* d_bound_first, int nprob,
                                           int64_t total_tiles, int64_t* d_splits, cudaStream_t stream)
{
    using SM = MergeBulkSmem<K, VALS, NT, VT>;
    auto kern = grouped_merge_bulk_kernel<K, VALS, NT, VT, CK>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    unsigned int* err = kernel_error_word();
    if (!err) return cudaErrorInvalidSymbol;
    const int64_t n_slots = total_tiles + nprob;
    grouped_partition_kernel<K><<<(unsigned)ceil_div(n_slots, 256), 256, 0, stream>>>(
        d_descs, d_bound_first, nprob, n_slots, (int64_t)NT * VT, d_splits);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || total_tiles == 0) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)total_tiles);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = SM::bytes;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, d_descs, d_tile_first, nprob, (const int64_t*)d_splits, err);
}

template <class K, bool VALS, int NT, int VT>
static cudaError_t launch_grouped_merge_t(const GroupMergeDesc* d_descs, const int64_t* d_tile_first,
                                          const int64_t* d_bound_first, int nprob, int64_t total_tiles,
                                          int64_t* d_splits, bool identity, cudaStream_t stream)
{
    if (identity)
        return launch_grouped_merge_ck<K, VALS, NT, VT, CODEC_IDENTITY>(d_descs, d_tile_first, d_bound_first,
                                                                        nprob, total_tiles, d_splits, stream);
    return launch_grouped_merge_ck<K, VALS, NT, VT, CODEC_RUNTIME>(d_descs, d_tile_first, d_bound_first, nprob,
                                                                   total_tiles, d_splits, stream);
}

// Grouped shapes: the default merge shapes of each key width.
int64_t grouped_merge_tile(int key_bytes) { return key_bytes == 8 ? 256 * 8 : 256 * 16; }
int64_t grouped_sort_tile(int key_bytes) { return key_bytes == 8 ? 256 * 8 : 256 * 16; }

cudaError_t launch_grouped_merge(int key_bytes, bool vals, const GroupMergeDesc* d_descs,
                                 const int64_t* d_tile_first, const int64_t* d_bound_first,
                                 int nprob, int64_t total_tiles, int64_t* d_splits, bool identity,
                                 cudaStream_t stream)
{
    if (nprob <= 0) return cudaSuccess;
    // TMA-staged tiles: 4-byte keys 256 x 16 (tile 4096, = the block-sort
    // tile, so sort passes pair whole runs), 8-byte keys 256 x 8 (2048).
    if (key_bytes == 4)
        return vals ? launch_grouped_merge_t<uint32_t, true, 256, 16>(d_descs, d_tile_first, d_bound_first, nprob, total_tiles, d_splits, identity, stream)
                    : launch_grouped_merge_t<uint32_t, false, 256, 16>(d_descs, d_tile_first, d_bound_first, nprob, total_tiles, d_splits, identity, stream);
    return vals ? launch_grouped_merge_t<uint64_t, true, 256, 8>(d_descs, d_tile_first, d_bound_first, nprob, total_tiles, d_splits, identity, stream)
                : launch_grouped_merge_t<uint64_t, false, 256, 8>(d_descs, d_tile_first, d_bound_first, nprob, total_tiles, d_splits, identity, stream);
}

template <class K, bool VALS, int NT, int VT>
static cudaError_t launch_grouped_sort_t(const GroupSortDesc* d_descs, const int64_t* d_tile_first,
                                         int nprob, int64_t total_tiles, cudaStream_t stream)
{
    using SM = SortSmem<K, VALS, NT, VT>;
    auto kern = grouped_block_sort_kernel<K, VALS, NT, VT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (total_tiles == 0) return cudaSuccess;
    kern<<<(unsigned)total_tiles, NT, SM::bytes, stream>>>(d_descs, d_tile_first, nprob);
    return cudaGetLastError();
}

cudaError_t launch_grouped_block_sort(int key_bytes, bool vals, const GroupSortDesc* d_descs,
                                      const int64_t* d_tile_first, int nprob, int64_t total_tiles,
                                      cudaStream_t stream)
{
    if (nprob <= 0) return cudaSuccess;
    if (key_bytes == 4)
        return vals ? launch_grouped_sort_t<uint32_t, true, 256, 16>(d_descs, d_tile_first, nprob, total_tiles, stream)
                    : launch_grouped_sort_t<uint32_t, false, 256, 16>(d_descs, d_tile_first, nprob, total_tiles, stream);
    return vals ? launch_grouped_sort_t<uint64_t, true, 256, 8>(d_descs, d_tile_first, nprob, total_tiles, stream)
                : launch_grouped_sort_t<uint64_t, false, 256, 8>(d_descs, d_tile_first, nprob, total_tiles, stream);
}

}  // namespace mp

using namespace mp;

extern "C" mp_status mp_merge_grouped(const mp_merge_desc* descs, int64_t nprob, int with_values,
                                      mp_stream_t stream)
{
    MP_RANGE("mp_merge_grouped");
    if (nprob < 0 || (nprob > 0 && !descs)) return fail(MP_ERR_INVALID_ARG, "mp_merge_grouped: bad descriptor array");
    if (nprob == 0) return MP_OK;
    if (nprob > (1 << 30)) return fail(MP_ERR_INVALID_ARG, "mp_merge_grouped: too many problems");
    KeyKind k0;
    if (!key_kind((mp_dtype)descs[0].dtype, &k0) || k0.bytes == 16)
        return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_merge_grouped: unknown or 128-bit dtype");
    const bool vals = with_values != 0;
    std::vector<GroupMergeDesc> h(nprob);
    std::vector<int64_t> first(2 * nprob);
    int64_t tiles = 0;
    bool all_identity = true;
    const int64_t T = grouped_merge_tile(k0.bytes);
    for (int64_t i = 0; i < nprob; ++i) {
        const mp_merge_desc& d = descs[i];
        KeyKind k;
        if (!key_kind((mp_dtype)d.dtype, &k) || k.bytes == 16)
            return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_merge_grouped: unknown or 128-bit dtype");
        if (k.bytes != k0.bytes) return fail(MP_ERR_INVALID_ARG, "mp_merge_grouped: key widths differ");
        mp_status st = check_merge_args_ext(k, d.a_keys, d.a_vals, d.na, d.b_keys, d.b_vals, d.nb,
                                            d.out_keys, d.out_vals, vals, "mp_merge_grouped");
        if (st != MP_OK) return st;
        GroupMergeDesc& g = h[i];
        g.a = d.a_keys;
        g.b = d.b_keys;
        g.av = d.a_vals;
        g.bv = d.b_vals;
        g.out = d.out_keys;
        g.outv = d.out_vals;
        g.na = d.na;
        g.nb = d.nb;
        g.run = 0;
        g.flip = k.flip;
        g.fmask = k.fmask;
        g.inv = k.inv;
        all_identity = all_identity && k.identity();
        first[i] = tiles;
        first[nprob + i] = tiles + i;
        tiles += ceil_div(d.na + d.nb, T);
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t desc_bytes = (((size_t)nprob * sizeof(GroupMergeDesc)) + 255) & ~(size_t)255;
    const size_t first_bytes = (((size_t)nprob * 16) + 255) & ~(size_t)255;
    const size_t split_bytes = (size_t)(tiles + nprob) * 8;
    char* d = nullptr;
    mp_status st = scratch_alloc((void**)&d, desc_bytes + first_bytes + split_bytes, s);
    if (st != MP_OK) return st;
    // The tables are copied from pageable memory: the copy is staged before
    // cudaMemcpyAsync returns, so the host vectors may go out of scope.
    std::vector<char> table(desc_bytes + first_bytes);
    memcpy(table.data(), h.data(), (size_t)nprob * sizeof(GroupMergeDesc));
    memcpy(table.data() + desc_bytes, first.data(), (size_t)nprob * 16);
    cudaError_t e = cudaMemcpyAsync(d, table.data(), table.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = launch_grouped_merge(k0.bytes, vals, (const GroupMergeDesc*)d, (const int64_t*)(d + desc_bytes),
                                 (const int64_t*)(d + desc_bytes) + nprob, (int)nprob, tiles,
                                 (int64_t*)(d + desc_bytes + first_bytes), all_identity, s);
    scratch_free(d, s);
    if (e != cudaSuccess) return cuda_fail(e, "mp_merge_grouped");
    return MP_OK;
}
