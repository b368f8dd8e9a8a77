// sort.cu -- stable merge sort: block sort of tiles, then Merge Path passes.
//
// Sec. I / Sec. III: merge sort is a sequence of merge rounds; each core
// first sorts N/p elements on its own, then rounds of Parallel Merge run
// one after the other.  Here a CTA sorts one tile of NT*VT keys in shared
// memory (each thread sorts VT keys in registers, then log2(NT) rounds of
// in-CTA Merge Path merge runs of doubling width), and the remaining
// ceil(log2(tiles)) rounds are Merge Path passes over HBM (partition kernel
// + merge-tile kernel, see merge.cu) that ping-pong between the keys and a
// workspace.  Every step is stable, so the whole sort is.
#include <algorithm>

#include "mp_device.cuh"
#include "mp_internal.h"
#include "mp_sort.cuh"

namespace mp {

template <class K, bool VALS, int NT, int VT>
__global__ void __launch_bounds__(NT) block_sort_kernel(const K* in, const uint32_t* vin, K* out,
                                                        uint32_t* vout, int64_t n, Codec<K> c)
{
    extern __shared__ __align__(16) unsigned char smem[];
    block_sort_body<K, VALS, NT, VT>(in, vin, out, vout, n, c, blockIdx.x, smem);
}

// Block-sort tile shape per key width.
static constexpr int BS_NT = 512;
static constexpr int BS_VT4 = 16;  // 4-byte keys: tile 8192
static constexpr int BS_VT8 = 8;   // 8-byte keys: tile 4096
static constexpr int BS_VT16 = 4;  // 16-byte keys: tile 2048

static int64_t block_tile(int key_bytes)
{
    return (int64_t)BS_NT * (key_bytes == 16 ? BS_VT16 : (key_bytes == 8 ? BS_VT8 : BS_VT4));
}

static Shape sort_merge_shape(int key_bytes)
{
    // Tile of the merge passes: a power of two dividing 2 * block tile (a
    // tile lies inside one run pair).  4-byte keys 256 x 16, 8-byte keys
    // 128 x 16 (the same 2048-element tile as 256 x 8, merged faster),
    // 16-byte keys 128 x 8.
    Shape s;
    s.nt = key_bytes == 4 ? 256 : 128;
    s.vt = key_bytes == 16 ? 8 : 16;
    s.staging = MP_STAGE_BULK;
    return s;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int ceil_log2(int64_t x)
{
    int p = 0;
    while (((int64_t)1 << p) < x) ++p;
    return p;
}

size_t sort_workspace_bytes(const KeyKind& kind, int64_t n, bool with_values)
{
    if (n <= 1) return 0;
    const int64_t tiles = ceil_div(n, sort_merge_shape(kind.bytes).tile());
    return align256((size_t)n * kind.bytes) + (with_values ? align256((size_t)n * 4) : 0) +
           align256((size_t)(tiles + 1) * 8);
}

template <class K, bool VALS, int NT, int VT>
static cudaError_t launch_block_sort(const K* in, const uint32_t* vin, K* out, uint32_t* vout,
                                     int64_t n, const KeyKind& kind, cudaStream_t stream)
{
    using SM = SortSmem<K, VALS, NT, VT>;
    auto kern = block_sort_kernel<K, VALS, NT, VT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SM::bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const Codec<K> c = make_codec<K>(kind.flip, kind.fmask, kind.inv);
    const int64_t blocks = ceil_div(n, (int64_t)NT * VT);
    kern<<<(unsigned)blocks, NT, SM::bytes, stream>>>(in, vin, out, vout, n, c);
    return cudaGetLastError();
}

static cudaError_t block_sort(const KeyKind& kind, const void* in, const uint32_t* vin, void* out,
                              uint32_t* vout, int64_t n, cudaStream_t stream)
{
    if (kind.bytes == 4) {
        if (vin)
            return launch_block_sort<uint32_t, true, BS_NT, BS_VT4>(
                (const uint32_t*)in, vin, (uint32_t*)out, vout, n, kind, stream);
        return launch_block_sort<uint32_t, false, BS_NT, BS_VT4>(
            (const uint32_t*)in, nullptr, (uint32_t*)out, nullptr, n, kind, stream);
    }
    if (kind.bytes == 16) {
        if (vin)
            return launch_block_sort<u128, true, BS_NT, BS_VT16>((const u128*)in, vin, (u128*)out, vout, n, kind,
                                                                 stream);
        return launch_block_sort<u128, false, BS_NT, BS_VT16>((const u128*)in, nullptr, (u128*)out, nullptr, n,
                                                              kind, stream);
    }
    if (vin)
        return launch_block_sort<uint64_t, true, BS_NT, BS_VT8>(
            (const uint64_t*)in, vin, (uint64_t*)out, vout, n, kind, stream);
    return launch_block_sort<uint64_t, false, BS_NT, BS_VT8>(
        (const uint64_t*)in, nullptr, (uint64_t*)out, nullptr, n, kind, stream);
}

mp_status sort_run(const KeyKind& kind, void* keys, uint32_t* vals, int64_t n, void* ws,
                   size_t ws_bytes, cudaStream_t stream)
{
    if (n <= 1) return MP_OK;
    const bool with_vals = vals != nullptr;
    const size_t need = sort_workspace_bytes(kind, n, with_vals);
    if (ws == nullptr || ws_bytes < need)
        return fail(MP_ERR_INVALID_ARG, "mp_sort: workspace smaller than mp_sort_workspace_bytes()");
    if (((uintptr_t)ws & 255) != 0) return fail(MP_ERR_INVALID_ARG, "mp_sort: workspace not 256-byte aligned");

    char* w = static_cast<char*>(ws);
    void* ws_keys = w;
    w += align256((size_t)n * kind.bytes);
    uint32_t* ws_vals = nullptr;
    if (with_vals) {
        ws_vals = reinterpret_cast<uint32_t*>(w);
        w += align256((size_t)n * 4);
    }
    int64_t* splits = reinterpret_cast<int64_t*>(w);

    const int64_t bt = block_tile(kind.bytes);
    const int passes = ceil_log2(ceil_div(n, bt));
    // The block sort writes where an even number of passes later ends in keys.
    void* cur = (passes & 1) ? ws_keys : keys;
    uint32_t* curv = (passes & 1) ? ws_vals : vals;
    void* oth = (passes & 1) ? keys : ws_keys;
    uint32_t* othv = (passes & 1) ? vals : ws_vals;

    cudaError_t e = block_sort(kind, keys, vals, cur, curv, n, stream);
    if (e != cudaSuccess) return cuda_fail(e, "block sort launch");

    const Shape ms = sort_merge_shape(kind.bytes);
    for (int p = 0; p < passes; ++p) {
        MergeProblem mp;
        mp.kind = kind;
        mp.vals = with_vals;
        mp.a = cur;
        mp.b = cur;
        mp.av = curv;
        mp.bv = curv;
        mp.out = oth;
        mp.outv = othv;
        mp.na = n;
        mp.nb = 0;
        mp.run = bt << p;
        e = launch_partition(mp, ms.tile(), splits, stream);
        if (e != cudaSuccess) return cuda_fail(e, "sort pass partition launch");
        e = launch_merge_tiles(mp, ms, splits, stream);
        if (e != cudaSuccess) return cuda_fail(e, "sort pass merge launch");
        std::swap(cur, oth);
        std::swap(curv, othv);
    }
    if (cur != keys) return fail(MP_ERR_INTERNAL, "sort: result not in the key buffer");
    return MP_OK;
}

}  // namespace mp
