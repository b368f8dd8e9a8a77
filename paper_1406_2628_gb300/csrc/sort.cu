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
#include "mp_bulk.cuh"

namespace mp {

// ENC_OUT: the runs are written encoded (unsigned order), for the merge
// passes that follow.
template <class K, bool VALS, int NT, int VT, bool ENC_OUT>
__global__ void __launch_bounds__(NT) block_sort_kernel(const K* in, const uint32_t* vin, K* out,
                                                        uint32_t* vout, int64_t n, Codec<K> c,
                                                        unsigned int* err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    block_sort_body<K, VALS, NT, VT, ENC_OUT, true>(in, vin, out, vout, n, c, blockIdx.x, smem, err);
}

// The last merge pass of a sort whose runs are encoded: keys are compared
// as they are and decoded on output (an encoded-input codec kind CK); the
// tile is merge_tile_bulk_body's, as in every other pass.
template <class K, bool VALS, int NT, int VT, int CK>
__global__ void __launch_bounds__(NT) sort_last_pass_kernel(TileArgs<K> p, unsigned int* err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    merge_tile_bulk_body<K, VALS, NT, VT, CK>(p, blockIdx.x, p.a_split, smem, err);
}

// Per sort mode (key width, with or without values): the block-sort tile
// NT x VT and the merge-pass tile.  A merge tile must divide twice the block
// tile, so that it lies inside one run pair in every pass.  With an odd
// number of outputs per thread the threads' runs start in different
// shared-memory banks (in the block sort and in the passes).  4-byte keys
// alone use 512 x 33 = 16,896-key blocks (2^28 keys need 14 passes, not the
// 15 of 8192-key blocks) and 128 x 33 pass tiles (2^28 keys: 8.58 ms against
// 8.80 ms with 256 x 33 tiles; 1024 x 33 blocks, one pass fewer, 8.89 ms:
// the larger block sort costs more than the pass it saves); the modes with
// values, the 8-byte and the 16-byte keys, whose threads hold more
// registers, sort 256-thread blocks (more CTAs resident per SM), which
// measured faster than the larger blocks' saved pass (16-byte keys: 256 x 9
// blocks and 128 x 9 pass tiles, 2^25 keys in 3.52 ms against 4.03 ms with
// 512 x 4 and 128 x 8).
struct SortMode {
    int bs_nt, bs_vt;  // block sort
    int nt, vt;        // merge passes (TMA-staged tiles)
};
#define MP_SORT_MODE_4 512, 33, 128, 33
#define MP_SORT_MODE_4V 256, 33, 128, 33
#define MP_SORT_MODE_8 256, 27, 128, 27
#define MP_SORT_MODE_8V 256, 27, 128, 27
#define MP_SORT_MODE_16 256, 9, 128, 9

static SortMode sort_mode(int key_bytes, bool vals)
{
    if (key_bytes == 4) return vals ? SortMode{MP_SORT_MODE_4V} : SortMode{MP_SORT_MODE_4};
    if (key_bytes == 8) return vals ? SortMode{MP_SORT_MODE_8V} : SortMode{MP_SORT_MODE_8};
    return SortMode{MP_SORT_MODE_16};
}

static int64_t block_tile(int key_bytes, bool vals)
{
    const SortMode m = sort_mode(key_bytes, vals);
    return (int64_t)m.bs_nt * m.bs_vt;
}

static Shape sort_merge_shape(int key_bytes, bool vals)
{
    const SortMode m = sort_mode(key_bytes, vals);
    return Shape{m.nt, m.vt, MP_STAGE_BULK};
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
    const int64_t tiles = ceil_div(n, sort_merge_shape(kind.bytes, with_values).tile());
    return align256((size_t)n * kind.bytes) + (with_values ? align256((size_t)n * 4) : 0) +
           align256((size_t)(tiles + 1) * 8);
}

template <class K, bool VALS, int NT, int VT, bool ENC_OUT>
static cudaError_t launch_block_sort(const K* in, const uint32_t* vin, K* out, uint32_t* vout,
                                     int64_t n, const KeyKind& kind, cudaStream_t stream)
{
    using SM = SortSmem<K, VALS, NT, VT>;
    auto kern = block_sort_kernel<K, VALS, NT, VT, ENC_OUT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SM::bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    unsigned int* err = kernel_error_word();
    if (!err) return cudaErrorInvalidSymbol;
    const Codec<K> c = make_codec<K>(kind.flip, kind.fmask, kind.inv);
    const int64_t blocks = ceil_div(n, (int64_t)NT * VT);
    kern<<<(unsigned)blocks, NT, SM::bytes, stream>>>(in, vin, out, vout, n, c, err);
    return cudaGetLastError();
}

// Block-sort launch of one mode, its tile taken from the mode's macro.
template <class K, bool VALS, int BNT, int BVT, int NT_, int VT_>
static cudaError_t block_sort_mode(const void* in, const uint32_t* vin, void* out, uint32_t* vout,
                                   int64_t n, const KeyKind& kind, bool enc_out, cudaStream_t stream)
{
    if (enc_out)
        return launch_block_sort<K, VALS, BNT, BVT, true>((const K*)in, vin, (K*)out, vout, n, kind, stream);
    return launch_block_sort<K, VALS, BNT, BVT, false>((const K*)in, vin, (K*)out, vout, n, kind, stream);
}

static cudaError_t block_sort(const KeyKind& kind, const void* in, const uint32_t* vin, void* out,
                              uint32_t* vout, int64_t n, bool enc_out, cudaStream_t stream)
{
    if (kind.bytes == 4) {
        if (vin) return block_sort_mode<uint32_t, true, MP_SORT_MODE_4V>(in, vin, out, vout, n, kind, enc_out, stream);
        return block_sort_mode<uint32_t, false, MP_SORT_MODE_4>(in, nullptr, out, nullptr, n, kind, enc_out, stream);
    }
    if (kind.bytes == 16) {
        if (vin) return block_sort_mode<u128, true, MP_SORT_MODE_16>(in, vin, out, vout, n, kind, enc_out, stream);
        return block_sort_mode<u128, false, MP_SORT_MODE_16>(in, nullptr, out, nullptr, n, kind, enc_out, stream);
    }
    if (vin) return block_sort_mode<uint64_t, true, MP_SORT_MODE_8V>(in, vin, out, vout, n, kind, enc_out, stream);
    return block_sort_mode<uint64_t, false, MP_SORT_MODE_8>(in, nullptr, out, nullptr, n, kind, enc_out, stream);
}

// Launch of the last pass over encoded runs (decoding codec fixed where the
// kind allows).
template <class K, bool VALS, int NT, int VT, int CK>
static cudaError_t launch_last_pass_ck(const MergeProblem& p, const int64_t* a_split, cudaStream_t stream)
{
    using SM = MergeBulkSmem<K, VALS, NT, VT>;
    auto kern = sort_last_pass_kernel<K, VALS, NT, VT, CK>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    unsigned int* err = kernel_error_word();
    if (!err) return cudaErrorInvalidSymbol;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ceil_div(p.total(), (int64_t)NT * VT));
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

template <class K, bool VALS, int BNT, int BVT, int NT, int VT>
static cudaError_t last_pass_mode(const MergeProblem& p, const int64_t* a_split, cudaStream_t stream)
{
    if (p.kind.signed_int()) return launch_last_pass_ck<K, VALS, NT, VT, CODEC_ENCODED_SIGNED>(p, a_split, stream);
    if constexpr (sizeof(K) == 4) {
        if (p.kind.ascending_float())
            return launch_last_pass_ck<K, VALS, NT, VT, CODEC_ENCODED_FLOAT>(p, a_split, stream);
    }
    return launch_last_pass_ck<K, VALS, NT, VT, CODEC_ENCODED_RUNTIME>(p, a_split, stream);
}

static cudaError_t last_pass(const MergeProblem& p, const int64_t* a_split, cudaStream_t stream)
{
    const bool v = p.vals;
    if (p.kind.bytes == 4)
        return v ? last_pass_mode<uint32_t, true, MP_SORT_MODE_4V>(p, a_split, stream)
                 : last_pass_mode<uint32_t, false, MP_SORT_MODE_4>(p, a_split, stream);
    if (p.kind.bytes == 16)
        return v ? last_pass_mode<u128, true, MP_SORT_MODE_16>(p, a_split, stream)
                 : last_pass_mode<u128, false, MP_SORT_MODE_16>(p, a_split, stream);
    return v ? last_pass_mode<uint64_t, true, MP_SORT_MODE_8V>(p, a_split, stream)
             : last_pass_mode<uint64_t, false, MP_SORT_MODE_8>(p, a_split, stream);
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

    const int64_t bt = block_tile(kind.bytes, with_vals);
    const Shape ms = sort_merge_shape(kind.bytes, with_vals);
    if ((2 * bt) % ms.tile() != 0) return fail(MP_ERR_INTERNAL, "sort: merge tile does not divide a run pair");
    const int passes = ceil_log2(ceil_div(n, bt));
    // The block sort writes where an even number of passes later ends in keys.
    void* cur = (passes & 1) ? ws_keys : keys;
    uint32_t* curv = (passes & 1) ? ws_vals : vals;
    void* oth = (passes & 1) ? keys : ws_keys;
    uint32_t* othv = (passes & 1) ? vals : ws_vals;

    // With merge passes to follow and a codec that is not the identity, the
    // runs stay encoded between the passes: they compare as unsigned keys
    // (no codec work in the intermediate passes) and the last pass decodes.
    const bool encoded = passes > 0 && !kind.identity();
    KeyKind plain = kind;
    plain.flip = plain.fmask = plain.inv = 0;
    cudaError_t e = block_sort(kind, keys, vals, cur, curv, n, encoded, stream);
    if (e != cudaSuccess) return cuda_fail(e, "block sort launch");

    for (int p = 0; p < passes; ++p) {
        const bool last_decodes = encoded && p == passes - 1;
        MergeProblem mp;
        mp.kind = encoded ? plain : kind;
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
        if (last_decodes) {
            mp.kind = kind;  // compared as encoded, decoded with kind's codec
            e = last_pass(mp, splits, stream);
        } else {
            e = launch_merge_tiles(mp, ms, splits, stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "sort pass merge launch");
        std::swap(cur, oth);
        std::swap(curv, othv);
    }
    if (cur != keys) return fail(MP_ERR_INTERNAL, "sort: result not in the key buffer");
    return MP_OK;
}

}  // namespace mp
