// merge_bulk.cu -- the TMA-staged merge tile kernels (MP_STAGE_BULK), the
// default tile of plain merges and of the merge passes of the sort.
//
// One CTA per tile of T = NT * VT outputs (Cor. 6): the tile's A and B
// windows (Lemma 16) are copied into shared memory by TMA bulk copies, each
// thread finds its split inside the window (Thm 17) and merges VT outputs
// serially, and the tile is written back with coalesced 128-bit stores (see
// mp_bulk.cuh).  Kernels are compiled per key codec: unsigned keys compare
// as they are, signed integers and ascending floats with their fixed
// encodings, and other kinds (descending order) with the runtime codec.
#include "mp_device.cuh"
#include "mp_internal.h"
#include "mp_tile.cuh"
#include "mp_bulk.cuh"

namespace mp {

template <class K, bool VALS, int NT, int VT, int CK>
__global__ void __launch_bounds__(NT) merge_tile_bulk_kernel(TileArgs<K> p, unsigned int* err)
{
    extern __shared__ __align__(16) unsigned char smem[];
    // Wait for the partition kernel (programmatic dependent launch).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    merge_tile_bulk_body<K, VALS, NT, VT, CK>(p, blockIdx.x, p.a_split, smem, err);
}

template <class K, bool VALS, int NT, int VT, int CK>
static cudaError_t launch_bulk_ck(const MergeProblem& p, const int64_t* a_split, cudaStream_t stream)
{
    using SM = MergeBulkSmem<K, VALS, NT, VT>;
    auto kern = merge_tile_bulk_kernel<K, VALS, NT, VT, CK>;
    static bool configured = false;  // attribute is per function, set once
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
static cudaError_t launch_bulk_t(const MergeProblem& p, const int64_t* a_split, cudaStream_t stream)
{
    if (p.kind.identity()) return launch_bulk_ck<K, VALS, NT, VT, CODEC_IDENTITY>(p, a_split, stream);
    if (p.kind.signed_int()) return launch_bulk_ck<K, VALS, NT, VT, CODEC_SIGNED>(p, a_split, stream);
    if constexpr (sizeof(K) == 4) {  // float keys are 32-bit
        if (p.kind.ascending_float()) return launch_bulk_ck<K, VALS, NT, VT, CODEC_FLOAT>(p, a_split, stream);
    }
    return launch_bulk_ck<K, VALS, NT, VT, CODEC_RUNTIME>(p, a_split, stream);
}

cudaError_t launch_merge_bulk(const MergeProblem& p, const Shape& s, const int64_t* a_split,
                              cudaStream_t stream)
{
    if (s.staging != MP_STAGE_BULK) return cudaErrorInvalidValue;
    const bool vals = p.vals;
    if (p.kind.bytes == 16) {
#define X(NT_, VT_)                                                                            \
        if (s.nt == NT_ && s.vt == VT_)                                                        \
            return vals ? launch_bulk_t<u128, true, NT_, VT_>(p, a_split, stream)              \
                        : launch_bulk_t<u128, false, NT_, VT_>(p, a_split, stream);
        MP_WIDE_SHAPES(X)
#undef X
        return cudaErrorInvalidValue;
    }
#define X(NT_, VT_)                                                                            \
    if (s.nt == NT_ && s.vt == VT_) {                                                          \
        if (p.kind.bytes == 4)                                                                 \
            return vals ? launch_bulk_t<uint32_t, true, NT_, VT_>(p, a_split, stream)          \
                        : launch_bulk_t<uint32_t, false, NT_, VT_>(p, a_split, stream);        \
        return vals ? launch_bulk_t<uint64_t, true, NT_, VT_>(p, a_split, stream)              \
                    : launch_bulk_t<uint64_t, false, NT_, VT_>(p, a_split, stream);            \
    }
    MP_BULK_SHAPES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace mp
