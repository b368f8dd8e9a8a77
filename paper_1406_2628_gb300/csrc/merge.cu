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

#include "mp_device.cuh"
#include "mp_internal.h"
#include "mp_tile.cuh"

namespace mp {

template <class K>
struct TileArgs {
    const K* a;
    const K* b;
    const uint32_t* av;
    const uint32_t* bv;
    K* out;
    uint32_t* outv;
    int64_t na, nb, run;
    int64_t total;
    const int64_t* a_split;
    Codec<K> codec;
};

// The merge pair that output index d belongs to (run == 0: the only pair).
template <class K>
struct Pair {
    const K* A;
    const K* B;
    const uint32_t* AV;
    const uint32_t* BV;
    int64_t na, nb, base;
};

template <class K>
__device__ __forceinline__ Pair<K> pair_at(const TileArgs<K>& p, int64_t d)
{
    Pair<K> q;
    if (p.run == 0) {
        q.A = p.a; q.B = p.b; q.AV = p.av; q.BV = p.bv;
        q.na = p.na; q.nb = p.nb; q.base = 0;
    } else {
        const int64_t w2 = 2 * p.run;
        const int64_t base = (d / w2) * w2;
        const int64_t rest = p.na - base;
        q.na = rest < p.run ? rest : p.run;
        const int64_t rest_b = rest - q.na;
        q.nb = rest_b < p.run ? rest_b : p.run;
        q.A = p.a + base;
        q.B = p.a + base + q.na;
        q.AV = p.av ? p.av + base : nullptr;
        q.BV = p.av ? p.av + base + q.na : nullptr;
        q.base = base;
    }
    return q;
}

// ---------------------------------------------------------------------------
// Partition: one thread per tile boundary, binary search along the diagonal
// in global memory (Alg. 2; at most ceil(log2(min(|A|,|B|)+1)) probes, Thm 14).
// ---------------------------------------------------------------------------
template <class K>
__global__ void __launch_bounds__(256) partition_kernel(TileArgs<K> p, int64_t spacing,
                                                        int64_t n_bounds, int64_t* a_split)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_bounds) return;
    const int64_t d = t * spacing < p.total ? t * spacing : p.total;
    const Pair<K> q = pair_at(p, d < p.total ? d : p.total - 1);
    const K* A = q.A;
    const K* B = q.B;
    const Codec<K> c = p.codec;
    a_split[t] = diagonal_search<K>([&](int64_t i) { return key_enc(__ldg(A + i), c); }, q.na,
                                    [&](int64_t i) { return key_enc(__ldg(B + i), c); }, q.nb,
                                    d - q.base);
    // Let a dependent merge launch (programmatic dependent launch) start its
    // prologue; it waits on griddepcontrol.wait before reading a_split.
    asm volatile("griddepcontrol.launch_dependents;");
}

// ---------------------------------------------------------------------------
// Merge tile kernel: one CTA per tile of NT*VT outputs.
// ---------------------------------------------------------------------------
template <class K, bool VALS, int NT, int VT>
__global__ void __launch_bounds__(NT) merge_tile_kernel(TileArgs<K> p)
{
    static_assert(VT % 4 == 0, "VT must be a multiple of 4");
    constexpr int T = NT * VT;
    extern __shared__ __align__(16) unsigned char smem[];

    const int tid = threadIdx.x;
    const int64_t tile = blockIdx.x;
    const int64_t d0 = tile * T;
    const int64_t d1 = d0 + T < p.total ? d0 + T : p.total;
    const Pair<K> q = pair_at(p, d0);
    const int64_t d0l = d0 - q.base, d1l = d1 - q.base;

    // Wait for the partition kernel (programmatic dependent launch).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // Split points are clamped into the grid and made monotone, so that
    // unsorted inputs or foreign split arrays give wrong output rather than
    // out-of-range accesses; for valid inputs the clamps change nothing.
    const int64_t a0 = clamp_split(p.a_split[tile], d0l, q.na, q.nb);
    int64_t a1 = (d1l == q.na + q.nb) ? q.na : clamp_split(p.a_split[tile + 1], d1l, q.na, q.nb);
    a1 = a1 < a0 ? a0 : (a1 > a0 + (d1l - d0l) ? a0 + (d1l - d0l) : a1);
    const int64_t b0 = d0l - a0, b1 = d1l - a1;
    const int la = (int)(a1 - a0), lb = (int)(b1 - b0);
    const int L = la + lb;

    const auto v = stage_tile<K, VALS, NT, VT>(smem, q.A + a0, la, q.B + b0, lb,
                                               VALS ? q.AV + a0 : nullptr,
                                               VALS ? q.BV + b0 : nullptr);
    // Per-thread split inside the window (Thm 17), then VT serial steps.
    {
        const int diag = tid * VT < L ? tid * VT : L;
        const int ai = smem_diagonal_search(v.sA, la, v.sB, lb, diag, p.codec);
        uint32_t packed[VT / 2];
        serial_merge_indices<K, VT>(v.sA, la, v.sB, lb, ai, diag - ai, p.codec, packed);
        put_indices<VT>(v.sidx, packed);
    }
    __syncthreads();
    store_tile<K, VALS, NT, VT>(v, p.out + d0, VALS ? p.outv + d0 : nullptr);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
template <class K>
static TileArgs<K> make_args(const MergeProblem& p, const int64_t* a_split)
{
    TileArgs<K> t;
    t.a = static_cast<const K*>(p.a);
    t.b = static_cast<const K*>(p.b);
    t.av = p.av;
    t.bv = p.bv;
    t.out = static_cast<K*>(p.out);
    t.outv = p.outv;
    t.na = p.na;
    t.nb = p.nb;
    t.run = p.run;
    t.total = p.total();
    t.a_split = a_split;
    t.codec.flip = (K)p.kind.flip;
    t.codec.fmask = (K)p.kind.fmask;
    return t;
}

cudaError_t launch_partition(const MergeProblem& p, int64_t spacing, int64_t* a_split,
                             cudaStream_t stream)
{
    const int64_t n_bounds = ceil_div(p.total(), spacing) + 1;
    const int threads = 256;
    const int64_t blocks = ceil_div(n_bounds, threads);
    if (p.kind.bytes == 4)
        partition_kernel<uint32_t><<<(unsigned)blocks, threads, 0, stream>>>(
            make_args<uint32_t>(p, nullptr), spacing, n_bounds, a_split);
    else
        partition_kernel<uint64_t><<<(unsigned)blocks, threads, 0, stream>>>(
            make_args<uint64_t>(p, nullptr), spacing, n_bounds, a_split);
    return cudaGetLastError();
}

template <class K, bool VALS, int NT, int VT>
static cudaError_t launch_tiles_t(const MergeProblem& p, const int64_t* a_split, cudaStream_t stream)
{
    using SM = TileSmem<K, VALS, NT, VT>;
    auto kern = merge_tile_kernel<K, VALS, NT, VT>;
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
    return cudaLaunchKernelEx(&cfg, kern, make_args<K>(p, a_split));
}

// Compiled tile shapes (NT, VT).
#define MP_MERGE_SHAPES(X) X(128, 8) X(256, 8) X(128, 16) X(256, 16) X(512, 8)

bool merge_shape_supported(int key_bytes, bool with_values, const Shape& s)
{
    (void)with_values;
    if (key_bytes != 4 && key_bytes != 8) return false;
    if (s.staging != MP_STAGE_VECTOR) return false;
#define X(NT_, VT_) if (s.nt == NT_ && s.vt == VT_) return true;
    MP_MERGE_SHAPES(X)
#undef X
    return false;
}

Shape default_merge_shape(int key_bytes, bool with_values, int64_t total)
{
    (void)with_values;
    (void)total;
    Shape s;
    s.nt = 256;
    s.vt = key_bytes == 8 ? 8 : 16;
    s.staging = MP_STAGE_VECTOR;
    return s;
}

cudaError_t launch_merge_tiles(const MergeProblem& p, const Shape& s, const int64_t* a_split,
                               cudaStream_t stream)
{
    const bool vals = p.vals;
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
