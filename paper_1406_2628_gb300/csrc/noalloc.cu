// noalloc.cu -- a merge entry point that allocates no memory.
//
// mp_merge_keys / mp_merge_pairs take their scratch (the split points
// between tiles) from a stream-ordered pool, which allocates device memory
// the first time it grows.  Some callers cannot allow that: code that runs
// inside another runtime's memory arena which has already reserved the
// device memory, or latency-critical loops in which an allocation call may
// block or synchronise.  mp_merge_noalloc runs the same two kernels with the
// split points kept in a fixed array compiled into the library instead.
//
// That array is shared by every call on a device, so calls whose work
// overlaps on the GPU (different streams, or other host threads) race on it;
// calls in one stream are ordered and safe.  Nothing in it needs to start
// at zero: the partition kernel writes every entry that the merge kernel
// then reads.  The array stays resident on every GPU that loads the library
// until the process exits.  The device memory behind it is taken when the
// CUDA runtime loads this file's module on a device; under CUDA's default
// lazy module loading that happens at the first call on each device (the
// cudaGetSymbolAddress lookup below), so that first call is the one that
// must come before an arena reserves the device's memory.
#include <mutex>

#include "mp_internal.h"

namespace mp {

// Split points: one per tile boundary.  2 MiB.
static constexpr int64_t kNoallocSplits = 262144;
static constexpr int kNoallocThreads = 256;
static constexpr int kNoallocItems = 16;
static constexpr int64_t kNoallocTile = (int64_t)kNoallocThreads * kNoallocItems;
static constexpr int64_t kNoallocMaxTotal = (kNoallocSplits - 1) * kNoallocTile;

static __device__ __align__(256) int64_t g_noalloc_splits[kNoallocSplits];

// Host-side address of g_noalloc_splits per device.  In host code the
// array's name is only a stand-in for the symbol, not a device address, so
// it is resolved with cudaGetSymbolAddress while the device is current.
static std::mutex g_noalloc_mu;
static int64_t* g_noalloc_ptr[64];

static mp_status noalloc_scratch(int64_t** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "mp_merge_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(MP_ERR_INTERNAL, "mp_merge_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_splits);
        if (e != cudaSuccess) return cuda_fail(e, "mp_merge_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = static_cast<int64_t*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return MP_OK;
}

}  // namespace mp

using namespace mp;

extern "C" mp_status mp_merge_noalloc(mp_dtype dtype, const void* a_keys, const uint32_t* a_vals,
                                      int64_t na, const void* b_keys, const uint32_t* b_vals,
                                      int64_t nb, void* out_keys, uint32_t* out_vals,
                                      mp_stream_t stream)
{
    MP_RANGE("mp_merge_noalloc");
    // Written so that no sum can overflow: negative sizes are left to
    // merge_prepare's checks.
    if (na >= 0 && nb >= 0 && (na > kNoallocMaxTotal || nb > kNoallocMaxTotal - na))
        return fail(MP_ERR_INVALID_ARG,
                    "mp_merge_noalloc: na + nb exceeds the fixed scratch limit of 1073737728 outputs");
    const int base = (int)dtype & 0xFF;
    if (base == MP_U128 || base == MP_I128)
        return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_merge_noalloc: 128-bit keys are not supported");
    MergeProblem p;
    Shape s;
    const bool vals = a_vals || b_vals || out_vals;
    const mp_plan plan{kNoallocThreads, kNoallocItems, MP_STAGE_BULK, 0};
    mp_status st = merge_prepare(dtype, a_keys, a_vals, na, b_keys, b_vals, nb, out_keys, out_vals,
                                 vals, &plan, "mp_merge_noalloc", &p, &s);
    if (st != MP_OK) return st;
    if (na + nb == 0) return MP_OK;
    int64_t* splits = nullptr;
    st = noalloc_scratch(&splits);
    if (st != MP_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = launch_partition(p, s.tile(), splits, cs);
    if (e == cudaSuccess) e = launch_merge_tiles(p, s, splits, cs);
    return e == cudaSuccess ? MP_OK : cuda_fail(e, "mp_merge_noalloc");
}
