/*
 * mp.h -- C ABI of the GB300 Merge Path library (libmp.so).
 *
 * Merge Path (Green, Odeh, Birk, "Merge Path - A Visually Intuitive Approach
 * to Parallel Merging"): the stable merge of two sorted arrays, split into
 * equal, independent pieces by binary searches along the cross diagonals of
 * the |A| x |B| merge grid (Sec. II, Alg. 1, Alg. 2), and the merge sort
 * built from it (Sec. I, Sec. III).  Every call runs CUDA kernels on the
 * current device; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Order: ascending.  Keys compare in their natural order; MP_F32 keys
 *    compare in IEEE-754 numeric order with -0.0 before +0.0.  NaN keys are
 *    outside the contract (mp_check_sorted reports them).  Merges are stable:
 *    on equal keys A's element comes first (Sec. II.A: the path moves right,
 *    i.e. takes B, only if A[i] > B[j]).  Sorts are stable.
 *  - Memory: unless a comment says "host", every pointer is a device pointer
 *    (cudaMalloc, a stream-ordered pool, or torch's allocator) on the
 *    current device.  The caller owns all memory it passes in; the library
 *    never frees it.  Key pointers must be aligned to the key size, value
 *    pointers to 4 bytes.  Outputs must not overlap inputs unless stated.
 *  - Values (payloads) are always uint32 and move with their keys.  A value
 *    pointer may be NULL when its array has zero elements.
 *  - Sizes are int64 element counts (arrays may exceed 2^31 elements).
 *  - Streams: work is enqueued on `stream` (NULL = the legacy default stream)
 *    and the call returns without waiting, unless its comment says it
 *    synchronises.  Argument errors are detected on the host and returned
 *    before anything is enqueued; errors of already-enqueued work surface
 *    from a later CUDA synchronisation, as with any CUDA launch.
 *  - Errors are returned as mp_status.  Nothing throws across the ABI and
 *    nothing aborts.  mp_last_error() gives a human-readable detail for the
 *    last failing call on the calling thread.
 *  - Scratch: calls that need temporary device memory take it from a
 *    library-owned stream-ordered pool (cudaMallocAsync semantics) unless
 *    they take an explicit workspace argument.
 */
#ifndef MP_H
#define MP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MP_API __attribute__((visibility("default")))
#else
#define MP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* mp_stream_t;

typedef enum mp_status {
    MP_OK = 0,
    MP_ERR_INVALID_ARG = 1,       /* bad size, NULL, misaligned or overlapping pointer */
    MP_ERR_UNSUPPORTED_DTYPE = 2, /* dtype not in mp_dtype */
    MP_ERR_NOT_SORTED = 3,        /* mp_check_sorted: input not ascending */
    MP_ERR_NAN = 4,               /* mp_check_sorted: an MP_F32 key is NaN */
    MP_ERR_NO_MEMORY = 5,         /* device or host allocation failed */
    MP_ERR_BUDGET = 6,            /* request larger than a queue's memory budget */
    MP_ERR_TIMEOUT = 7,           /* a bounded wait ran out */
    MP_ERR_CUDA = 8,              /* a CUDA runtime call failed (see mp_last_error) */
    MP_ERR_INTERNAL = 9,          /* a library invariant failed */
    MP_ERR_NOT_READY = 10         /* a polled result is not finished yet */
} mp_status;

typedef enum mp_dtype {
    MP_I32 = 0, /* int32_t  */
    MP_U32 = 1, /* uint32_t */
    MP_F32 = 2, /* float (IEEE-754 binary32), -0.0 < +0.0, no NaN */
    MP_U64 = 3, /* uint64_t */
    MP_I64 = 4  /* int64_t  */
} mp_dtype;

/* Tile shape of the merge kernels.  block_threads (NT) threads per CTA, each
 * producing items_per_thread (VT) outputs, so one CTA produces a tile of
 * NT*VT outputs (Alg. 1's "length", one Merge Path segment per CTA; Cor. 7).
 * Zero fields mean "choose automatically" (tuned table, see mp_autotune). */
typedef struct mp_plan {
    int32_t block_threads;
    int32_t items_per_thread;
    int32_t staging;  /* MP_STAGE_AUTO, MP_STAGE_VECTOR (128-bit loads) or MP_STAGE_BULK (1D TMA) */
    int32_t reserved; /* must be 0 */
} mp_plan;

#define MP_STAGE_AUTO 0
#define MP_STAGE_VECTOR 1
#define MP_STAGE_BULK 2

/* Text for a status code (static storage, never NULL). */
MP_API const char* mp_status_string(mp_status status);

/* Detail of the last error returned on the calling thread ("" if none). */
MP_API const char* mp_last_error(void);

/* Size in bytes of one key of `dtype`, or 0 for an unknown dtype. */
MP_API size_t mp_dtype_size(mp_dtype dtype);

/*
 * mp_merge_keys -- stable merge of two sorted key arrays (Alg. 1).
 *   a[0..na), b[0..nb): sorted ascending, device.  out[0..na+nb): device,
 *   must not overlap a or b.  na = nb = 0 is a no-op.  Ties take A first.
 * Runs a partition kernel (Alg. 2 at every tile boundary, Thm 9 / Thm 14)
 * and a merge kernel (one tile per CTA, Cor. 6).  Scratch: (tiles+1) int64
 * split points from the library pool.
 */
MP_API mp_status mp_merge_keys(mp_dtype dtype, const void* a, int64_t na,
                        const void* b, int64_t nb, void* out, mp_stream_t stream);

/*
 * mp_merge_pairs -- as mp_merge_keys, moving a uint32 value with every key.
 *   a_vals[i] travels with a_keys[i], b_vals[j] with b_keys[j].  Outputs
 *   out_keys / out_vals (na+nb each) must not overlap any input.
 */
MP_API mp_status mp_merge_pairs(mp_dtype dtype,
                         const void* a_keys, const uint32_t* a_vals, int64_t na,
                         const void* b_keys, const uint32_t* b_vals, int64_t nb,
                         void* out_keys, uint32_t* out_vals, mp_stream_t stream);

/*
 * mp_merge_path_partition -- the split points alone (Alg. 2, Thm 9).
 *   For t = 0 .. ceil((na+nb)/spacing), writes a_split[t] = number of A
 *   elements among the first d_t = min(t*spacing, na+nb) outputs of the
 *   stable merge (the crossing of the Merge Path with cross diagonal d_t;
 *   b_split = d_t - a_split).  a_split: device, ceil((na+nb)/spacing)+1
 *   int64 entries.  spacing >= 1.
 */
MP_API mp_status mp_merge_path_partition(mp_dtype dtype, const void* a, int64_t na,
                                  const void* b, int64_t nb, int64_t spacing,
                                  int64_t* a_split, mp_stream_t stream);

/*
 * mp_merge_plan -- mp_merge_keys / mp_merge_pairs with an explicit tile
 * plan (NULL = automatic).  An unsupported plan returns MP_ERR_INVALID_ARG;
 * mp_plan_supported() lists the compiled shapes.  Values are merged when any
 * of a_vals, b_vals, out_vals is non-NULL; pass all three NULL to merge keys
 * only.
 */
MP_API mp_status mp_merge_plan(mp_dtype dtype,
                        const void* a_keys, const uint32_t* a_vals, int64_t na,
                        const void* b_keys, const uint32_t* b_vals, int64_t nb,
                        void* out_keys, uint32_t* out_vals,
                        const mp_plan* plan, mp_stream_t stream);

/* 1 if (block_threads, items_per_thread, staging) is a compiled merge shape. */
MP_API int mp_plan_supported(const mp_plan* plan);

/*
 * mp_merge_tile_items -- the tile length T (outputs per CTA) that
 * mp_merge_plan / mp_merge_partitioned use for this dtype, payload choice,
 * total output length and plan (NULL = automatic).  0 if the plan is not
 * supported or the dtype unknown.
 */
MP_API int64_t mp_merge_tile_items(mp_dtype dtype, int with_values, int64_t total,
                                   const mp_plan* plan);

/*
 * mp_merge_partitioned -- the merge kernel of Alg. 1 alone, given the split
 * points: a_split must hold mp_merge_path_partition(..., spacing = T, ...)
 * for T = mp_merge_tile_items(dtype, a_vals != NULL, na + nb, plan) and the
 * same inputs (device, ceil((na+nb)/T)+1 int64).  Arguments otherwise as in
 * mp_merge_plan.  Lets a caller reuse split points, or time the merge
 * kernel apart from the partition kernel (the paper times the partition
 * step separately, Sec. VI).
 */
MP_API mp_status mp_merge_partitioned(mp_dtype dtype,
                                      const void* a_keys, const uint32_t* a_vals, int64_t na,
                                      const void* b_keys, const uint32_t* b_vals, int64_t nb,
                                      void* out_keys, uint32_t* out_vals,
                                      const int64_t* a_split, const mp_plan* plan,
                                      mp_stream_t stream);

/*
 * mp_merge_pairs_host -- SYNCHRONOUS end-to-end merge of HOST arrays.
 *   All six pointers are host memory (page-locked memory gives the best
 *   copy rate; pageable works).  The library takes device buffers from its
 *   pool, copies the inputs in, runs mp_merge_pairs on `stream`, copies the
 *   outputs back and waits for `stream`.  a_vals = b_vals = out_vals = NULL
 *   merges keys only.  MP_ERR_NO_MEMORY if the device cannot hold the
 *   inputs and outputs.
 */
MP_API mp_status mp_merge_pairs_host(mp_dtype dtype,
                                     const void* a_keys, const uint32_t* a_vals, int64_t na,
                                     const void* b_keys, const uint32_t* b_vals, int64_t nb,
                                     void* out_keys, uint32_t* out_vals, mp_stream_t stream);

/*
 * mp_sort_workspace_bytes -- device workspace that mp_sort needs for n keys
 * (with_values != 0: plus uint32 values).  0 for n <= 1.
 */
MP_API size_t mp_sort_workspace_bytes(mp_dtype dtype, int64_t n, int with_values);

/*
 * mp_sort -- stable merge sort in place (Sec. I, Sec. III).
 *   keys[0..n) (and vals[0..n) if not NULL) are sorted ascending by key.
 *   A block-sort kernel sorts tiles of the array in shared memory, then
 *   ceil(log2(tiles)) Merge Path passes merge run pairs of doubling width
 *   between keys and the workspace.  workspace: device, at least
 *   mp_sort_workspace_bytes(dtype, n, vals != NULL) bytes, 256-byte
 *   aligned, not overlapping keys/vals; its contents are clobbered.
 */
MP_API mp_status mp_sort(mp_dtype dtype, void* keys, uint32_t* vals, int64_t n,
                  void* workspace, size_t workspace_bytes, mp_stream_t stream);

/*
 * mp_merge_batched -- nseg independent stable merges in one launch.
 *   Segment s merges a[a_off[s] .. a_off[s+1]) with b[b_off[s] .. b_off[s+1])
 *   into out[a_off[s]+b_off[s] .. a_off[s+1]+b_off[s+1]).
 *   a_off, b_off: device int64 arrays of nseg+1 nondecreasing entries with
 *   a_off[0] = b_off[0] = 0; na_total = a_off[nseg] and nb_total =
 *   b_off[nseg] must be passed from the host (the launch is sized from them
 *   without reading device memory).  Segments may be empty.
 *   a_vals/b_vals/out_vals: NULL for keys only, else uint32 values.
 * Merge Path runs over the concatenated output of all segments (the
 * concatenation is itself one merge ordered by (segment, key), Cor. 6), so
 * tiles are equal in size whatever the segment lengths and may straddle
 * segments.  plan: NULL = automatic.
 */
MP_API mp_status mp_merge_batched(mp_dtype dtype,
                           const void* a, const int64_t* a_off,
                           const void* b, const int64_t* b_off,
                           int64_t nseg, int64_t na_total, int64_t nb_total,
                           void* out,
                           const uint32_t* a_vals, const uint32_t* b_vals,
                           uint32_t* out_vals,
                           const mp_plan* plan, mp_stream_t stream);

/*
 * mp_check_sorted -- SYNCHRONOUS check that keys[0..n) is ascending and, for
 * MP_F32, free of NaN.  Returns MP_OK, MP_ERR_NOT_SORTED or MP_ERR_NAN
 * (NaN wins if both).  Waits for `stream`.
 */
MP_API mp_status mp_check_sorted(mp_dtype dtype, const void* keys, int64_t n, mp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* MP_H */
