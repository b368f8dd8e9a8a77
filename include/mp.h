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
 *  - Order: ascending, or descending with MP_DESCENDING.  Keys compare in
 *    their natural order; MP_F32 keys
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
    MP_I64 = 4, /* int64_t  */
    /* Multi-word keys: 128-bit integers, two 64-bit words per key, the low
     * word first in memory (little-endian), 16-byte aligned.  Supported by
     * the plain merges (tile plans MP_STAGE_BULK (128,8) / (256,8) / (128,12) /
     * (128,9) and the streaming plans), mp_merge_path_partition, mp_sort, mp_set_operation
     * and mp_check_sorted; the batched, grouped, queued, checksum and
     * allocation-free entry points return MP_ERR_UNSUPPORTED_DTYPE. */
    MP_U128 = 5, /* unsigned 128-bit */
    MP_I128 = 6  /* signed 128-bit (two's complement) */
} mp_dtype;

/* Order flag, OR'ed into the dtype argument of any entry point: keys are in
 * DESCENDING order (inputs sorted descending, results descending).  The
 * paper assumes ascending order without loss of generality (Sec. II.A); the
 * descending merge is the same method on complemented keys, and stays
 * stable (on equal keys A's element still comes first). */
#define MP_DESCENDING 0x100

/* Tile shape of the merge kernels.  block_threads (NT) threads per CTA, each
 * producing items_per_thread (VT) outputs, so one CTA produces a tile of
 * NT*VT outputs (Alg. 1's "length", one Merge Path segment per CTA; Cor. 7).
 * Zero fields mean "choose automatically" (tuned table, see mp_autotune). */
typedef struct mp_plan {
    int32_t block_threads;
    int32_t items_per_thread;
    int32_t staging;  /* MP_STAGE_AUTO, _VECTOR, _BULK, _WARP or _STREAM (below) */
    int32_t reserved; /* must be 0 */
} mp_plan;

#define MP_STAGE_AUTO 0
#define MP_STAGE_VECTOR 1 /* windows via 128-bit loads through registers; per-thread serial merge */
#define MP_STAGE_BULK 2   /* windows via TMA bulk copies; per-thread serial merge */
#define MP_STAGE_WARP 3   /* windows via TMA bulk copies; warp-cooperative rank merge */
/* Partition-free streaming merge (Alg. 3): one launch, no split-point
 * array.  Each CTA owns R consecutive tiles of the output, finds the splits
 * at both ends of its share (Alg. 2, one warp per end), then walks its share
 * tile by tile, carrying the path position; A and B stream through
 * shared-memory ring buffers filled by TMA bulk copies a few tiles ahead.
 * Plain merges only (mp_merge_keys/_pairs/_plan, graphs); mp_merge_partitioned
 * rejects it (it takes no split points). */
#define MP_STAGE_STREAM 4

/* Status, error detail and key sizes: library utilities, with no
 * counterpart in the paper.
 * Text for a status code (static storage, never NULL). */
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
 * split points from the library pool.  Small merges (up to a few million
 * outputs) take the single-launch streaming merge instead (MP_STAGE_STREAM,
 * no scratch) unless the tuned table says otherwise.
 */
MP_API mp_status mp_merge_keys(mp_dtype dtype, const void* a, int64_t na,
                        const void* b, int64_t nb, void* out, mp_stream_t stream);

/*
 * mp_merge_pairs -- as mp_merge_keys, moving a uint32 value with every key
 * (Alg. 1; the paper merges bare keys, and each value follows its key's
 * move along the path).
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
 * plan (NULL = automatic): Alg. 1 with a chosen segment length per CTA
 * (equal segments, Cor. 7).  An unsupported plan returns MP_ERR_INVALID_ARG;
 * mp_plan_supported() lists the compiled shapes.  Values are merged when any
 * of a_vals, b_vals, out_vals is non-NULL; pass all three NULL to merge keys
 * only.
 */
MP_API mp_status mp_merge_plan(mp_dtype dtype,
                        const void* a_keys, const uint32_t* a_vals, int64_t na,
                        const void* b_keys, const uint32_t* b_vals, int64_t nb,
                        void* out_keys, uint32_t* out_vals,
                        const mp_plan* plan, mp_stream_t stream);

/* 1 if (block_threads, items_per_thread, staging) is a compiled merge shape
 * (a library query; no counterpart in the paper). */
MP_API int mp_plan_supported(const mp_plan* plan);

/*
 * mp_merge_resolve_plan -- the shape mp_merge_plan would run for this dtype,
 * payload choice (with_values != 0), total output length and plan (NULL or
 * zero fields: automatic, which consults the tuned table and may pick the
 * streaming plan for small merges).  Writes it to *resolved (staging never
 * MP_STAGE_AUTO).  MP_ERR_INVALID_ARG for an unsupported plan or a NULL
 * resolved; MP_ERR_UNSUPPORTED_DTYPE for an unknown dtype.  (A library
 * query: the paper fixes the segment length as (|A|+|B|)/p, Alg. 1.)
 * The environment variable MP_FORCE_PLAN="NT,VT[,staging]" (staging:
 * vector, bulk, warp, stream or its MP_STAGE_* number), read at each call,
 * replaces every automatic merge plan (for experiments; an unsupported one
 * makes the calls return MP_ERR_INVALID_ARG).  Every public call and
 * serving step is also an NVTX range named after the call, for profilers'
 * timelines.
 */
MP_API mp_status mp_merge_resolve_plan(mp_dtype dtype, int with_values, int64_t total, const mp_plan* plan,
                                       mp_plan* resolved);

/*
 * mp_merge_tile_items -- the tile length T (outputs per CTA; Alg. 1's
 * per-core length (|A|+|B|)/p with p = the number of tiles) that
 * mp_merge_partitioned uses for this dtype, payload choice, total output
 * length and plan (NULL = automatic; the automatic choice here is always a
 * partitioned tile plan, while an automatic mp_merge_plan / mp_merge_keys
 * may take the streaming plan for small merges).  0 if the plan is not
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
 *   inputs and outputs.  The merge is Alg. 1; the paper's arrays sit in one
 *   shared memory, so the copies and their pipelining have no counterpart
 *   in it.
 */
MP_API mp_status mp_merge_pairs_host(mp_dtype dtype,
                                     const void* a_keys, const uint32_t* a_vals, int64_t na,
                                     const void* b_keys, const uint32_t* b_vals, int64_t nb,
                                     void* out_keys, uint32_t* out_vals, mp_stream_t stream);

/*
 * mp_merge_checksum -- the merge with its results kept on chip: the
 * experiment in Sec. VI (Fig. 5) that writes merge results to a register
 * instead of memory, to separate the read side from the write side.
 *   Merges A and B (values too when a_vals/b_vals are set) exactly as
 *   mp_merge_pairs would, but stores nothing: every output j (key bits k_j
 *   zero-extended to 64 bits, value v_j or 0) is folded into
 *   *checksum = sum over j of f(k_j, v_j, j) mod 2^64 with
 *     h = k_j * 0x9E3779B97F4A7C15;  h ^= v_j * 0xBF58476D1CE4E5B9 (values only);
 *     h ^= (j + 1) * 0x94D049BB133111EB;  f = h ^ (h >> 29),
 *   an order-sensitive digest of the merged sequence.  checksum: device
 *   pointer to one 8-byte-aligned uint64, zeroed by the call then
 *   accumulated.  Global traffic: the read of A and B only.
 */
MP_API mp_status mp_merge_checksum(mp_dtype dtype,
                                   const void* a_keys, const uint32_t* a_vals, int64_t na,
                                   const void* b_keys, const uint32_t* b_vals, int64_t nb,
                                   uint64_t* checksum, mp_stream_t stream);

/*
 * Merge-based set operations.  Sec. I names joins of database query results
 * and merges of adjacency lists as uses of merging; these are the merge with
 * a keep-or-drop decision per output.  Multiset semantics: a key held m
 * times by A and n times by B appears
 *   MP_SET_UNION                 max(m, n) times: A's m copies, then B's
 *                                copies after the m-th;
 *   MP_SET_INTERSECTION          min(m, n) times: A's first min(m, n) copies;
 *   MP_SET_DIFFERENCE            max(m - n, 0) times: A's copies after the
 *                                n-th (A minus B);
 *   MP_SET_SYMMETRIC_DIFFERENCE  |m - n| times: A's copies after the n-th or
 *                                B's copies after the m-th.
 * On duplicate-free inputs these are the ordinary set operations.  Output is
 * ascending (descending with MP_DESCENDING), equal keys keep merge order (A's
 * copies before B's), and every emitted element carries its own value.
 */
typedef enum mp_setop {
    MP_SET_UNION = 0,
    MP_SET_INTERSECTION = 1,
    MP_SET_DIFFERENCE = 2,
    MP_SET_SYMMETRIC_DIFFERENCE = 3
} mp_setop;

/* Output capacity (elements) mp_set_operation needs for the set operations
 * above (Sec. I): na + nb for union and
 * symmetric difference, min(na, nb) for intersection, na for difference;
 * -1 for an unknown op or a negative size. */
MP_API int64_t mp_set_capacity(mp_setop op, int64_t na, int64_t nb);

/*
 * mp_set_operation -- set operation `op` of sorted A and B.
 *   a_keys[0..na), b_keys[0..nb): sorted, device.  out_keys (and out_vals
 *   when values are given: any of a_vals, b_vals, out_vals non-NULL) hold
 *   mp_set_capacity(op, na, nb) elements, device, not overlapping an input.
 *   out_count: device pointer to one int64, set to the result length.
 * Kernels: the partition (Alg. 2 at every tile boundary, Cor. 6), then one
 * pass that merges each tile, decides which outputs it keeps, finds the
 * tile's offset in the result from the kept counts of the tiles before it
 * (a look-back over their published counts, tiles taken in order) and
 * writes its kept outputs contiguously there (the last tile also writes the
 * result length); without values the pass runs on one or two persistent
 * CTAs per SM that overlap the copies, walks, look-backs and stores of
 * consecutive tiles.  Scratch from the library pool: about 16 bytes per tile
 * of 2048 to 8832 outputs.  Asynchronous; inputs that are not sorted give
 * an unspecified subsequence and, where a tile's output would pass the
 * capacity, set bit 2 of mp_kernel_error() (that tile writes nothing).
 */
MP_API mp_status mp_set_operation(mp_setop op, mp_dtype dtype,
                                  const void* a_keys, const uint32_t* a_vals, int64_t na,
                                  const void* b_keys, const uint32_t* b_vals, int64_t nb,
                                  void* out_keys, uint32_t* out_vals, int64_t* out_count,
                                  mp_stream_t stream);

/*
 * mp_sort_workspace_bytes -- device workspace that mp_sort needs for n keys
 * (with_values != 0: plus uint32 values): the second buffer between which
 * the merge rounds of Sec. III alternate, plus split points.  0 for n <= 1.
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

/* ------------------------------------------------------------------------
 * Autotuning of tile shapes.  The paper fixes only that segments are equal
 * (Cor. 7); choosing their length and the thread shape per problem size is
 * this library's own and has no counterpart in the paper.
 * ------------------------------------------------------------------------ */

/*
 * mp_autotune_merge -- SYNCHRONOUS.  Times every compiled tile shape of the
 * merge kernels on the given problem (arguments as in mp_merge_plan; the
 * output arrays are overwritten with the merge), each the fastest of `reps`
 * partition + merge runs under CUDA events, and records the fastest for
 * this device, key width, payload choice and size class floor(log2(na+nb)).
 * Later calls with automatic plans (plan NULL or zero fields) in that class
 * use it.  *best (if not NULL) receives it.
 */
MP_API mp_status mp_autotune_merge(mp_dtype dtype,
                                   const void* a_keys, const uint32_t* a_vals, int64_t na,
                                   const void* b_keys, const uint32_t* b_vals, int64_t nb,
                                   void* out_keys, uint32_t* out_vals, int reps, mp_plan* best,
                                   mp_stream_t stream);

/* As mp_autotune_merge, for mp_merge_batched (arguments as there). */
MP_API mp_status mp_autotune_batched(mp_dtype dtype,
                                     const void* a, const int64_t* a_off,
                                     const void* b, const int64_t* b_off,
                                     int64_t nseg, int64_t na_total, int64_t nb_total, void* out,
                                     const uint32_t* a_vals, const uint32_t* b_vals,
                                     uint32_t* out_vals, int reps, mp_plan* best,
                                     mp_stream_t stream);

/* Save / load / clear the tuned-shape table (text, one entry per line).  If
 * the environment variable MP_TUNE_CACHE names a file, it is loaded on first
 * use of an automatic plan. */
MP_API mp_status mp_tune_save(const char* path);
MP_API mp_status mp_tune_load(const char* path);
MP_API void mp_tune_clear(void);

/* ------------------------------------------------------------------------
 * CUDA graphs: capture a merge once, replay it with one launch.  The graph
 * bakes in every pointer and size given at creation (the caller keeps those
 * buffers alive and may change their contents between replays) and owns its
 * scratch, so a replay allocates nothing.  A launch-overhead measure with
 * no counterpart in the paper; the replayed work is Alg. 1 (or the batched
 * merge) unchanged.
 * ------------------------------------------------------------------------ */
typedef struct mp_graph mp_graph;

/* Arguments as mp_merge_plan (values merged when any value pointer is set). */
MP_API mp_status mp_graph_merge_create(mp_dtype dtype,
                                       const void* a_keys, const uint32_t* a_vals, int64_t na,
                                       const void* b_keys, const uint32_t* b_vals, int64_t nb,
                                       void* out_keys, uint32_t* out_vals, const mp_plan* plan,
                                       mp_graph** graph);

/* Arguments as mp_merge_batched (the offsets' contents are read at replay). */
MP_API mp_status mp_graph_batched_create(mp_dtype dtype,
                                         const void* a, const int64_t* a_off,
                                         const void* b, const int64_t* b_off,
                                         int64_t nseg, int64_t na_total, int64_t nb_total,
                                         void* out, const uint32_t* a_vals,
                                         const uint32_t* b_vals, uint32_t* out_vals,
                                         const mp_plan* plan, mp_graph** graph);

/* Enqueue one replay on `stream`. */
MP_API mp_status mp_graph_launch(mp_graph* graph, mp_stream_t stream);

/* Waits for the device, then frees the graph and its scratch. */
MP_API mp_status mp_graph_destroy(mp_graph* graph);

/*
 * mp_kernel_error -- SYNCHRONOUS (waits for the device).  Bit flags set by
 * kernels whose bounded waits ran out (1: an mbarrier wait of a TMA-staged
 * merge timed out; the CTA stopped early and its tiles are incomplete;
 * 2: a set operation's tile output would pass the capacity, which only
 * unsorted inputs cause; that tile wrote nothing; 4: a set operation's
 * bounded wait for an earlier tile's kept count ran out, which only follows
 * flag 1; the tile's place in the output is wrong).
 * 0 means no kernel reported a problem since the last reset.  reset != 0
 * clears the flags after reading them.  (Robustness of this library; no
 * counterpart in the paper.)
 */
MP_API mp_status mp_kernel_error(unsigned int* code, int reset);

/*
 * mp_kernel_status -- waits for `stream`, then turns the flags of
 * mp_kernel_error into a status: MP_ERR_TIMEOUT if flag 1 or 4 is set (a
 * bounded wait ran out, so some output was not written or misplaced),
 * MP_ERR_NOT_SORTED if flag 2 is set (a set operation met unsorted input),
 * else MP_OK.  reset != 0 clears the flags it read.  The flags are shared by
 * all streams of the device.  (Robustness of this library; no counterpart
 * in the paper.)
 */
MP_API mp_status mp_kernel_status(mp_stream_t stream, int reset);

/* Fault kinds of mp_inject_fault. */
typedef enum mp_fault {
    MP_FAULT_SCRATCH_ALLOC = 1, /* the next `count` scratch allocations from the
                                   library's pool fail: the call returns
                                   MP_ERR_NO_MEMORY before enqueuing anything */
    MP_FAULT_QUEUE_STEP = 2,    /* the next `count` steps of any request queue
                                   fail as a rejected launch would, without
                                   launching: every request in such a step
                                   finishes with MP_ERR_CUDA */
    MP_FAULT_STAGE_WAIT = 3     /* count > 0: from now on the first mbarrier
                                   wait of every TMA-staged merge tile gives up
                                   without polling (its bounded drain wait still
                                   lets the copies land), so the tile writes
                                   nothing and flag 1 of mp_kernel_error is set;
                                   count == 0 turns this off.  SYNCHRONOUS:
                                   waits for the device. */
} mp_fault;

/*
 * mp_inject_fault -- a test hook for the error paths: makes failures happen
 * on the host (allocation, queue step) or makes a device wait run out on
 * purpose, without faulting the GPU.  count >= 0 (0 cancels).  Global to
 * the process (the stage-wait switch: to the current device).  Returns
 * MP_ERR_INVALID_ARG for an unknown kind or a negative count.  (Robustness
 * of this library; no counterpart in the paper.)
 */
MP_API mp_status mp_inject_fault(mp_fault kind, int64_t count);

/*
 * mp_merge_noalloc -- the merge of mp_merge_plan (values move when any value
 * pointer is non-NULL) for callers that must not allocate device memory on
 * the call path: code running inside another runtime's memory arena that
 * already holds the device's memory, or latency-critical loops in which an
 * allocation call may block or synchronise.  The paper has no counterpart;
 * this is a deployment variant of Alg. 1.
 *   It calls no cudaMalloc, cudaFree or allocating library routine: the
 *   split points live in a fixed 2 MiB array compiled into the library
 *   (262144 entries, TMA-staged tiles of 4096 outputs, 256 threads x 16
 *   items), which
 *   every GPU that loads the library holds until the process exits.
 *   na + nb may be at most 1073737728; larger sizes return
 *   MP_ERR_INVALID_ARG before anything is enqueued.
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.  Under CUDA's default lazy module loading
 *   that lookup is also when the runtime loads the array's module and so
 *   takes its 2 MiB of device memory: make the first call before another
 *   runtime's arena reserves the device's memory (or set
 *   CUDA_MODULE_LOADING=EAGER).  Later calls take no memory.
 *   All calls share the one array: calls whose work overlaps on the GPU
 *   (other streams, other host threads) race and must not be issued; calls
 *   on one stream are ordered.  No part of the array needs to start at zero
 *   (each call's partition kernel writes every entry its merge kernel reads).
 */
MP_API mp_status mp_merge_noalloc(mp_dtype dtype,
                                  const void* a_keys, const uint32_t* a_vals, int64_t na,
                                  const void* b_keys, const uint32_t* b_vals, int64_t nb,
                                  void* out_keys, uint32_t* out_vals, mp_stream_t stream);

/* One problem of mp_merge_grouped. */
typedef struct mp_merge_desc {
    int32_t dtype;    /* mp_dtype of this problem's keys */
    int32_t reserved; /* must be 0 */
    const void* a_keys;
    const uint32_t* a_vals; /* NULL if keys only (or na == 0) */
    int64_t na;
    const void* b_keys;
    const uint32_t* b_vals;
    int64_t nb;
    void* out_keys; /* na + nb keys */
    uint32_t* out_vals;
} mp_merge_desc;

/*
 * mp_merge_grouped -- nprob independent stable merges, each with its own
 * pointers, in one partition launch and one merge launch (Alg. 1 per
 * problem; every problem is cut into equal tiles, Cor. 7, and the tiles of
 * all problems share one grid).  descs: HOST array of nprob descriptors
 * (copied before the call returns); every problem's arrays follow the
 * rules of mp_merge_pairs (device memory, sorted, no overlap).  All dtypes
 * in one call must have the same key width; with_values != 0 moves values
 * for every problem.  Scratch (descriptor table + split points) comes from
 * the library pool.
 */
MP_API mp_status mp_merge_grouped(const mp_merge_desc* descs, int64_t nprob, int with_values,
                                  mp_stream_t stream);

/*
 * mp_check_sorted -- SYNCHRONOUS check of the precondition of Sec. II.A
 * (inputs sorted): that keys[0..n) is ascending and, for MP_F32, free of
 * NaN.  Returns MP_OK, MP_ERR_NOT_SORTED or MP_ERR_NAN
 * (NaN wins if both).  Waits for `stream`.
 */
MP_API mp_status mp_check_sorted(mp_dtype dtype, const void* keys, int64_t n, mp_stream_t stream);

/* ------------------------------------------------------------------------
 * Request queue: continuous batching of merge and sort requests.
 *
 * Requests are admitted in arrival order while the queue's device-memory
 * budget and slot limit allow; an admitted request keeps its buffers on the
 * device until it completes.  A scheduler thread runs steps; each step
 * advances every admitted request by one stage in one grouped launch per
 * key width and payload choice: a merge is one stage (Alg. 1), a sort is a
 * block-sort stage plus one stage per Merge Path pass (Sec. I, Sec. III), so
 * requests of any size share the GPU and later arrivals join at the next
 * step.  Results are written to the caller's buffers; memory and budget
 * are released as soon as a request's last stage has run.  The paper has
 * no serving layer; this is a systems pattern around its merge.
 * ------------------------------------------------------------------------ */
typedef struct mp_queue mp_queue;

typedef enum mp_op { MP_OP_MERGE = 0, MP_OP_SORT = 1 } mp_op;

/* Where a request's inputs come from. */
typedef enum mp_source {
    MP_SRC_HOST = 0,     /* host arrays, copied in at admission */
    MP_SRC_DEVICE = 1,   /* device arrays, copied in at admission */
    MP_SRC_GENERATE = 2  /* synthetic, generated on the device from `seed` (see mp_generate) */
} mp_source;

/* Where its result goes. */
typedef enum mp_sink {
    MP_SINK_HOST = 0,    /* out_keys/out_vals are host arrays */
    MP_SINK_DEVICE = 1,  /* out_keys/out_vals are device arrays */
    MP_SINK_DISCARD = 2  /* result dropped (load generation) */
} mp_sink;

typedef struct mp_request {
    int32_t op;          /* mp_op */
    int32_t dtype;       /* mp_dtype of the keys */
    int32_t with_values; /* nonzero: uint32 values travel with the keys */
    int32_t source;      /* mp_source */
    int32_t sink;        /* mp_sink */
    int32_t reserved;    /* 0 */
    const void* a_keys;  /* merge: A (sorted); sort: the keys to sort */
    const uint32_t* a_vals;
    int64_t na;          /* merge: |A|; sort: n */
    const void* b_keys;  /* merge: B (sorted); sort: unused */
    const uint32_t* b_vals;
    int64_t nb;          /* merge: |B|; sort: must be 0 */
    uint64_t seed;       /* MP_SRC_GENERATE only */
    void* out_keys;      /* na (+ nb) keys, unless MP_SINK_DISCARD */
    uint32_t* out_vals;
} mp_request;

typedef struct mp_result {
    mp_status status;
    int32_t op;
    int64_t n;           /* number of output elements */
    double t_submit;     /* mp_clock_seconds() at submission */
    double t_admit;      /* ... when admitted (buffers allocated, inputs enqueued) */
    double t_done;       /* ... when the scheduler saw the result copied out */
} mp_result;

typedef struct mp_queue_stats {
    uint64_t submitted, completed, failed;
    uint64_t steps;       /* scheduler steps run */
    uint64_t launches;    /* kernel launches made by steps */
    uint64_t peak_bytes;  /* highest device bytes held by admitted requests */
    uint64_t waiting, active, bytes_in_use;
} mp_queue_stats;

/* Monotonic host clock (seconds) used for the timestamps in mp_result (part
 * of the serving layer, which has no counterpart in the paper). */
MP_API double mp_clock_seconds(void);

/*
 * mp_queue_create -- a queue on the current device.  budget_bytes: device
 * memory that admitted requests may hold together (a request needs about
 * 2 x its output bytes, inputs included); max_active: admitted requests at
 * once.  The queue owns a scheduler thread, two streams and a memory pool.
 */
MP_API mp_status mp_queue_create(size_t budget_bytes, int max_active, mp_queue** q);

/*
 * mp_queue_submit -- non-blocking.  Copies *r; the caller's input arrays
 * must stay valid until the request is admitted and its output arrays until
 * mp_queue_wait reports it done.  MP_ERR_BUDGET if the request alone needs
 * more than the budget; argument errors as for mp_merge_pairs / mp_sort.
 * Generated inputs (MP_SRC_GENERATE) support MP_U32 and MP_U64 keys.
 */
MP_API mp_status mp_queue_submit(mp_queue* q, const mp_request* r, uint64_t* ticket);

/*
 * mp_queue_wait -- wait for a request: timeout_ns < 0 waits without limit,
 * 0 polls (MP_ERR_NOT_READY if not done), > 0 waits at most that long
 * (MP_ERR_TIMEOUT).  On MP_OK, *res holds the request's own status and
 * timestamps and the ticket is retired.
 */
MP_API mp_status mp_queue_wait(mp_queue* q, uint64_t ticket, int64_t timeout_ns, mp_result* res);

MP_API mp_status mp_queue_get_stats(mp_queue* q, mp_queue_stats* stats);

/* Drains all submitted requests, stops the scheduler and frees the queue. */
MP_API mp_status mp_queue_destroy(mp_queue* q);

/*
 * mp_generate -- synthetic keys on the device (the generator behind
 * MP_SRC_GENERATE; input generation, no counterpart in the paper).  SplitMix64 (Steele, Lea, Flood 2014) as a counter-based
 * generator: x_i = mix(seed ^ (stream_id * 0xD1B54A32D192ED03) +
 * (i + 1) * 0x9E3779B97F4A7C15).  sorted != 0: key_i = i * stride +
 * (x_i mod stride) with stride = floor(2^w / n) (strictly increasing);
 * sorted == 0: key_i = top w bits of x_i (w = key bits).  vals (may be NULL)
 * get val_base + i.  MP_U32 or MP_U64 keys.
 */
MP_API mp_status mp_generate(mp_dtype dtype, void* keys, uint32_t* vals, int64_t n, uint64_t seed,
                             uint64_t stream_id, int sorted, uint32_t val_base, mp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* MP_H */
