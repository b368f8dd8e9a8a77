// mp_internal.h -- host-side declarations shared by the library's sources.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "mp.h"

namespace mp {

// Key width and codec parameters of a dtype (see Codec in mp_device.cuh).
struct KeyKind {
    int bytes;       // 4 or 8
    uint64_t flip;   // top bit for signed and float keys
    uint64_t fmask;  // all ones for float keys
    uint64_t inv;    // all ones for descending order (MP_DESCENDING)
    bool identity() const { return flip == 0 && fmask == 0 && inv == 0; }
    // Ascending signed integers / ascending floats (fixed codecs).
    bool signed_int() const { return flip != 0 && fmask == 0 && inv == 0; }
    bool ascending_float() const { return fmask != 0 && inv == 0; }
};
bool key_kind(mp_dtype dtype, KeyKind* out);

// A merge tile shape: NT threads x VT items per thread.
struct Shape {
    int nt;
    int vt;
    int staging;  // MP_STAGE_VECTOR, _BULK, _WARP or _STREAM
    int64_t tile() const { return (int64_t)nt * vt; }
};

// One merge problem for the tile kernels.  run == 0: a single merge of
// a[0..na) and b[0..nb).  run > 0: one pass of the merge sort over
// a[0..na) (b unused, nb = 0): run pairs [2jw, 2jw+w) and [2jw+w, 2jw+2w)
// with w = run are merged, each into the same positions of out.
struct MergeProblem {
    KeyKind kind;
    const void* a;
    const void* b;
    bool vals;           // move uint32 values with the keys
    const uint32_t* av;  // may be NULL when its side is empty
    const uint32_t* bv;
    void* out;
    uint32_t* outv;
    int64_t na;
    int64_t nb;
    int64_t run;
    int64_t total() const { return run ? na : na + nb; }
};

inline int64_t ceil_div(int64_t x, int64_t y) { return (x + y - 1) / y; }

// Split points at diagonals min(t * spacing, total), t = 0..ceil(total/spacing).
cudaError_t launch_partition(const MergeProblem& p, int64_t spacing, int64_t* a_split,
                             cudaStream_t stream);
// One CTA per tile of shape.tile() outputs; a_split from launch_partition
// with spacing = shape.tile().
cudaError_t launch_merge_tiles(const MergeProblem& p, const Shape& shape, const int64_t* a_split,
                               cudaStream_t stream);
bool merge_shape_supported(int key_bytes, bool with_values, const Shape& shape);
// The TMA-staged tile kernels (merge_bulk.cu): 4- and 8-byte keys in the
// MP_BULK_SHAPES, 16-byte keys in the MP_WIDE_SHAPES (NT, VT).
#define MP_BULK_SHAPES(X) X(128, 8) X(256, 8) X(128, 12) X(256, 12) X(128, 16) X(256, 16) X(128, 27) X(128, 33) X(256, 33)
#define MP_WIDE_SHAPES(X) X(128, 8) X(256, 8) X(128, 12) X(128, 9)
cudaError_t launch_merge_bulk(const MergeProblem& p, const Shape& shape, const int64_t* a_split,
                              cudaStream_t stream);
// Partition-free streaming merge (stream.cu): one launch, no scratch.
cudaError_t launch_merge_stream(const MergeProblem& p, const Shape& shape, cudaStream_t stream);
bool stream_shape_supported(const Shape& shape);
std::vector<Shape> stream_shapes();
// Automatic plans use the streaming merge up to this many outputs.
int64_t stream_auto_limit(int key_bytes, bool with_values);
Shape stream_default_shape(int key_bytes, bool with_values);
Shape default_merge_shape(int key_bytes, bool with_values, int64_t total);  // tuned table first
Shape builtin_merge_shape(int key_bytes, bool with_values);                 // the shipped default
std::vector<Shape> merge_shapes();

// Autotuner cache (tune.cu): op is "merge" or "batched".
bool tuned_shape(const char* op, int key_bytes, bool vals, int64_t total, Shape* s);
void record_shape(const char* op, int key_bytes, bool vals, int64_t total, const Shape& s);

// Batched merge (batched.cu): validation, then launch with caller scratch of
// batched_scratch_bytes() bytes.
struct BatchedProblem {
    KeyKind kind;
    const void* a;
    const void* b;
    const int64_t* a_off;
    const int64_t* b_off;
    int64_t nseg, na, nb;
    void* out;
    bool vals;
    const uint32_t* av;
    const uint32_t* bv;
    uint32_t* outv;
};
mp_status batched_prepare(mp_dtype dtype, const void* a, const int64_t* a_off, const void* b,
                          const int64_t* b_off, int64_t nseg, int64_t na_total, int64_t nb_total,
                          void* out, const uint32_t* a_vals, const uint32_t* b_vals,
                          uint32_t* out_vals, const mp_plan* plan, BatchedProblem* q, Shape* s);
size_t batched_scratch_bytes(const BatchedProblem& q, const Shape& s);
cudaError_t batched_launch(const BatchedProblem& q, const Shape& s, void* scratch, cudaStream_t stream);

// Plain merge: validation, then launch with caller scratch (split points).
mp_status merge_prepare(mp_dtype dtype, const void* a, const uint32_t* av, int64_t na,
                        const void* b, const uint32_t* bv, int64_t nb, void* out, uint32_t* outv,
                        bool vals, const mp_plan* plan, const char* fn, MergeProblem* p, Shape* s,
                        bool allow_stream = true);

// Merge sort.
size_t sort_workspace_bytes(const KeyKind& kind, int64_t n, bool with_values);
mp_status sort_run(const KeyKind& kind, void* keys, uint32_t* vals, int64_t n, void* ws,
                   size_t ws_bytes, cudaStream_t stream);

// Grouped launches (grouped.cu): many independent problems, each with its
// own pointers and codec, one key width per launch.
struct GroupMergeDesc {
    const void* a;
    const void* b;
    const uint32_t* av;
    const uint32_t* bv;
    void* out;
    uint32_t* outv;
    int64_t na, nb, run;  // run > 0: sort pass over a[0..na) (see MergeProblem)
    uint64_t flip, fmask, inv;
};
struct GroupSortDesc {
    const void* in;
    const uint32_t* vin;
    void* out;
    uint32_t* vout;
    int64_t n;
    uint64_t flip, fmask, inv;
};
// tile_first[p]: first tile of problem p (prefix of ceil(total/T));
// bound_first[p] = tile_first[p] + p; d_splits: total_tiles + nprob int64.
// identity: every problem has unsigned ascending keys (compiled codec).
cudaError_t launch_grouped_merge(int key_bytes, bool vals, const GroupMergeDesc* d_descs,
                                 const int64_t* d_tile_first, const int64_t* d_bound_first,
                                 int nprob, int64_t total_tiles, int64_t* d_splits, bool identity,
                                 cudaStream_t stream);
cudaError_t launch_grouped_block_sort(int key_bytes, bool vals, const GroupSortDesc* d_descs,
                                      const int64_t* d_tile_first, int nprob, int64_t total_tiles,
                                      cudaStream_t stream);
int64_t grouped_merge_tile(int key_bytes);
int64_t grouped_sort_tile(int key_bytes);

// Merge argument checks (api.cu).
mp_status check_merge_args_ext(const KeyKind& k, const void* a, const uint32_t* av, int64_t na,
                               const void* b, const uint32_t* bv, int64_t nb, const void* out,
                               const uint32_t* outv, bool vals, const char* fn, int64_t out_n = -1);

// Merge-based set operations (setops.cu): splits from launch_partition with
// spacing setop_tile(key bytes, values); status: one zeroed 64-bit word per
// tile, tile_counter: one zeroed word.
int64_t setop_tile(int key_bytes, bool vals);
cudaError_t launch_setop(const MergeProblem& p, int op, const int64_t* splits, unsigned long long* status,
                         unsigned int* tile_counter, int64_t cap, int64_t* count, cudaStream_t stream);

// Read-only merge (results folded into a checksum, merge.cu).
int64_t checksum_tile(int key_bytes, bool vals);
// partial: one uint64 per tile (scratch), sum: the result word.
cudaError_t launch_merge_checksum(const MergeProblem& p, const int64_t* a_split,
                                  unsigned long long* partial, unsigned long long* sum,
                                  cudaStream_t stream);

// Device address of the word kernels set when a bounded wait runs out.
// The word after it is the staging-wait fault switch (mp_inject_fault):
// nonzero makes bulk_stage's first wait give up without polling.
unsigned int* kernel_error_word();
cudaError_t set_stage_wait_fault(bool on);

// Host-side fault injection: true (and one fewer left) if the next event of
// this mp_fault kind is to fail.
bool take_fault(int kind);

// An NVTX range around a public call or a serving step (shows up in a
// profiler's timeline; without a profiler attached it costs a branch).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define MP_RANGE(name) ::mp::NvtxRange mp_nvtx_range_(name)

// Errors: record a detail for mp_last_error() and return the status.
mp_status fail(mp_status st, const std::string& detail);
mp_status cuda_fail(cudaError_t err, const char* where);

// Stream-ordered scratch from the library's memory pool on the current device.
mp_status scratch_alloc(void** ptr, size_t bytes, cudaStream_t stream);
void scratch_free(void* ptr, cudaStream_t stream);

}  // namespace mp
