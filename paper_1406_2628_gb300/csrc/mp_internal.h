// mp_internal.h -- host-side declarations shared by the library's sources.
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "mp.h"

namespace mp {

// Key width and codec parameters of a dtype (see Codec in mp_device.cuh).
struct KeyKind {
    int bytes;       // 4 or 8
    uint64_t flip;   // top bit for signed and float keys
    uint64_t fmask;  // all ones for float keys
};
bool key_kind(mp_dtype dtype, KeyKind* out);

// A merge tile shape: NT threads x VT items per thread.
struct Shape {
    int nt;
    int vt;
    int staging;  // MP_STAGE_VECTOR or MP_STAGE_BULK
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
Shape default_merge_shape(int key_bytes, bool with_values, int64_t total);

// Merge sort.
size_t sort_workspace_bytes(const KeyKind& kind, int64_t n, bool with_values);
mp_status sort_run(const KeyKind& kind, void* keys, uint32_t* vals, int64_t n, void* ws,
                   size_t ws_bytes, cudaStream_t stream);

// Errors: record a detail for mp_last_error() and return the status.
mp_status fail(mp_status st, const std::string& detail);
mp_status cuda_fail(cudaError_t err, const char* where);

// Stream-ordered scratch from the library's memory pool on the current device.
mp_status scratch_alloc(void** ptr, size_t bytes, cudaStream_t stream);
void scratch_free(void* ptr, cudaStream_t stream);

}  // namespace mp
