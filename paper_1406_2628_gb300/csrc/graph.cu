// graph.cu -- CUDA-graph objects for repeated merges.
//
// A merge is two launches (partition, then merge tiles) plus scratch (one
// launch and no scratch with the streaming plan); a
// caller that repeats the same merge on the same buffers (a batched merge
// over fixed segment offsets, a pipeline stage) can capture it once and
// replay it with one cudaGraphLaunch.  The graph owns its scratch (split
// points), allocated when it is created, so a replay allocates nothing.
#include "mp_internal.h"

struct mp_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* scratch = nullptr;
    int device = 0;
};

namespace mp {

template <class F>
static mp_status capture(F&& enqueue, size_t scratch_bytes, mp_graph** out)
{
    mp_graph* g = new (std::nothrow) mp_graph();
    if (!g) return fail(MP_ERR_NO_MEMORY, "mp_graph: allocation");
    cudaStream_t s = nullptr;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaMalloc(&g->scratch, scratch_bytes < 256 ? 256 : scratch_bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = enqueue(g->scratch, s);
        e = cudaStreamEndCapture(s, &g->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        if (g->scratch) cudaFree(g->scratch);
        delete g;
        return cuda_fail(e, "mp_graph: capture");
    }
    *out = g;
    return MP_OK;
}

}  // namespace mp

using namespace mp;

extern "C" {

mp_status mp_graph_merge_create(mp_dtype dtype, const void* a_keys, const uint32_t* a_vals, int64_t na,
                                const void* b_keys, const uint32_t* b_vals, int64_t nb, void* out_keys,
                                uint32_t* out_vals, const mp_plan* plan, mp_graph** graph)
{
    if (!graph) return fail(MP_ERR_INVALID_ARG, "mp_graph_merge_create: NULL result pointer");
    *graph = nullptr;
    MergeProblem p;
    Shape s;
    const bool vals = a_vals || b_vals || out_vals;
    mp_status st = merge_prepare(dtype, a_keys, a_vals, na, b_keys, b_vals, nb, out_keys, out_vals, vals,
                                 plan, "mp_graph_merge_create", &p, &s);
    if (st != MP_OK) return st;
    const bool streaming = s.staging == MP_STAGE_STREAM;
    const int64_t bounds = streaming ? 0 : ceil_div(na + nb, s.tile()) + 1;
    return capture(
        [&](void* scratch, cudaStream_t cs) -> cudaError_t {
            if (na + nb == 0) return cudaSuccess;
            if (streaming) return launch_merge_stream(p, s, cs);
            cudaError_t e = launch_partition(p, s.tile(), (int64_t*)scratch, cs);
            if (e == cudaSuccess) e = launch_merge_tiles(p, s, (const int64_t*)scratch, cs);
            return e;
        },
        (size_t)bounds * 8, graph);
}

mp_status mp_graph_batched_create(mp_dtype dtype, const void* a, const int64_t* a_off, const void* b,
                                  const int64_t* b_off, int64_t nseg, int64_t na_total, int64_t nb_total,
                                  void* out, const uint32_t* a_vals, const uint32_t* b_vals,
                                  uint32_t* out_vals, const mp_plan* plan, mp_graph** graph)
{
    if (!graph) return fail(MP_ERR_INVALID_ARG, "mp_graph_batched_create: NULL result pointer");
    *graph = nullptr;
    BatchedProblem q;
    Shape s;
    mp_status st = batched_prepare(dtype, a, a_off, b, b_off, nseg, na_total, nb_total, out, a_vals, b_vals,
                                   out_vals, plan, &q, &s);
    if (st != MP_OK) return st;
    return capture([&](void* scratch, cudaStream_t cs) { return batched_launch(q, s, scratch, cs); },
                   batched_scratch_bytes(q, s), graph);
}

mp_status mp_graph_launch(mp_graph* g, mp_stream_t stream)
{
    if (!g) return fail(MP_ERR_INVALID_ARG, "mp_graph_launch: NULL graph");
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? MP_OK : cuda_fail(e, "mp_graph_launch");
}

mp_status mp_graph_destroy(mp_graph* g)
{
    if (!g) return MP_OK;
    // The scratch may still be read by a replay in flight: wait for the
    // device before freeing it (cudaFree would synchronise anyway).
    cudaError_t e = cudaDeviceSynchronize();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->scratch) cudaFree(g->scratch);
    delete g;
    return e == cudaSuccess ? MP_OK : cuda_fail(e, "mp_graph_destroy");
}

}  // extern "C"
