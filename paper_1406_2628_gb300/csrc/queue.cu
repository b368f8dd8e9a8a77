// queue.cu -- request queue with continuous batching (mp_queue_*).
//
// Requests (a merge of two sorted arrays, or a sort) are admitted in
// arrival order as long as the device-memory budget and the slot limit
// allow; admitted requests keep their buffers resident on the device until
// they complete.  A scheduler thread runs steps: each step advances every
// admitted request by one stage with one grouped launch per key width and
// payload choice (grouped.cu): a merge needs one stage (Alg. 1), a sort
// needs a block-sort stage and then one stage per Merge Path pass (Sec. I,
// Sec. III), so sorts of any size progress pass by pass beside merges and
// beside requests that arrive later.  Results are copied to the caller's
// buffers (host or device) and the request's memory and budget are
// released as soon as its last stage has run.  Every host wait is bounded.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mp_device.cuh"
#include "mp_internal.h"

namespace mp {

static double clock_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------------
// Synthetic inputs for MP_SRC_GENERATE, SplitMix64 as a counter-based
// generator (Steele, Lea, Flood 2014): element i of stream s under seed k is
// mix(k ^ (s * 0xD1B54A32D192ED03) + (i + 1) * 0x9E3779B97F4A7C15).
// Sorted arrays: key[i] = i * stride + (x_i mod stride), stride =
// floor(2^w / n) (w = key bits), strictly increasing when stride >= 1.
// Unsorted arrays (sort requests): key[i] = top w bits of x_i.
// Values: the element's source index (B's indices follow A's).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix_at(uint64_t seed, uint64_t stream, uint64_t i)
{
    uint64_t z = (seed ^ (stream * 0xD1B54A32D192ED03ull)) + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class K>
__global__ void generate_kernel(K* keys, uint32_t* vals, int64_t n, uint64_t seed, uint64_t stream,
                                int sorted, uint32_t val_base)
{
    const uint64_t stride64 = sizeof(K) == 8 ? (~0ull) / (uint64_t)(n > 0 ? n : 1)
                                             : (0x100000000ull / (uint64_t)(n > 0 ? n : 1));
    const uint64_t stride = stride64 > 0 ? stride64 : 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = splitmix_at(seed, stream, (uint64_t)i);
        K k;
        if (sorted)
            k = (K)((uint64_t)i * stride + x % stride);
        else
            k = sizeof(K) == 8 ? (K)x : (K)(x >> 32);
        keys[i] = k;
        if (vals) vals[i] = val_base + (uint32_t)i;
    }
}

static cudaError_t generate(int key_bytes, void* keys, uint32_t* vals, int64_t n, uint64_t seed,
                            uint64_t stream_id, bool sorted, uint32_t val_base, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t blocks = ceil_div(n, threads);
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (key_bytes == 4)
        generate_kernel<uint32_t><<<(unsigned)blocks, threads, 0, s>>>((uint32_t*)keys, vals, n, seed,
                                                                       stream_id, sorted ? 1 : 0, val_base);
    else
        generate_kernel<uint64_t><<<(unsigned)blocks, threads, 0, s>>>((uint64_t*)keys, vals, n, seed,
                                                                       stream_id, sorted ? 1 : 0, val_base);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Jobs.
// ---------------------------------------------------------------------------
enum JobState { JOB_WAITING = 0, JOB_ACTIVE = 1, JOB_DONE = 2 };

struct Job {
    uint64_t ticket = 0;
    mp_request req = {};
    KeyKind kind = {};
    bool vals = false;
    int64_t n = 0;
    size_t bytes = 0;
    char* mem = nullptr;
    void* x = nullptr;  // merge: A, then B, then out; sort: X (result) and Y
    void* b = nullptr;
    void* out = nullptr;
    uint32_t* xv = nullptr;
    uint32_t* bv = nullptr;
    uint32_t* outv = nullptr;
    void* y = nullptr;
    uint32_t* yv = nullptr;
    int stage = 0;
    int nstages = 1;
    int passes = 0;
    bool last_enqueued = false;
    cudaEvent_t ready = nullptr;
    cudaEvent_t done = nullptr;
    bool wait_ready = false;
    mp_status status = MP_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int state = JOB_WAITING;
};

}  // namespace mp

using namespace mp;

struct mp_queue {
    int device = 0;
    size_t budget = 0;
    int max_active = 0;
    std::mutex mu;
    std::condition_variable cv_work;
    std::condition_variable cv_done;
    std::deque<Job*> waiting;
    std::vector<Job*> active;
    std::unordered_map<uint64_t, Job*> jobs;
    uint64_t next_ticket = 1;
    size_t used = 0;
    bool stop = false;
    std::thread worker;
    cudaStream_t s_compute = nullptr;
    cudaStream_t s_copy = nullptr;
    cudaMemPool_t pool = nullptr;
    // Step resources, double-buffered by step parity.
    cudaEvent_t step_ev[2] = {nullptr, nullptr};
    bool step_used[2] = {false, false};
    char* h_table[2] = {nullptr, nullptr};
    size_t h_table_bytes[2] = {0, 0};
    char* d_table[2] = {nullptr, nullptr};
    size_t d_table_bytes[2] = {0, 0};
    // Statistics.
    mp_queue_stats stats = {};
};

namespace mp {

static void finish_job_locked(mp_queue* q, Job* j, mp_status st)
{
    j->status = st;
    j->t_done = clock_s();
    j->state = JOB_DONE;
    if (j->mem) cudaFreeAsync(j->mem, q->s_compute);
    j->mem = nullptr;
    q->used -= j->bytes;
    if (j->ready) cudaEventDestroy(j->ready);
    if (j->done) cudaEventDestroy(j->done);
    j->ready = j->done = nullptr;
    q->stats.completed++;
    if (st != MP_OK) q->stats.failed++;
}

static int block_sort_passes(int key_bytes, int64_t n)
{
    const int64_t bt = grouped_sort_tile(key_bytes);
    int64_t blocks = ceil_div(n, bt);
    int p = 0;
    while (((int64_t)1 << p) < blocks) ++p;
    return p;
}

static size_t job_bytes(const mp_request& r, const KeyKind& k)
{
    const bool vals = r.with_values != 0;
    const size_t per = (size_t)k.bytes + (vals ? 4 : 0);
    if (r.op == MP_OP_MERGE) {
        const int64_t n = r.na + r.nb;
        return al256((size_t)r.na * k.bytes) + al256((size_t)r.nb * k.bytes) + al256((size_t)n * k.bytes) +
               (vals ? al256((size_t)r.na * 4) + al256((size_t)r.nb * 4) + al256((size_t)n * 4) : 0) + 256;
    }
    (void)per;
    return 2 * (al256((size_t)r.na * k.bytes) + (vals ? al256((size_t)r.na * 4) : 0)) + 256;
}

// Allocate the job's device block and enqueue its inputs on the copy stream.
static mp_status admit(mp_queue* q, Job* j)
{
    const KeyKind& k = j->kind;
    const mp_request& r = j->req;
    cudaError_t e = cudaMallocFromPoolAsync((void**)&j->mem, j->bytes, q->pool, q->s_copy);
    if (e != cudaSuccess) return cuda_fail(e, "queue admission: allocation");
    char* p = j->mem;
    auto carve = [&](size_t bytes) { char* r0 = p; p += al256(bytes); return r0; };
    if (r.op == MP_OP_MERGE) {
        j->x = carve((size_t)r.na * k.bytes);
        j->b = carve((size_t)r.nb * k.bytes);
        j->out = carve((size_t)j->n * k.bytes);
        if (j->vals) {
            j->xv = (uint32_t*)carve((size_t)r.na * 4);
            j->bv = (uint32_t*)carve((size_t)r.nb * 4);
            j->outv = (uint32_t*)carve((size_t)j->n * 4);
        }
    } else {
        j->x = carve((size_t)r.na * k.bytes);
        j->y = carve((size_t)r.na * k.bytes);
        if (j->vals) {
            j->xv = (uint32_t*)carve((size_t)r.na * 4);
            j->yv = (uint32_t*)carve((size_t)r.na * 4);
        }
        j->out = j->x;
        j->outv = j->xv;
    }
    const size_t kb = (size_t)k.bytes;
    if (r.source == MP_SRC_GENERATE) {
        if (r.op == MP_OP_MERGE) {
            e = generate(k.bytes, j->x, j->xv, r.na, r.seed, 1, true, 0, q->s_copy);
            if (e == cudaSuccess) e = generate(k.bytes, j->b, j->bv, r.nb, r.seed, 2, true, (uint32_t)r.na, q->s_copy);
        } else {
            e = generate(k.bytes, j->x, j->xv, r.na, r.seed, 3, false, 0, q->s_copy);
        }
    } else {
        const cudaMemcpyKind kind = r.source == MP_SRC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        if (r.na) e = cudaMemcpyAsync(j->x, r.a_keys, r.na * kb, kind, q->s_copy);
        if (e == cudaSuccess && j->vals && r.na) e = cudaMemcpyAsync(j->xv, r.a_vals, r.na * 4, kind, q->s_copy);
        if (r.op == MP_OP_MERGE) {
            if (e == cudaSuccess && r.nb) e = cudaMemcpyAsync(j->b, r.b_keys, r.nb * kb, kind, q->s_copy);
            if (e == cudaSuccess && j->vals && r.nb) e = cudaMemcpyAsync(j->bv, r.b_vals, r.nb * 4, kind, q->s_copy);
        }
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(j->ready, q->s_copy);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "queue admission: inputs");
    j->wait_ready = true;
    j->t_admit = clock_s();
    j->state = JOB_ACTIVE;
    return MP_OK;
}

// Copy the result out (after its last stage) and record completion.
static cudaError_t enqueue_result(mp_queue* q, Job* j)
{
    const mp_request& r = j->req;
    cudaError_t e = cudaSuccess;
    const size_t kb = (size_t)j->kind.bytes;
    if (r.sink != MP_SINK_DISCARD && j->n > 0) {
        const cudaMemcpyKind kind = r.sink == MP_SINK_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        e = cudaMemcpyAsync(r.out_keys, j->out, j->n * kb, kind, q->s_compute);
        if (e == cudaSuccess && j->vals) e = cudaMemcpyAsync(r.out_vals, j->outv, j->n * 4, kind, q->s_compute);
    }
    if (e == cudaSuccess) e = cudaEventRecord(j->done, q->s_compute);
    return e;
}

struct StepGroups {
    std::vector<GroupMergeDesc> m[2][2];  // [key width 4/8][values]
    std::vector<GroupSortDesc> s[2][2];
};

static cudaError_t grow_tables(mp_queue* q, int slot, size_t bytes)
{
    if (q->h_table_bytes[slot] < bytes) {
        if (q->h_table[slot]) cudaFreeHost(q->h_table[slot]);
        size_t nb = std::max(bytes, (size_t)1 << 20);
        cudaError_t e = cudaMallocHost((void**)&q->h_table[slot], nb);
        if (e != cudaSuccess) { q->h_table[slot] = nullptr; q->h_table_bytes[slot] = 0; return e; }
        q->h_table_bytes[slot] = nb;
    }
    if (q->d_table_bytes[slot] < bytes) {
        if (q->d_table[slot]) cudaFree(q->d_table[slot]);
        size_t nb = std::max(bytes, (size_t)1 << 20);
        cudaError_t e = cudaMalloc((void**)&q->d_table[slot], nb);
        if (e != cudaSuccess) { q->d_table[slot] = nullptr; q->d_table_bytes[slot] = 0; return e; }
        q->d_table_bytes[slot] = nb;
    }
    return cudaSuccess;
}

// Build and launch one step over the given jobs; returns the number of
// kernel launches.
static cudaError_t run_step(mp_queue* q, std::vector<Job*>& work, int slot, uint64_t* launches)
{
    MP_RANGE("mp_queue step");
    // An injected fault (mp_inject_fault) fails the step the way a rejected
    // launch would, before anything is enqueued.
    if (take_fault(MP_FAULT_QUEUE_STEP)) return cudaErrorInvalidConfiguration;
    StepGroups g;
    for (Job* j : work) {
        const int w = j->kind.bytes == 8 ? 1 : 0;
        const int v = j->vals ? 1 : 0;
        if (j->req.op == MP_OP_MERGE) {
            GroupMergeDesc d = {j->x, j->b, j->xv, j->bv, j->out, j->outv, j->req.na, j->req.nb, 0,
                                j->kind.flip, j->kind.fmask, j->kind.inv};
            g.m[w][v].push_back(d);
        } else if (j->stage == 0) {
            // Block sort into the buffer from which an even number of
            // remaining passes ends in X.
            void* dst = (j->passes & 1) ? j->y : j->x;
            uint32_t* dstv = (j->passes & 1) ? j->yv : j->xv;
            GroupSortDesc d = {j->x, j->xv, dst, dstv, j->n, j->kind.flip, j->kind.fmask, j->kind.inv};
            g.s[w][v].push_back(d);
        } else {
            const int p = j->stage - 1;  // pass index
            const bool src_is_y = ((j->passes - p) & 1) != 0;
            void* src = src_is_y ? j->y : j->x;
            uint32_t* srcv = src_is_y ? j->yv : j->xv;
            void* dst = src_is_y ? j->x : j->y;
            uint32_t* dstv = src_is_y ? j->xv : j->yv;
            GroupMergeDesc d = {src, src, srcv, srcv, dst, dstv, j->n, 0,
                                grouped_sort_tile(j->kind.bytes) << p, j->kind.flip, j->kind.fmask,
                                j->kind.inv};
            g.m[w][v].push_back(d);
        }
    }
    // Lay out every group's table in one pinned buffer: descriptors, tile
    // firsts, boundary firsts, then the split scratch (device only).
    struct Plan { int kind; int w; int v; size_t off_desc, off_first, off_splits; int n; int64_t tiles; };
    std::vector<Plan> plans;
    size_t off = 0;
    for (int w = 0; w < 2; ++w)
        for (int v = 0; v < 2; ++v) {
            if (!g.s[w][v].empty()) {
                Plan pl{1, w, v, 0, 0, 0, (int)g.s[w][v].size(), 0};
                pl.off_desc = off; off = al256(off + pl.n * sizeof(GroupSortDesc));
                pl.off_first = off; off = al256(off + (size_t)pl.n * 8);
                plans.push_back(pl);
            }
            if (!g.m[w][v].empty()) {
                Plan pl{0, w, v, 0, 0, 0, (int)g.m[w][v].size(), 0};
                pl.off_desc = off; off = al256(off + pl.n * sizeof(GroupMergeDesc));
                pl.off_first = off; off = al256(off + (size_t)pl.n * 16);
                plans.push_back(pl);
            }
        }
    const size_t table_bytes = off;
    size_t split_bytes = 0;
    for (Plan& pl : plans) {
        const int kb = pl.w ? 8 : 4;
        if (pl.kind == 1) {
            int64_t t = 0;
            for (auto& d : g.s[pl.w][pl.v]) t += ceil_div(d.n, grouped_sort_tile(kb));
            pl.tiles = t;
        } else {
            int64_t t = 0;
            for (auto& d : g.m[pl.w][pl.v]) t += ceil_div(d.run ? d.na : d.na + d.nb, grouped_merge_tile(kb));
            pl.tiles = t;
            pl.off_splits = al256(table_bytes) + split_bytes;
            split_bytes = al256(split_bytes + (size_t)(t + pl.n) * 8);
        }
    }
    cudaError_t e = grow_tables(q, slot, al256(table_bytes) + split_bytes);
    if (e != cudaSuccess) return e;
    char* h = q->h_table[slot];
    char* dt = q->d_table[slot];
    for (Plan& pl : plans) {
        const int kb = pl.w ? 8 : 4;
        int64_t* first = (int64_t*)(h + pl.off_first);
        if (pl.kind == 1) {
            auto& v = g.s[pl.w][pl.v];
            memcpy(h + pl.off_desc, v.data(), v.size() * sizeof(GroupSortDesc));
            int64_t t = 0;
            for (size_t i = 0; i < v.size(); ++i) { first[i] = t; t += ceil_div(v[i].n, grouped_sort_tile(kb)); }
        } else {
            auto& v = g.m[pl.w][pl.v];
            memcpy(h + pl.off_desc, v.data(), v.size() * sizeof(GroupMergeDesc));
            int64_t t = 0;
            for (size_t i = 0; i < v.size(); ++i) {
                first[i] = t;
                first[v.size() + i] = t + (int64_t)i;
                t += ceil_div(v[i].run ? v[i].na : v[i].na + v[i].nb, grouped_merge_tile(kb));
            }
        }
    }
    if (table_bytes) e = cudaMemcpyAsync(dt, h, table_bytes, cudaMemcpyHostToDevice, q->s_compute);
    if (e != cudaSuccess) return e;
    // Block sorts first (a request's block sort and its first pass are in
    // different steps, so order within a step does not matter).
    for (Plan& pl : plans) {
        const int kb = pl.w ? 8 : 4;
        if (pl.kind == 1) {
            e = launch_grouped_block_sort(kb, pl.v != 0, (const GroupSortDesc*)(dt + pl.off_desc),
                                          (const int64_t*)(dt + pl.off_first), pl.n, pl.tiles, q->s_compute);
            *launches += 1;
        } else {
            bool identity = true;  // every problem of the launch has unsigned ascending keys
            for (const GroupMergeDesc& d : g.m[pl.w][pl.v]) identity = identity && !d.flip && !d.fmask && !d.inv;
            e = launch_grouped_merge(kb, pl.v != 0, (const GroupMergeDesc*)(dt + pl.off_desc),
                                     (const int64_t*)(dt + pl.off_first), (const int64_t*)(dt + pl.off_first) + pl.n,
                                     pl.n, pl.tiles, (int64_t*)(dt + pl.off_splits), identity, q->s_compute);
            *launches += pl.tiles ? 2 : 1;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static void worker_main(mp_queue* q)
{
    cudaSetDevice(q->device);
    uint64_t step = 0;
    std::vector<Job*> work;
    std::vector<Job*> completing;
    for (;;) {
        work.clear();
        completing.clear();
        {
            std::unique_lock<std::mutex> lk(q->mu);
            // Completions.
            for (size_t i = 0; i < q->active.size();) {
                Job* j = q->active[i];
                if (j->last_enqueued) {
                    cudaError_t qe = cudaEventQuery(j->done);
                    if (qe != cudaErrorNotReady) {
                        // A status recorded when the job's step failed to
                        // launch stands, although its done event completes.
                        const mp_status st = j->status != MP_OK ? j->status
                                             : qe == cudaSuccess ? MP_OK
                                                                 : cuda_fail(qe, "queue step");
                        finish_job_locked(q, j, st);
                        q->active[i] = q->active.back();
                        q->active.pop_back();
                        q->cv_done.notify_all();
                        continue;
                    }
                }
                ++i;
            }
            // Admissions, strictly in arrival order (no starvation).
            while (!q->waiting.empty() && (int)q->active.size() < q->max_active &&
                   q->used + q->waiting.front()->bytes <= q->budget) {
                Job* j = q->waiting.front();
                q->waiting.pop_front();
                q->used += j->bytes;
                q->stats.peak_bytes = std::max<uint64_t>(q->stats.peak_bytes, q->used);
                mp_status st = admit(q, j);
                if (st != MP_OK) {
                    finish_job_locked(q, j, st);
                    q->cv_done.notify_all();
                    continue;
                }
                q->active.push_back(j);
            }
            for (Job* j : q->active)
                if (!j->last_enqueued) work.push_back(j);
            if (work.empty()) {
                if (q->stop && q->waiting.empty() && q->active.empty()) break;
                if (q->active.empty())
                    q->cv_work.wait_for(lk, std::chrono::milliseconds(2));
                else {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(20));
                }
                continue;
            }
        }
        // At most two steps in flight: wait for the step that used this
        // slot's tables (bounded by that step's own duration).
        const int slot = (int)(step & 1);
        if (q->step_used[slot]) cudaEventSynchronize(q->step_ev[slot]);
        for (Job* j : work)
            if (j->wait_ready) {
                cudaStreamWaitEvent(q->s_compute, j->ready, 0);
                j->wait_ready = false;
            }
        uint64_t launches = 0;
        cudaError_t e = run_step(q, work, slot, &launches);
        for (Job* j : work) {
            j->stage++;
            if (j->stage >= j->nstages) completing.push_back(j);
        }
        for (Job* j : completing)
            if (e == cudaSuccess) e = enqueue_result(q, j);
        if (e == cudaSuccess) e = cudaEventRecord(q->step_ev[slot], q->s_compute);
        q->step_used[slot] = true;
        std::unique_lock<std::mutex> lk(q->mu);
        q->stats.steps++;
        q->stats.launches += launches;
        if (e != cudaSuccess) {
            mp_status st = cuda_fail(e, "queue step");
            for (Job* j : work) {
                j->last_enqueued = true;
                cudaEventRecord(j->done, q->s_compute);
                j->status = st;
            }
        } else {
            for (Job* j : completing) j->last_enqueued = true;
        }
        ++step;
    }
}

}  // namespace mp

extern "C" {

double mp_clock_seconds(void) { return clock_s(); }

mp_status mp_queue_create(size_t budget_bytes, int max_active, mp_queue** out)
{
    if (!out) return fail(MP_ERR_INVALID_ARG, "mp_queue_create: NULL result pointer");
    *out = nullptr;
    if (budget_bytes == 0 || max_active <= 0) return fail(MP_ERR_INVALID_ARG, "mp_queue_create: zero budget or slots");
    mp_queue* q = new (std::nothrow) mp_queue();
    if (!q) return fail(MP_ERR_NO_MEMORY, "mp_queue_create");
    cudaError_t e = cudaGetDevice(&q->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->s_compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->s_copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->step_ev[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->step_ev[1], cudaEventDisableTiming);
    if (e == cudaSuccess) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = q->device;
        e = cudaMemPoolCreate(&q->pool, &props);
        if (e == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(q->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e != cudaSuccess) {
        mp_status st = cuda_fail(e, "mp_queue_create");
        if (q->s_compute) cudaStreamDestroy(q->s_compute);
        if (q->s_copy) cudaStreamDestroy(q->s_copy);
        for (auto& ev : q->step_ev) if (ev) cudaEventDestroy(ev);
        if (q->pool) cudaMemPoolDestroy(q->pool);
        delete q;
        return st;
    }
    q->budget = budget_bytes;
    q->max_active = max_active;
    q->worker = std::thread(worker_main, q);
    *out = q;
    return MP_OK;
}

mp_status mp_queue_submit(mp_queue* q, const mp_request* r, uint64_t* ticket)
{
    if (!q || !r || !ticket) return fail(MP_ERR_INVALID_ARG, "mp_queue_submit: NULL argument");
    KeyKind k;
    if (!key_kind((mp_dtype)r->dtype, &k) || k.bytes == 16)
        return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_queue_submit: unknown or 128-bit dtype");
    if (r->op != MP_OP_MERGE && r->op != MP_OP_SORT) return fail(MP_ERR_INVALID_ARG, "mp_queue_submit: unknown op");
    if (r->source != MP_SRC_HOST && r->source != MP_SRC_DEVICE && r->source != MP_SRC_GENERATE)
        return fail(MP_ERR_INVALID_ARG, "mp_queue_submit: unknown source");
    if (r->sink != MP_SINK_HOST && r->sink != MP_SINK_DEVICE && r->sink != MP_SINK_DISCARD)
        return fail(MP_ERR_INVALID_ARG, "mp_queue_submit: unknown sink");
    if (r->na < 0 || r->nb < 0 || (r->op == MP_OP_SORT && r->nb != 0))
        return fail(MP_ERR_INVALID_ARG, "mp_queue_submit: bad sizes (sorts use na only)");
    if (r->source == MP_SRC_GENERATE && r->dtype != MP_U32 && r->dtype != MP_U64)
        return fail(MP_ERR_INVALID_ARG, "mp_queue_submit: generated inputs are MP_U32 or MP_U64 keys");
    const bool vals = r->with_values != 0;
    if (r->source != MP_SRC_GENERATE) {
        if ((r->na > 0 && !r->a_keys) || (r->op == MP_OP_MERGE && r->nb > 0 && !r->b_keys) ||
            (vals && ((r->na > 0 && !r->a_vals) || (r->op == MP_OP_MERGE && r->nb > 0 && !r->b_vals))))
            return fail(MP_ERR_INVALID_ARG, "mp_queue_submit: NULL input pointer");
    }
    const int64_t n = r->na + (r->op == MP_OP_MERGE ? r->nb : 0);
    if (r->sink != MP_SINK_DISCARD && n > 0 && (!r->out_keys || (vals && !r->out_vals)))
        return fail(MP_ERR_INVALID_ARG, "mp_queue_submit: NULL output pointer");
    Job* j = new (std::nothrow) Job();
    if (!j) return fail(MP_ERR_NO_MEMORY, "mp_queue_submit");
    j->req = *r;
    j->kind = k;
    j->vals = vals;
    j->n = n;
    j->bytes = job_bytes(*r, k);
    if (r->op == MP_OP_SORT) {
        j->passes = n > 1 ? block_sort_passes(k.bytes, n) : 0;
        j->nstages = 1 + j->passes;
    }
    j->t_submit = clock_s();
    std::lock_guard<std::mutex> lk(q->mu);
    if (j->bytes > q->budget) {
        delete j;
        return fail(MP_ERR_BUDGET, "mp_queue_submit: request needs more device memory than the budget");
    }
    if (q->stop) {
        delete j;
        return fail(MP_ERR_INVALID_ARG, "mp_queue_submit: queue is shutting down");
    }
    j->ticket = q->next_ticket++;
    q->jobs[j->ticket] = j;
    q->waiting.push_back(j);
    q->stats.submitted++;
    *ticket = j->ticket;
    q->cv_work.notify_one();
    return MP_OK;
}

mp_status mp_queue_wait(mp_queue* q, uint64_t ticket, int64_t timeout_ns, mp_result* res)
{
    if (!q || !res) return fail(MP_ERR_INVALID_ARG, "mp_queue_wait: NULL argument");
    std::unique_lock<std::mutex> lk(q->mu);
    auto it = q->jobs.find(ticket);
    if (it == q->jobs.end()) return fail(MP_ERR_INVALID_ARG, "mp_queue_wait: unknown ticket");
    Job* j = it->second;
    auto done = [&] { return j->state == JOB_DONE; };
    if (!done()) {
        if (timeout_ns == 0) return MP_ERR_NOT_READY;
        if (timeout_ns < 0)
            q->cv_done.wait(lk, done);
        else if (!q->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), done))
            return fail(MP_ERR_TIMEOUT, "mp_queue_wait: timed out");
    }
    res->status = j->status;
    res->op = j->req.op;
    res->n = j->n;
    res->t_submit = j->t_submit;
    res->t_admit = j->t_admit;
    res->t_done = j->t_done;
    q->jobs.erase(it);
    delete j;
    return MP_OK;
}

mp_status mp_queue_get_stats(mp_queue* q, mp_queue_stats* s)
{
    if (!q || !s) return fail(MP_ERR_INVALID_ARG, "mp_queue_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(q->mu);
    *s = q->stats;
    s->waiting = q->waiting.size();
    s->active = q->active.size();
    s->bytes_in_use = q->used;
    return MP_OK;
}

mp_status mp_queue_destroy(mp_queue* q)
{
    if (!q) return MP_OK;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        q->stop = true;
        q->cv_work.notify_all();
    }
    if (q->worker.joinable()) q->worker.join();
    cudaStreamSynchronize(q->s_compute);
    cudaStreamSynchronize(q->s_copy);
    for (auto& kv : q->jobs) delete kv.second;
    for (int i = 0; i < 2; ++i) {
        if (q->h_table[i]) cudaFreeHost(q->h_table[i]);
        if (q->d_table[i]) cudaFree(q->d_table[i]);
        if (q->step_ev[i]) cudaEventDestroy(q->step_ev[i]);
    }
    cudaStreamDestroy(q->s_compute);
    cudaStreamDestroy(q->s_copy);
    cudaMemPoolDestroy(q->pool);
    delete q;
    return MP_OK;
}

mp_status mp_generate(mp_dtype dtype, void* keys, uint32_t* vals, int64_t n, uint64_t seed,
                      uint64_t stream_id, int sorted, uint32_t val_base, mp_stream_t stream)
{
    KeyKind k;
    if (!key_kind(dtype, &k) || (dtype != MP_U32 && dtype != MP_U64))
        return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_generate: MP_U32 or MP_U64 keys only");
    if (n < 0 || (n > 0 && !keys)) return fail(MP_ERR_INVALID_ARG, "mp_generate: bad arguments");
    cudaError_t e = generate(k.bytes, keys, vals, n, seed, stream_id, sorted != 0, val_base, (cudaStream_t)stream);
    return e == cudaSuccess ? MP_OK : cuda_fail(e, "mp_generate");
}

}  // extern "C"
