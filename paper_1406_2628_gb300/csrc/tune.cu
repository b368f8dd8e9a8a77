// tune.cu -- tile-shape autotuner and its cache.
//
// The best tile shape (threads per CTA NT, items per thread VT) of the merge
// kernels depends on the key width, on whether values move, and on the
// problem size (the partition cost grows with the number of tiles, the merge
// kernel's efficiency with the tile count per SM).  mp_autotune_merge times
// every compiled shape on the caller's own data (partition + merge, CUDA
// events, the fastest of `reps` runs) and records the winner for the size
// class floor(log2(na+nb)); automatic plans consult this table first.  The
// table can be saved to and loaded from a text file (one entry per line:
// "<device name>|<op>|<key bytes>|<values>|<size class> <NT> <VT> <staging>");
// if the environment variable MP_TUNE_CACHE names a file it is loaded on
// first use.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mp_internal.h"

namespace mp {

static std::mutex g_tune_mu;
static std::map<std::string, Shape> g_tune;
static bool g_tune_env_loaded = false;

static std::string device_name()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return "unknown";
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    std::string n(prop.name);
    for (char& c : n)
        if (c == '|' || c == ' ') c = '_';
    return n;
}

static int size_class(int64_t total)
{
    int c = 0;
    while (c < 62 && ((int64_t)1 << (c + 1)) <= total) ++c;
    return c;
}

static std::string tune_key(const char* op, int key_bytes, bool vals, int64_t total)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s|%s|%d|%d|%d", device_name().c_str(), op, key_bytes, vals ? 1 : 0,
             size_class(total));
    return buf;
}

static int load_file_locked(const char* path)
{
    FILE* f = fopen(path, "r");
    if (!f) return -1;
    char key[256];
    int nt, vt, st, n = 0;
    while (fscanf(f, "%255s %d %d %d", key, &nt, &vt, &st) == 4) {
        Shape s{nt, vt, st};
        g_tune[key] = s;
        ++n;
    }
    fclose(f);
    return n;
}

static void maybe_load_env_locked()
{
    if (g_tune_env_loaded) return;
    g_tune_env_loaded = true;
    const char* p = getenv("MP_TUNE_CACHE");
    if (p && *p) load_file_locked(p);
}

bool tuned_shape(const char* op, int key_bytes, bool vals, int64_t total, Shape* s)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    maybe_load_env_locked();
    auto it = g_tune.find(tune_key(op, key_bytes, vals, total));
    if (it == g_tune.end()) return false;
    *s = it->second;
    return true;
}

void record_shape(const char* op, int key_bytes, bool vals, int64_t total, const Shape& s)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(op, key_bytes, vals, total)] = s;
}

}  // namespace mp

using namespace mp;

extern "C" {

mp_status mp_autotune_merge(mp_dtype dtype, const void* a_keys, const uint32_t* a_vals, int64_t na,
                            const void* b_keys, const uint32_t* b_vals, int64_t nb, void* out_keys,
                            uint32_t* out_vals, int reps, mp_plan* best, mp_stream_t stream)
{
    KeyKind k;
    if (!key_kind(dtype, &k)) return fail(MP_ERR_UNSUPPORTED_DTYPE, "mp_autotune_merge: unknown dtype");
    const bool vals = a_vals || b_vals || out_vals;
    mp_status st = check_merge_args_ext(k, a_keys, a_vals, na, b_keys, b_vals, nb, out_keys, out_vals,
                                        vals, "mp_autotune_merge");
    if (st != MP_OK) return st;
    if (na + nb == 0) return fail(MP_ERR_INVALID_ARG, "mp_autotune_merge: empty problem");
    if (reps < 1) reps = 1;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(MP_ERR_CUDA, "mp_autotune_merge: events");
    Shape best_s{0, 0, 0};
    float best_ms = 1e30f;
    std::vector<Shape> cands = merge_shapes();
    for (const Shape& c : stream_shapes()) cands.push_back(c);
    for (const Shape& cand : cands) {
        const bool ok = cand.staging == MP_STAGE_STREAM ? stream_shape_supported(cand)
                                                        : merge_shape_supported(k.bytes, vals, cand);
        if (!ok) continue;
        mp_plan p{cand.nt, cand.vt, cand.staging, 0};
        // Warm-up (also sets kernel attributes), then the fastest of reps.
        st = mp_merge_plan(dtype, a_keys, a_vals, na, b_keys, b_vals, nb, out_keys, out_vals, &p, stream);
        if (st != MP_OK) break;
        float cand_ms = 1e30f;
        for (int r = 0; r < reps && st == MP_OK; ++r) {
            cudaEventRecord(e0, s);
            st = mp_merge_plan(dtype, a_keys, a_vals, na, b_keys, b_vals, nb, out_keys, out_vals, &p, stream);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = fail(MP_ERR_CUDA, "mp_autotune_merge: timing"); break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < cand_ms) cand_ms = ms;
        }
        if (st != MP_OK) break;
        if (cand_ms < best_ms) {
            best_ms = cand_ms;
            best_s = cand;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MP_OK) return st;
    record_shape("merge", k.bytes, vals, na + nb, best_s);
    if (best) *best = mp_plan{best_s.nt, best_s.vt, best_s.staging, 0};
    return MP_OK;
}

mp_status mp_tune_save(const char* path)
{
    if (!path) return fail(MP_ERR_INVALID_ARG, "mp_tune_save: NULL path");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    FILE* f = fopen(path, "w");
    if (!f) return fail(MP_ERR_INVALID_ARG, std::string("mp_tune_save: cannot write ") + path);
    for (auto& kv : g_tune) fprintf(f, "%s %d %d %d\n", kv.first.c_str(), kv.second.nt, kv.second.vt, kv.second.staging);
    fclose(f);
    return MP_OK;
}

mp_status mp_tune_load(const char* path)
{
    if (!path) return fail(MP_ERR_INVALID_ARG, "mp_tune_load: NULL path");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (load_file_locked(path) < 0) return fail(MP_ERR_INVALID_ARG, std::string("mp_tune_load: cannot read ") + path);
    return MP_OK;
}

void mp_tune_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

}  // extern "C"
