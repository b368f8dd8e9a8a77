/*
 * mp_oracle.c -- plain, slow, single-threaded CPU oracle for Merge Path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * bench's CPU-baseline leg may load this library.  The product (the CUDA
 * library in paper_1406_2628_gb300/) never calls it and shares no code,
 * header, table or helper with it.
 *
 * What it computes (Green, Odeh, Birk, "Merge Path - A Visually Intuitive
 * Approach to Parallel Merging"):
 *
 *   merge   Sec. I (the sequential merge: repeatedly take the smaller head)
 *           and Sec. II.A (path construction: move right, i.e. take B, iff
 *           A[i] > B[j], else move down, i.e. take A).  Ties therefore take
 *           A first, which makes the merge stable.
 *   split   Alg. 2 (Diagonal Intersection) in the paper's order and
 *           notation, with the garbled lower bound replaced by
 *           a_bottom = max(0, diag - |B|) and with out-of-range probes read
 *           as sentinels (A[-1] = B[-1] = -inf, A[|A|] = B[|B|] = +inf).
 *   sort    Sec. I / Sec. III: bottom-up merge sort, rounds of widths
 *           1, 2, 4, ... each merging adjacent run pairs with the merge
 *           above (left run plays A).  Stable.
 *   batched Cor. 6 applied to many independent (A_s, B_s) pairs: each
 *           segment is merged on its own and written at its offset
 *           a_off[s] + b_off[s] of the concatenated output.
 *   set_op  merge-based set operations (Sec. I names joins of database
 *           query results and merges of adjacency lists as uses of
 *           merging).  The same two-pointer walk as the merge, where equal
 *           heads form a matched pair.  Multiset semantics: a key present
 *           m times in A and n times in B appears
 *             union         max(m, n) times: A's m copies, then B's last
 *                           max(n - m, 0) copies;
 *             intersection  min(m, n) times: A's first min(m, n) copies;
 *             difference    max(m - n, 0) times: A's last m - n copies;
 *             symmetric     |m - n| times: A's last m - n copies, or B's
 *                           last n - m copies.
 *           On duplicate-free inputs these are the ordinary set operations.
 *
 * Key order.  Integers use their natural order (including the 128-bit
 * multi-word keys, stored as two 64-bit words, low word first).  float32
 * uses the IEEE-754 numeric order with -0.0 ordered before +0.0 (NaN is not
 * a valid input).
 * Values (payloads) are uint32 and move with their keys.
 *
 * Pins: every function here is checked by tests/test_oracle_*.py against a
 * brute force (tagged concatenation + a library stable sort), closed forms
 * from the paper (all of A greater than all of B, Sec. I) and invariants
 * (Lemma 8 / Cor. 12 monotone split points, Alg. 2's acceptance test,
 * Thm 14's step bound).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ---- Def. 1: the Merge Matrix entry M[i,j] = 1 iff A[i] > B[j]. -------- */

static int gt_i32(int32_t x, int32_t y) { return x > y; }
static int gt_u32(uint32_t x, uint32_t y) { return x > y; }
static int gt_u64(uint64_t x, uint64_t y) { return x > y; }
static int gt_i64(int64_t x, int64_t y) { return x > y; }
/* Multi-word keys: 128-bit integers (two 64-bit words, low word first). */
static int gt_u128(unsigned __int128 x, unsigned __int128 y) { return x > y; }
static int gt_i128(__int128 x, __int128 y) { return x > y; }
/* float32: numeric order, and among equal zeros +0.0 is greater than -0.0. */
static int gt_f32(float x, float y)
{
    if (x > y) return 1;
    if (x == y && x == 0.0f) return !signbit(x) && signbit(y);
    return 0;
}

/*
 * ORACLE_TYPE(suffix, T) emits, for key type T:
 *   oracle_merge_<suffix>     two-pointer merge (Sec. I, Sec. II.A)
 *   oracle_split_<suffix>     Alg. 2 diagonal intersection
 *   oracle_sort_<suffix>      bottom-up merge sort (Sec. I)
 *   oracle_merge_batched_<suffix>  one merge per segment (Cor. 6)
 *   oracle_set_op_<suffix>    union / intersection / difference / symmetric
 */
#define ORACLE_TYPE(SFX, T)                                                          \
                                                                                     \
/* Merge A (na keys) and B (nb keys) into out (na+nb keys).  av/bv/outv are the  */ \
/* uint32 payloads; pass NULL for all three to merge keys only.                  */ \
void oracle_merge_##SFX(const T* a, const uint32_t* av, int64_t na,                  \
                        const T* b, const uint32_t* bv, int64_t nb,                  \
                        T* out, uint32_t* outv)                                      \
{                                                                                    \
    int64_t i = 0, j = 0, k = 0;                                                     \
    while (i < na || j < nb) {                                                       \
        /* Sec. II.A: right (take B) iff A[i] > B[j]; once the bottom or right */  \
        /* edge is reached, only one direction remains.                       */  \
        int take_b;                                                                  \
        if (i == na) take_b = 1;                                                     \
        else if (j == nb) take_b = 0;                                                \
        else take_b = gt_##SFX(a[i], b[j]);                                          \
        if (take_b) {                                                                \
            out[k] = b[j];                                                           \
            if (outv) outv[k] = bv[j];                                               \
            j++;                                                                     \
        } else {                                                                     \
            out[k] = a[i];                                                           \
            if (outv) outv[k] = av[i];                                               \
            i++;                                                                     \
        }                                                                            \
        k++;                                                                         \
    }                                                                                \
}                                                                                    \
                                                                                     \
/* Alg. 2: where the Merge Path crosses cross diagonal `diag` (0-based: diag is  */ \
/* the number of outputs before the crossing point).  Returns a_start; the      */ \
/* caller gets b_start = diag - a_start.  *steps (if not NULL) receives the      */ \
/* number of loop iterations, each of which compares one element of A with one  */ \
/* element of B on each side (Thm 14 counts these).  Returns -1 if diag is out  */ \
/* of [0, na+nb], -2 if the search window empties (inputs not sorted).          */ \
int64_t oracle_split_##SFX(const T* a, int64_t na, const T* b, int64_t nb,          \
                           int64_t diag, int64_t* steps)                             \
{                                                                                    \
    if (diag < 0 || diag > na + nb) return -1;                                       \
    int64_t a_top = diag > na ? na : diag;                                           \
    int64_t b_top = diag > na ? diag - na : 0;                                       \
    /* The printed lower bound (a_bottom <- b_top) is garbled; the lowest point  */ \
    /* of the diagonal inside the grid has a = max(0, diag - |B|).               */ \
    int64_t a_bottom = diag - nb > 0 ? diag - nb : 0;                                \
    int64_t n_steps = 0;                                                             \
    for (;;) {                                                                       \
        /* Invariant: the crossing lies in [a_bottom, a_top].  It cannot empty */   \
        /* for sorted inputs; report a failed search instead of looping.      */   \
        if (a_top < a_bottom) return -2;                                             \
        int64_t offset = (a_top - a_bottom) / 2;                                     \
        int64_t a_i = a_top - offset;                                                \
        int64_t b_i = b_top + offset;                                                \
        n_steps++;                                                                   \
        /* A[a_i] > B[b_i - 1], with A[na] = +inf and B[-1] = -inf. */               \
        int upper_ok = (a_i >= na) || (b_i <= 0) || gt_##SFX(a[a_i], b[b_i - 1]);   \
        if (upper_ok) {                                                              \
            /* A[a_i - 1] <= B[b_i], with A[-1] = -inf and B[nb] = +inf. */          \
            int lower_ok = (a_i <= 0) || (b_i >= nb) || !gt_##SFX(a[a_i - 1], b[b_i]); \
            if (lower_ok) {                                                          \
                if (steps) *steps = n_steps;                                         \
                return a_i;                                                          \
            }                                                                        \
            a_top = a_i - 1;                                                         \
            b_top = b_i + 1;                                                         \
        } else {                                                                     \
            a_bottom = a_i + 1;                                                      \
        }                                                                            \
    }                                                                                \
}                                                                                    \
                                                                                     \
/* Bottom-up merge sort of keys[0..n) (and vals, if not NULL), in place.          */ \
/* Round r merges the adjacent sorted runs [i, i+w) and [i+w, i+2w), w = 2^r,     */ \
/* with the merge above, left run as A.  Returns 0, or -1 if out of memory.       */ \
int oracle_sort_##SFX(T* keys, uint32_t* vals, int64_t n)                            \
{                                                                                    \
    if (n <= 1) return 0;                                                            \
    T* tk = (T*)malloc((size_t)n * sizeof(T));                                       \
    uint32_t* tv = vals ? (uint32_t*)malloc((size_t)n * sizeof(uint32_t)) : NULL;    \
    if (!tk || (vals && !tv)) { free(tk); free(tv); return -1; }                     \
    T* src = keys; T* dst = tk;                                                      \
    uint32_t* srcv = vals; uint32_t* dstv = tv;                                      \
    for (int64_t w = 1; w < n; w *= 2) {                                             \
        for (int64_t lo = 0; lo < n; lo += 2 * w) {                                  \
            int64_t mid = lo + w < n ? lo + w : n;                                   \
            int64_t hi = lo + 2 * w < n ? lo + 2 * w : n;                            \
            oracle_merge_##SFX(src + lo, srcv ? srcv + lo : NULL, mid - lo,          \
                               src + mid, srcv ? srcv + mid : NULL, hi - mid,        \
                               dst + lo, dstv ? dstv + lo : NULL);                   \
        }                                                                            \
        T* t = src; src = dst; dst = t;                                              \
        uint32_t* u = srcv; srcv = dstv; dstv = u;                                   \
    }                                                                                \
    if (src != keys) {                                                               \
        memcpy(keys, src, (size_t)n * sizeof(T));                                    \
        if (vals) memcpy(vals, srcv, (size_t)n * sizeof(uint32_t));                  \
    }                                                                                \
    free(tk); free(tv);                                                              \
    return 0;                                                                        \
}                                                                                    \
                                                                                     \
/* nseg independent merges.  Segment s merges a[a_off[s], a_off[s+1]) with       */ \
/* b[b_off[s], b_off[s+1]) into out[a_off[s] + b_off[s], ...).  Offsets are host  */ \
/* arrays of nseg+1 entries.                                                      */ \
void oracle_merge_batched_##SFX(const T* a, const uint32_t* av, const int64_t* a_off, \
                                const T* b, const uint32_t* bv, const int64_t* b_off, \
                                int64_t nseg, T* out, uint32_t* outv)                \
{                                                                                    \
    for (int64_t s = 0; s < nseg; s++) {                                             \
        int64_t c = a_off[s] + b_off[s];                                             \
        oracle_merge_##SFX(a + a_off[s], av ? av + a_off[s] : NULL,                  \
                           a_off[s + 1] - a_off[s],                                  \
                           b + b_off[s], bv ? bv + b_off[s] : NULL,                  \
                           b_off[s + 1] - b_off[s],                                  \
                           out + c, outv ? outv + c : NULL);                         \
    }                                                                                \
}                                                                                    \
                                                                                     \
/* Set operation op (0 union, 1 intersection, 2 difference A - B, 3 symmetric   */ \
/* difference) of sorted A and B.  Emitted keys go to out (values to outv if    */ \
/* not NULL: an emitted element keeps its own side's value).  Returns the      */ \
/* number of outputs.  out must hold na + nb keys.                              */ \
int64_t oracle_set_op_##SFX(int op, const T* a, const uint32_t* av, int64_t na,    \
                            const T* b, const uint32_t* bv, int64_t nb,            \
                            T* out, uint32_t* outv)                                \
{                                                                                    \
    const int keep_a_alone = (op == 0 || op == 2 || op == 3);                        \
    const int keep_b_alone = (op == 0 || op == 3);                                   \
    const int keep_pair = (op == 0 || op == 1);                                      \
    int64_t i = 0, j = 0, k = 0;                                                     \
    while (i < na && j < nb) {                                                       \
        if (gt_##SFX(a[i], b[j])) {          /* B's head is smaller */             \
            if (keep_b_alone) {                                                      \
                out[k] = b[j];                                                       \
                if (outv) outv[k] = bv[j];                                           \
                k++;                                                                 \
            }                                                                        \
            j++;                                                                     \
        } else if (gt_##SFX(b[j], a[i])) {   /* A's head is smaller */             \
            if (keep_a_alone) {                                                      \
                out[k] = a[i];                                                       \
                if (outv) outv[k] = av[i];                                           \
                k++;                                                                 \
            }                                                                        \
            i++;                                                                     \
        } else {                             /* equal heads: a matched pair */     \
            if (keep_pair) {                                                         \
                out[k] = a[i];                                                       \
                if (outv) outv[k] = av[i];                                           \
                k++;                                                                 \
            }                                                                        \
            i++;                                                                     \
            j++;                                                                     \
        }                                                                            \
    }                                                                                \
    for (; i < na; i++)                                                              \
        if (keep_a_alone) {                                                          \
            out[k] = a[i];                                                           \
            if (outv) outv[k] = av[i];                                               \
            k++;                                                                     \
        }                                                                            \
    for (; j < nb; j++)                                                              \
        if (keep_b_alone) {                                                          \
            out[k] = b[j];                                                           \
            if (outv) outv[k] = bv[j];                                               \
            k++;                                                                     \
        }                                                                            \
    return k;                                                                        \
}

ORACLE_TYPE(i32, int32_t)
ORACLE_TYPE(u32, uint32_t)
ORACLE_TYPE(f32, float)
ORACLE_TYPE(u64, uint64_t)
ORACLE_TYPE(i64, int64_t)
ORACLE_TYPE(u128, unsigned __int128)
ORACLE_TYPE(i128, __int128)
