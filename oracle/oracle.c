/*
 * oracle.c — plain CPU oracle for exact k-smallest selection.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg.  Shares nothing with the CUDA library.
 *
 * Every function sorts the whole input once with qsort and a comparator that
 * states the order directly (see oracle.h); there is no sampling, no
 * partitioning and no recursion here, so the result can be checked against
 * the definition by eye:
 *   Section 2  : objects are made unique as pairs (value, position);
 *   Section 4  : the answer is the set of pairs of rank <= k and the pair of
 *                rank k;
 *   Appendix A : for sorted sequences, the answer is also expressed as the
 *                number of selected objects per sequence (split positions).
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t key; /* raw key bits, zero-extended */
    uint64_t idx; /* position: the tie-break of Section 2 */
} orc_pair;

int oracle_key_bytes(int dtype)
{
    switch (dtype) {
    case ORC_U32: return 4;
    case ORC_I32: return 4;
    case ORC_F32: return 4;
    case ORC_BF16: return 2;
    case ORC_U64: return 8;
    default: return 0;
    }
}

static int cmp_unsigned(uint64_t a, uint64_t b)
{
    return (a < b) ? -1 : (a > b) ? 1 : 0;
}

static int cmp_signed32(uint64_t a, uint64_t b)
{
    int32_t x = (int32_t)(uint32_t)a;
    int32_t y = (int32_t)(uint32_t)b;
    return (x < y) ? -1 : (x > y) ? 1 : 0;
}

/* IEEE 754-2008 clause 5.10 totalOrder for a sign-magnitude pattern of
 * `bits` bits: sign bit first, then the magnitude field. */
static int cmp_total_order(uint64_t a, uint64_t b, int bits)
{
    uint64_t sign_bit = (uint64_t)1 << (bits - 1);
    uint64_t mag_mask = sign_bit - 1;
    int neg_a = (a & sign_bit) != 0;
    int neg_b = (b & sign_bit) != 0;
    uint64_t mag_a = a & mag_mask;
    uint64_t mag_b = b & mag_mask;
    if (neg_a != neg_b)
        return neg_a ? -1 : 1;          /* every negative precedes every positive */
    if (!neg_a)
        return cmp_unsigned(mag_a, mag_b); /* positives: larger magnitude is larger */
    return cmp_unsigned(mag_b, mag_a);     /* negatives: larger magnitude is smaller */
}

int oracle_key_cmp(int dtype, uint64_t a, uint64_t b)
{
    switch (dtype) {
    case ORC_U32: return cmp_unsigned(a & 0xffffffffu, b & 0xffffffffu);
    case ORC_U64: return cmp_unsigned(a, b);
    case ORC_I32: return cmp_signed32(a, b);
    case ORC_F32: return cmp_total_order(a & 0xffffffffu, b & 0xffffffffu, 32);
    case ORC_BF16: return cmp_total_order(a & 0xffffu, b & 0xffffu, 16);
    default: return 0;
    }
}

/* qsort has no context argument, so one comparator per dtype. */
#define ORC_PAIR_CMP(name, dt)                                           \
    static int name(const void *pa, const void *pb)                     \
    {                                                                    \
        const orc_pair *x = (const orc_pair *)pa;                        \
        const orc_pair *y = (const orc_pair *)pb;                        \
        int c = oracle_key_cmp(dt, x->key, y->key);                      \
        if (c != 0)                                                      \
            return c;                                                    \
        return cmp_unsigned(x->idx, y->idx); /* Section 2 tie-break */   \
    }
ORC_PAIR_CMP(pair_cmp_u32, ORC_U32)
ORC_PAIR_CMP(pair_cmp_i32, ORC_I32)
ORC_PAIR_CMP(pair_cmp_f32, ORC_F32)
ORC_PAIR_CMP(pair_cmp_bf16, ORC_BF16)
ORC_PAIR_CMP(pair_cmp_u64, ORC_U64)

typedef int (*orc_cmp_fn)(const void *, const void *);

static orc_cmp_fn pair_cmp_for(int dtype)
{
    switch (dtype) {
    case ORC_U32: return pair_cmp_u32;
    case ORC_I32: return pair_cmp_i32;
    case ORC_F32: return pair_cmp_f32;
    case ORC_BF16: return pair_cmp_bf16;
    case ORC_U64: return pair_cmp_u64;
    default: return 0;
    }
}

static uint64_t load_key(const void *keys, uint64_t i, int dtype)
{
    switch (oracle_key_bytes(dtype)) {
    case 2: return ((const uint16_t *)keys)[i];
    case 4: return ((const uint32_t *)keys)[i];
    case 8: return ((const uint64_t *)keys)[i];
    default: return 0;
    }
}

/* Builds and sorts the n pairs; caller frees the result. */
static orc_pair *sorted_pairs(const void *keys, uint64_t n, int dtype)
{
    orc_cmp_fn cmp = pair_cmp_for(dtype);
    orc_pair *v;
    uint64_t i;
    if (!cmp || n == 0)
        return 0;
    v = (orc_pair *)malloc(n * sizeof(orc_pair));
    if (!v)
        return 0;
    for (i = 0; i < n; ++i) {
        v[i].key = load_key(keys, i, dtype);
        v[i].idx = i;
    }
    qsort(v, (size_t)n, sizeof(orc_pair), cmp);
    return v;
}

int oracle_sort_order(const void *keys, uint64_t n, int dtype, uint32_t *perm)
{
    orc_pair *v;
    uint64_t i;
    if (!keys || !perm || n == 0 || n > 0xffffffffull)
        return -1;
    v = sorted_pairs(keys, n, dtype);
    if (!v)
        return -1;
    for (i = 0; i < n; ++i)
        perm[i] = (uint32_t)v[i].idx;
    free(v);
    return 0;
}

int oracle_select(const void *keys, uint64_t n, int dtype, uint64_t k,
                  uint32_t *sel_idx, uint32_t *kth_idx)
{
    orc_pair *v;
    uint64_t i;
    if (!keys || !sel_idx || !kth_idx || k < 1 || k > n || n > 0xffffffffull)
        return -1;
    v = sorted_pairs(keys, n, dtype);
    if (!v)
        return -1;
    for (i = 0; i < k; ++i)             /* ranks 1..k */
        sel_idx[i] = (uint32_t)v[i].idx;
    *kth_idx = (uint32_t)v[k - 1].idx;  /* the object of rank k */
    free(v);
    return 0;
}

/* The run r with run_off[r] <= g < run_off[r+1] (bisection over the
 * non-decreasing offsets; empty runs are skipped because their interval is
 * empty). */
static uint32_t run_holding(const uint64_t *run_off, uint32_t p, uint64_t g)
{
    uint32_t lo = 0, hi = p; /* invariant: run_off[lo] <= g < run_off[hi] */
    while (hi - lo > 1) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (run_off[mid] <= g)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

int oracle_select_runs(const uint64_t *keys, const uint64_t *run_off, uint32_t p,
                       uint64_t k, uint64_t *split, uint32_t *kth_run,
                       uint64_t *kth_pos)
{
    uint64_t total, i;
    uint32_t r;
    orc_pair *v;
    if (!keys || !run_off || !split || !kth_run || !kth_pos || p == 0)
        return -1;
    if (run_off[0] != 0)
        return -1;
    for (r = 0; r < p; ++r)
        if (run_off[r + 1] < run_off[r])
            return -1;
    total = run_off[p];
    if (k < 1 || k > total || total > 0xffffffffull)
        return -1;
    /* Concatenated index orders pairs by (run, position) among equal keys. */
    v = sorted_pairs(keys, total, ORC_U64);
    if (!v)
        return -1;
    for (r = 0; r < p; ++r)
        split[r] = 0;
    for (i = 0; i < k; ++i) {
        uint64_t g = v[i].idx;
        r = run_holding(run_off, p, g);
        split[r] += 1;
        if (i == k - 1) {
            *kth_run = r;
            *kth_pos = g - run_off[r];
        }
    }
    free(v);
    return 0;
}

int oracle_runs_delete_min(const uint64_t *keys, const uint64_t *run_off, uint32_t p,
                           uint64_t *cursor, uint64_t k, uint32_t *kth_run,
                           uint64_t *kth_pos)
{
    uint64_t remain = 0, i, j, len;
    uint32_t r;
    orc_pair *v;
    orc_cmp_fn cmp = pair_cmp_for(ORC_U64);
    if (!keys || !run_off || !cursor || !kth_run || !kth_pos || p == 0)
        return -1;
    if (run_off[0] != 0 || run_off[p] > 0xffffffffull)
        return -1;
    for (r = 0; r < p; ++r) {
        if (run_off[r + 1] < run_off[r])
            return -1;
        len = run_off[r + 1] - run_off[r];
        if (cursor[r] > len)
            return -1;
        remain += len - cursor[r];
    }
    if (k < 1 || k > remain)
        return -1;
    /* The queue's content: every pair at or after its run's cursor (room
     * for all run_off[p] pairs, j of them filled). */
    v = (orc_pair *)malloc((run_off[p] ? run_off[p] : 1) * sizeof(orc_pair));
    if (!v)
        return -1;
    j = 0;
    for (r = 0; r < p; ++r)
        for (i = run_off[r] + cursor[r]; i < run_off[r + 1]; ++i) {
            v[j].key = keys[i];
            v[j].idx = i;
            ++j;
        }
    qsort(v, (size_t)j, sizeof(orc_pair), cmp);
    /* deleteMin*: the k smallest leave the queue, each run's cursor moving
     * past those of its own. */
    for (i = 0; i < k; ++i) {
        r = run_holding(run_off, p, v[i].idx);
        cursor[r] += 1;
        if (i == k - 1) {
            *kth_run = r;
            *kth_pos = v[i].idx - run_off[r];
        }
    }
    free(v);
    return 0;
}

int oracle_select_batched(const void *keys, const uint64_t *row_off,
                          const uint32_t *row_k, uint32_t rows, int dtype,
                          const uint64_t *out_off, uint32_t *sel_idx,
                          uint32_t *kth_idx)
{
    uint32_t i;
    int w = oracle_key_bytes(dtype);
    if (!keys || !row_off || !row_k || !out_off || !sel_idx || !kth_idx || w == 0)
        return -1;
    for (i = 0; i < rows; ++i) {
        uint64_t n = row_off[i + 1] - row_off[i];
        const char *row = (const char *)keys + row_off[i] * (uint64_t)w;
        if (row_off[i + 1] < row_off[i])
            return -1;
        if (oracle_select(row, n, dtype, row_k[i], sel_idx + out_off[i],
                          kth_idx + i) != 0)
            return -1;
    }
    return 0;
}
