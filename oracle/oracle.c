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

#include <math.h>
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

/* The largest first: values descending, equal values by ascending index. */
#define ORC_PAIR_CMP_DESC(name, dt)                                      \
    static int name(const void *pa, const void *pb)                     \
    {                                                                    \
        const orc_pair *x = (const orc_pair *)pa;                        \
        const orc_pair *y = (const orc_pair *)pb;                        \
        int c = oracle_key_cmp(dt, y->key, x->key);                      \
        if (c != 0)                                                      \
            return c;                                                    \
        return cmp_unsigned(x->idx, y->idx);                             \
    }
ORC_PAIR_CMP_DESC(pair_cmp_desc_u32, ORC_U32)
ORC_PAIR_CMP_DESC(pair_cmp_desc_i32, ORC_I32)
ORC_PAIR_CMP_DESC(pair_cmp_desc_f32, ORC_F32)
ORC_PAIR_CMP_DESC(pair_cmp_desc_bf16, ORC_BF16)
ORC_PAIR_CMP_DESC(pair_cmp_desc_u64, ORC_U64)

typedef int (*orc_cmp_fn)(const void *, const void *);

static orc_cmp_fn pair_cmp_desc_for(int dtype)
{
    switch (dtype) {
    case ORC_U32: return pair_cmp_desc_u32;
    case ORC_I32: return pair_cmp_desc_i32;
    case ORC_F32: return pair_cmp_desc_f32;
    case ORC_BF16: return pair_cmp_desc_bf16;
    case ORC_U64: return pair_cmp_desc_u64;
    default: return 0;
    }
}

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

int oracle_select_largest(const void *keys, uint64_t n, int dtype, uint64_t k,
                          uint32_t *sel_idx, uint32_t *kth_idx)
{
    orc_cmp_fn cmp = pair_cmp_desc_for(dtype);
    orc_pair *v;
    uint64_t i;
    if (!keys || !sel_idx || !kth_idx || !cmp || k < 1 || k > n || n > 0xffffffffull)
        return -1;
    v = (orc_pair *)malloc(n * sizeof(orc_pair));
    if (!v)
        return -1;
    for (i = 0; i < n; ++i) {
        v[i].key = load_key(keys, i, dtype);
        v[i].idx = i;
    }
    qsort(v, (size_t)n, sizeof(orc_pair), cmp);
    for (i = 0; i < k; ++i)
        sel_idx[i] = (uint32_t)v[i].idx;
    *kth_idx = sel_idx[k - 1]; /* the pair of rank k in this order */
    free(v);
    return 0;
}

/* The rank of one pair without sorting: the pairs (keys[i], i) that come
 * before (keys[pos], pos) in the order of oracle_select (ascending values) or
 * of oracle_select_largest (descending values), equal values by position.
 * One comparison per element, straight from the definition of the order. */
int oracle_pairs_before(const void *keys, uint64_t n, int dtype, uint64_t pos,
                        int descending, uint64_t *count)
{
    uint64_t i, c = 0, v;
    if (!keys || !count || !oracle_key_bytes(dtype) || pos >= n)
        return -1;
    v = load_key(keys, pos, dtype);
    for (i = 0; i < n; ++i) {
        int d = oracle_key_cmp(dtype, load_key(keys, i, dtype), v);
        if (descending)
            d = -d;
        if (d < 0 || (d == 0 && i < pos))
            ++c;
    }
    *count = c;
    return 0;
}

/* Whether a claimed answer is exactly the k smallest pairs (or, with
 * descending = 1, the k largest), checked from the definition without a sort:
 *   (1) the claimed rank-k pair (keys[kth], kth) has k - 1 pairs before it;
 *   (2) the k claimed positions are distinct (a bitmap of n bits);
 *   (3) no claimed pair comes after the rank-k pair;
 *   (4) every claimed output key (out_keys, may be NULL) has the bits of the
 *       input key at its position, and the claimed rank-k key (kth_key, may
 *       be NULL) those of keys[kth].
 * (1)-(3) leave exactly one set: k distinct pairs, none after the pair that
 * has exactly k - 1 before it, are the k pairs up to it.  Returns 0 when all
 * hold, the number of the first failed condition otherwise, -1 on bad
 * arguments or allocation failure. */
int oracle_check_selection(const void *keys, uint64_t n, int dtype, uint64_t k,
                           int descending, const uint32_t *sel_idx, const void *out_keys,
                           uint64_t kth, const void *kth_key)
{
    uint64_t before = 0, i, kv;
    uint8_t *seen;
    if (!keys || !sel_idx || !oracle_key_bytes(dtype) || k < 1 || k > n || kth >= n)
        return -1;
    if (oracle_pairs_before(keys, n, dtype, kth, descending, &before) != 0)
        return -1;
    if (before != k - 1)
        return 1;
    seen = (uint8_t *)calloc((size_t)(n / 8 + 1), 1);
    if (!seen)
        return -1;
    kv = load_key(keys, kth, dtype);
    for (i = 0; i < k; ++i) {
        uint64_t x = sel_idx[i];
        int d;
        if (x >= n || (seen[x / 8] >> (x % 8)) & 1u) {
            free(seen);
            return 2;
        }
        seen[x / 8] |= (uint8_t)(1u << (x % 8));
        d = oracle_key_cmp(dtype, load_key(keys, x, dtype), kv);
        if (descending)
            d = -d;
        if (d > 0 || (d == 0 && x > kth)) {
            free(seen);
            return 3;
        }
        if (out_keys && load_key(out_keys, i, dtype) != load_key(keys, x, dtype)) {
            free(seen);
            return 4;
        }
    }
    free(seen);
    if (kth_key && load_key(kth_key, 0, dtype) != kv)
        return 4;
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

/* ------------------------------------------------------------------------
 * Top-k most frequent objects (Section 7).
 * ------------------------------------------------------------------------ */

/* Philox4x32-10 from its published definition (Salmon, Moraes, Dror, Shaw,
 * SC'11): ten rounds of two 32x32->64 multiplications whose halves are
 * permuted and xor-ed with the counter words and the round key; the key
 * grows by the Weyl constants between rounds. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    int round;
    for (round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

uint64_t oracle_sample_threshold(double rho)
{
    if (!(rho > 0.0))
        return 0;
    if (rho >= 1.0)
        return (uint64_t)1 << 32;
    return (uint64_t)floor(ldexp(rho, 32));
}

int oracle_bernoulli_sample(uint64_t n, uint64_t seed, uint64_t threshold, uint8_t *mask)
{
    uint64_t i;
    uint32_t ctr[4], key[2], out[4];
    if (!mask && n)
        return -1;
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    for (i = 0; i < n; ++i) {
        uint64_t j = i / 4;
        if (i % 4 == 0) {
            ctr[0] = (uint32_t)j;
            ctr[1] = (uint32_t)(j >> 32);
            ctr[2] = ORACLE_SAMPLE_STREAM;
            ctr[3] = 0;
            oracle_philox4x32_10(ctr, key, out);
        }
        mask[i] = (uint64_t)out[i % 4] < threshold ? 1 : 0;
    }
    return 0;
}

typedef struct {
    uint32_t obj;
    uint64_t count;
} orc_freq;

static int cmp_u32(const void *pa, const void *pb)
{
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    return a < b ? -1 : a > b ? 1 : 0;
}

/* More frequent first; equal counts by the smaller object. */
static int cmp_freq(const void *pa, const void *pb)
{
    const orc_freq *x = (const orc_freq *)pa, *y = (const orc_freq *)pb;
    if (x->count != y->count)
        return x->count > y->count ? -1 : 1;
    return x->obj < y->obj ? -1 : x->obj > y->obj ? 1 : 0;
}

/* Sorts `m` objects and counts runs of equal ones; returns the number of
 * distinct objects written to `out` (room for m). */
static uint64_t count_objects(uint32_t *objs, uint64_t m, orc_freq *out)
{
    uint64_t i, d = 0;
    qsort(objs, (size_t)m, sizeof(uint32_t), cmp_u32);
    for (i = 0; i < m; ++i) {
        if (d > 0 && out[d - 1].obj == objs[i]) {
            out[d - 1].count += 1;
        } else {
            out[d].obj = objs[i];
            out[d].count = 1;
            ++d;
        }
    }
    return d;
}

int oracle_frequent(const uint32_t *obj, uint64_t n, const uint8_t *mask, uint32_t k,
                    uint32_t kstar, int exact, uint32_t *out_obj, uint64_t *out_cnt,
                    uint64_t *sample_size)
{
    uint64_t i, m = 0, d;
    uint32_t *sample, *cand;
    orc_freq *freq;
    if (!obj || !mask || !out_obj || !out_cnt || k == 0 || n == 0)
        return -1;
    if (exact && kstar < k)
        return -1;
    /* Step 1: the Bernoulli sample (the decisions are given). */
    sample = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    freq = (orc_freq *)malloc((size_t)n * sizeof(orc_freq));
    if (!sample || !freq) {
        free(sample);
        free(freq);
        return -1;
    }
    for (i = 0; i < n; ++i)
        if (mask[i])
            sample[m++] = obj[i];
    if (sample_size)
        *sample_size = m;
    /* Step 2: count the sampled objects. */
    d = count_objects(sample, m, freq);
    /* Step 3: the most frequently sampled ones (k for PAC, k* for EC). */
    qsort(freq, (size_t)d, sizeof(orc_freq), cmp_freq);
    if (!exact) {
        if (k > d) {
            free(sample);
            free(freq);
            return -1;
        }
        for (i = 0; i < k; ++i) {
            out_obj[i] = freq[i].obj;
            out_cnt[i] = freq[i].count;
        }
        free(sample);
        free(freq);
        return 0;
    }
    if (kstar > d) {
        free(sample);
        free(freq);
        return -1;
    }
    /* Step 4 (EC): count the k* candidates exactly over the whole input. */
    cand = sample; /* reuse: the k* candidate objects, sorted */
    for (i = 0; i < kstar; ++i)
        cand[i] = freq[i].obj;
    qsort(cand, kstar, sizeof(uint32_t), cmp_u32);
    for (i = 0; i < kstar; ++i) {
        freq[i].obj = cand[i];
        freq[i].count = 0;
    }
    for (i = 0; i < n; ++i) {
        uint32_t lo = 0, hi = kstar; /* binary search among the candidates */
        while (lo < hi) {
            uint32_t mid = lo + (hi - lo) / 2;
            if (cand[mid] < obj[i])
                lo = mid + 1;
            else
                hi = mid;
        }
        if (lo < kstar && cand[lo] == obj[i])
            freq[lo].count += 1;
    }
    /* Step 5: the k most frequent candidates by exact count. */
    qsort(freq, kstar, sizeof(orc_freq), cmp_freq);
    for (i = 0; i < k; ++i) {
        out_obj[i] = freq[i].obj;
        out_cnt[i] = freq[i].count;
    }
    free(sample);
    free(freq);
    return 0;
}

int oracle_frequent_plan(uint64_t n, uint32_t k, double eps, double delta, uint32_t pes,
                         int exact, double *rho, uint32_t *kstar)
{
    double rho_n, ks;
    if (!rho || !kstar || n == 0 || k == 0 || !(eps > 0.0) || !(delta > 0.0) ||
        !(delta < 1.0) || pes == 0)
        return -1;
    if (!exact) {
        /* Equation sampleSize (Section 7.1). */
        double a = 3.0 / k * log(4.0 * n / delta);
        double b = 2.0 * log(2.0 * k / delta);
        rho_n = 4.0 / (eps * eps) * (a > b ? a : b);
        *kstar = k;
    } else {
        /* Section 7.2: k* = max(k, (1/eps) sqrt((2 log p / p) ln(n/delta))),
         * sample size 2 ln(n/delta) / (eps^2 k*). */
        ks = sqrt(2.0 * log2((double)pes) / pes * log(n / delta)) / eps;
        ks = ceil(ks);
        *kstar = ks > k ? (ks > 4294967295.0 ? 0xffffffffu : (uint32_t)ks) : k;
        rho_n = 2.0 / (eps * eps * *kstar) * log(n / delta);
    }
    *rho = rho_n >= (double)n ? 1.0 : rho_n / n;
    return 0;
}
