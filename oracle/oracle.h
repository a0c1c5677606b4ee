/*
 * oracle.h — CPU oracle for exact k-smallest selection (TEST INFRASTRUCTURE).
 *
 * This header and oracle.c are test infrastructure.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load them.  The
 * product path (the CUDA library) shares no code, header, table or constant
 * with this directory, and neither side includes the other.
 *
 * What it computes (paper, Section 2 "Preliminaries" and Section 4):
 *   - the objects are made unique by replacing value v of object x by the
 *     pair (v, x), x = the object's position in the input (Section 2);
 *   - selection returns the objects of rank <= k, i.e. the k smallest pairs,
 *     and the object of rank k (Section 4, problem statement; Algorithm
 *     "select" returns the object of rank k);
 *   - multisequence selection returns, for p sorted sequences, how many of
 *     each sequence lie among the k smallest of the union (Section 4.2 and
 *     Appendix A, Algorithm msSelect), ties ordered by (run, position).
 *
 * Value order per key type:
 *   ORC_U32, ORC_U64 : unsigned integer order;
 *   ORC_I32          : two's-complement signed order;
 *   ORC_F32, ORC_BF16: IEEE 754-2008 totalOrder (clause 5.10) on the bit
 *                      pattern: every negative pattern precedes every positive
 *                      one; among positives a larger magnitude field is larger;
 *                      among negatives a larger magnitude field is smaller.
 *                      Hence -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN.
 *
 * Method: build all n pairs, sort them once with a comparator written from the
 * order above (C library qsort), take the first k.  Plain and slow on purpose.
 */
#ifndef TOPK_ORACLE_H
#define TOPK_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_U32 = 0, ORC_I32 = 1, ORC_F32 = 2, ORC_BF16 = 3, ORC_U64 = 4 };

/* Key width in bytes of a dtype code, 0 if unknown. */
int oracle_key_bytes(int dtype);

/* Compare two raw key bit patterns (zero-extended into 64 bits) under the
 * value order of `dtype`.  Returns -1, 0 or +1. */
int oracle_key_cmp(int dtype, uint64_t a, uint64_t b);

/* Full ascending order of the n pairs (keys[i], i): perm[r] = index of the
 * pair of rank r+1.  keys holds n keys of `dtype` in host memory.
 * Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_sort_order(const void *keys, uint64_t n, int dtype, uint32_t *perm);

/* The k largest: pairs ordered by value descending, equal values by
 * ascending index (the position tie-break of Section 2 kept), first k taken.
 * Arguments and returns as oracle_select. */
int oracle_select_largest(const void *keys, uint64_t n, int dtype, uint64_t k,
                          uint32_t *sel_idx, uint32_t *kth_idx);

/* The k smallest pairs.  sel_idx receives their k indices in ascending pair
 * order; *kth_idx the index of the pair of rank k.  Needs 1 <= k <= n,
 * n < 2^32.  Returns 0, or -1 on bad arguments. */
int oracle_select(const void *keys, uint64_t n, int dtype, uint64_t k,
                  uint32_t *sel_idx, uint32_t *kth_idx);

/* How many pairs (keys[i], i) precede the pair (keys[pos], pos): in the
 * order of oracle_select when descending = 0, of oracle_select_largest when
 * descending = 1.  The pair of rank k has k - 1 before it.  One pass over
 * the keys, no sort (for checks at sizes where sorting is slow).  Returns 0,
 * or -1 on bad arguments. */
int oracle_pairs_before(const void *keys, uint64_t n, int dtype, uint64_t pos,
                        int descending, uint64_t *count);

/* Checks a claimed selection against the definition without sorting (for
 * sizes where the full sort is slow): positions sel_idx[0..k) with output keys
 * out_keys[0..k) (NULL: not checked), rank-k position kth and rank-k key
 * kth_key[0] (NULL: not checked), for the k smallest (descending = 0) or the
 * k largest (descending = 1).  Returns 0 if it is exactly that set with the
 * right keys; 1 if the rank-k pair has the wrong rank, 2 if a position
 * repeats or is out of range, 3 if a claimed pair comes after the rank-k
 * pair, 4 if an output key differs from the input key at its position;
 * -1 on bad arguments. */
int oracle_check_selection(const void *keys, uint64_t n, int dtype, uint64_t k,
                           int descending, const uint32_t *sel_idx, const void *out_keys,
                           uint64_t kth, const void *kth_key);

/* Multisequence selection over p runs stored back to back in `keys`
 * (u64 keys; run r is keys[run_off[r] .. run_off[r+1]) ).  Pairs are ordered
 * by (key, run, position), i.e. by (key, concatenated index).  split[r]
 * receives the number of the k smallest pairs that lie in run r; *kth_run and
 * *kth_pos the run and position of the pair of rank k.  The runs need not be
 * sorted for this definition; when they are, split[r] is the prefix of run r
 * that is selected.  Needs 1 <= k <= total, total < 2^32.  Returns 0 or -1. */
int oracle_select_runs(const uint64_t *keys, const uint64_t *run_off, uint32_t p,
                       uint64_t k, uint64_t *split, uint32_t *kth_run,
                       uint64_t *kth_pos);

/* Bulk deleteMin* (Section 5) of a priority queue held as p runs with
 * cursors: the queue holds the pairs of run r at positions >= cursor[r].
 * The k smallest of them, ordered as in oracle_select_runs, are deleted:
 * cursor[r] (in/out) grows by the number of them in run r; *kth_run and
 * *kth_pos receive the largest pair deleted.  The runs need not be sorted
 * for this definition; when they are, the deleted pairs of run r are
 * positions old cursor .. new cursor - 1.  Needs 1 <= k <= remaining,
 * cursor[r] <= run length, total < 2^32.  Returns 0 or -1 (cursor untouched
 * on -1). */
int oracle_runs_delete_min(const uint64_t *keys, const uint64_t *run_off, uint32_t p,
                           uint64_t *cursor, uint64_t k, uint32_t *kth_run,
                           uint64_t *kth_pos);

/* Independent selections over `rows` rows stored back to back:
 * row i is keys[row_off[i] .. row_off[i+1]) with its own k = row_k[i].
 * The selected indices (row-local, ascending pair order) of row i go to
 * sel_idx[out_off[i] .. out_off[i] + row_k[i]); kth_idx[i] gets row i's
 * rank-k index.  Returns 0 or -1. */
int oracle_select_batched(const void *keys, const uint64_t *row_off,
                          const uint32_t *row_k, uint32_t rows, int dtype,
                          const uint64_t *out_off, uint32_t *sel_idx,
                          uint32_t *kth_idx);

/* ---- Top-k most frequent objects (Section 7) ---- */

/* Philox4x32-10 (Salmon et al., SC'11): out = the four output words for
 * counter ctr[0..3] and key key[0..1]. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Counter word 2 of the sampling stream. */
#define ORACLE_SAMPLE_STREAM 0x53414d50u

/* Integer threshold of sampling probability rho: floor(rho * 2^32), 2^32
 * for rho >= 1, 0 for rho <= 0. */
uint64_t oracle_sample_threshold(double rho);

/* Bernoulli sample decisions (Section 7.1): element i is sampled iff word
 * i % 4 of Philox4x32-10 at counter (i / 4 low, i / 4 high,
 * ORACLE_SAMPLE_STREAM, 0) and key (seed low, seed high) is below
 * `threshold`.  mask[i] = 1 when sampled.  Returns 0 or -1. */
int oracle_bernoulli_sample(uint64_t n, uint64_t seed, uint64_t threshold, uint8_t *mask);

/* Algorithm PAC (exact = 0, Section 7.1) or EC (exact = 1, Section 7.2) on
 * one PE, the sample given as mask: counts the sampled objects; PAC
 * returns the k most frequently sampled objects with their sample counts;
 * EC takes the k* most frequently sampled ones, counts them over the whole
 * input and returns the k most frequent of them with their exact counts.
 * "Most frequent" orders by count, larger first, then by the smaller
 * object.  Output in that order.  *sample_size (may be NULL) receives the
 * number of sampled elements.  Returns -1 when fewer than k (PAC) or k*
 * (EC) distinct objects were sampled. */
int oracle_frequent(const uint32_t *obj, uint64_t n, const uint8_t *mask, uint32_t k,
                    uint32_t kstar, int exact, uint32_t *out_obj, uint64_t *out_cnt,
                    uint64_t *sample_size);

/* Sampling probability and k* from the accuracy targets: PAC by equation
 * sampleSize (Section 7.1), EC by Section 7.2 (log p taken base 2).  rho is
 * clamped to 1.  Returns 0 or -1. */
int oracle_frequent_plan(uint64_t n, uint32_t k, double eps, double delta, uint32_t pes,
                         int exact, double *rho, uint32_t *kstar);

#ifdef __cplusplus
}
#endif
#endif
