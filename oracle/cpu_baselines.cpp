// cpu_baselines.cpp — timed CPU baselines for the benchmark (TEST
// INFRASTRUCTURE: loaded only by bench.py's CPU-baseline leg and its tests;
// the CUDA library neither loads nor shares anything with it).
//
// Two ordinary ways to select the k smallest float32 keys on a CPU, against
// which the GPU's throughput is reported:
//   * sort-and-take on every host core: the keys are made into 64-bit pairs
//     (an order-preserving unsigned image of the key, then the position, so
//     equal keys are ordered by position as in the paper's Section 2), each
//     thread sorts one contiguous chunk with std::sort, and the k smallest
//     pairs are taken by merging the sorted chunks (a heap of chunk heads);
//   * selection on one core: std::nth_element on the same pairs.
// The image of an IEEE binary32 pattern: negative patterns complemented,
// non-negative ones with the sign bit set, so unsigned order is totalOrder.
#include <algorithm>
#include <cstdint>
#include <queue>
#include <thread>
#include <utility>
#include <vector>

namespace {

inline uint64_t pair_of(uint32_t bits, uint64_t pos) {
    const uint32_t img = (bits & 0x80000000u) ? ~bits : (bits | 0x80000000u);
    return ((uint64_t)img << 32) | pos;
}

void make_pairs(const uint32_t* bits, uint64_t lo, uint64_t hi, uint64_t* out) {
    for (uint64_t i = lo; i < hi; ++i) out[i] = pair_of(bits[i], i);
}

uint64_t chunk_begin(uint64_t n, int threads, int t) { return n * (uint64_t)t / (uint64_t)threads; }

} // namespace

extern "C" {

// Builds the n pairs of `bits` into work[0..n) and sorts `threads` contiguous
// chunks of it, one per thread.  n < 2^32.  Returns 0, or -1 on bad arguments.
int cpu_sort_chunks_f32(const uint32_t* bits, uint64_t n, int threads, uint64_t* work) {
    if (!bits || !work || threads < 1 || n >= (1ull << 32)) return -1;
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t) {
        pool.emplace_back([=] {
            const uint64_t lo = chunk_begin(n, threads, t), hi = chunk_begin(n, threads, t + 1);
            make_pairs(bits, lo, hi, work);
            std::sort(work + lo, work + hi);
        });
    }
    for (auto& th : pool) th.join();
    return 0;
}

// The k smallest pairs of work[0..n) sorted in `threads` chunks (as left by
// cpu_sort_chunks_f32), merged: sel_idx[0..k) receives their positions in
// ascending order, *kth_idx the position of the k-th.  Returns 0 or -1.
int cpu_take_k(const uint64_t* work, uint64_t n, int threads, uint64_t k, uint32_t* sel_idx,
               uint32_t* kth_idx) {
    if (!work || !sel_idx || !kth_idx || threads < 1 || k < 1 || k > n) return -1;
    typedef std::pair<uint64_t, int> head; // (pair, chunk)
    std::priority_queue<head, std::vector<head>, std::greater<head>> heads;
    std::vector<uint64_t> at(threads), end(threads);
    for (int t = 0; t < threads; ++t) {
        at[t] = chunk_begin(n, threads, t);
        end[t] = chunk_begin(n, threads, t + 1);
        if (at[t] < end[t]) heads.push(head(work[at[t]], t));
    }
    uint64_t last = 0;
    for (uint64_t i = 0; i < k; ++i) {
        const head h = heads.top();
        heads.pop();
        last = h.first;
        sel_idx[i] = (uint32_t)h.first;
        const int t = h.second;
        if (++at[t] < end[t]) heads.push(head(work[at[t]], t));
    }
    *kth_idx = (uint32_t)last;
    return 0;
}

// Selection on one core: the n pairs of `bits` in work[0..n), then
// std::nth_element for rank k; the k smallest pairs end up in work[0..k) in
// some order.  *kth_idx receives the rank-k position.  Returns 0 or -1.
int cpu_nth_element_f32(const uint32_t* bits, uint64_t n, uint64_t k, uint64_t* work, uint32_t* kth_idx) {
    if (!bits || !work || !kth_idx || k < 1 || k > n || n >= (1ull << 32)) return -1;
    make_pairs(bits, 0, n, work);
    std::nth_element(work, work + (k - 1), work + n);
    *kth_idx = (uint32_t)work[k - 1];
    return 0;
}

} // extern "C"
