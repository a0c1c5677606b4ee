// runs.cu — topk_select_sorted_runs: selection of rank k across p locally
// sorted runs (paper, Section 4.2; Appendix A, Algorithm msSelect), with d
// pivots per round as in Section 4.3 "Multiple Concurrent Trials".
//
// Order: pairs (key, g) where g = off[r] + pos is the concatenated index, so
// ties are ordered by (run, position).  Every run r keeps a bracket
// [lo_r, hi_r): positions below lo_r are known to be selected, positions from
// hi_r on are known not to be.  Initially hi_r = min(len_r, k): only the
// first k objects of each run can be selected (Appendix A).
//
// One round (k_runs_round, one block per pivot):
//   - pivot v_j is drawn uniformly from the undecided objects (a prefix sum
//     over the bracket sizes locates it, Appendix A);
//   - every run counts its bracket objects below v_j by binary search
//     ("find j such that s[1..j] < v", Appendix A), the block sums them into
//     the pivot's rank (the paper's sum reduction);
//   - the last block to finish (block-done counter, no waiting) keeps the
//     highest pivot below rank k and the lowest above it, narrows every
//     bracket and draws the next pivots; a pivot of rank exactly k ends the
//     search.
// When at most T objects remain undecided, k_runs_finish gathers them into
// one block, selects the remaining rank among them and derives the splits.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "internal.h"
#include "select_core.cuh"

namespace topk {

constexpr int RUN_NT = 256;
constexpr int RUN_FIN_NT = 1024;
constexpr u32 RUN_T = 8192;         // objects finished in one block
constexpr u32 RUN_MAX_D = 256;      // pivots per round
constexpr u32 RUN_MAX_BLOCK_ROUNDS = 512;

enum : u32 { RPH_RUN = 0, RPH_FINISH = 1, RPH_DONE = 2, RPH_ERROR = 3 };

struct RunsState {
    u64 total;    // objects in all runs
    u64 k_rem;    // rank (1-based) sought among the undecided objects
    u64 m;        // undecided objects
    u64 kmin, kmax; // flexible k: the range still allowed, counted among the undecided objects
    u64 committed;  // objects already selected (below every lo_r)
    u32 phase, round, status, rounds_grid;
    u32 rounds_block, pad0;
};

struct RunsArgs {
    const u64* keys;
    const u64* off; // p + 1
    u32 p;
    u64 k;
    u32 d;          // pivots per round
    u64 seed;
    u32 flags;
    u64* lo;        // p
    u64* hi;        // p
    u64* prefix;    // p + 1: exclusive prefix of hi - lo
    u32* cnt;       // d * p: bracket objects of run r below pivot j
    u64* piv_key;   // d
    u64* piv_g;     // d: concatenated index
    u32* piv_run;   // d
    u64* piv_rank;  // d: undecided objects below pivot j
    RunsState* st;
    u32* counter;   // block-done counter (zero between rounds)
    u32* err;
    u64* split;     // p (caller)
    u64* kth_key;   // 1 (caller)
    u32* kth_run;
    u64* kth_pos;
    // bulk priority queue (Section 5): run r starts at its cursor start[r]
    // (objects before it were deleted); nullptr = every run from 0
    const u64* start;
    // flexible k (Section 4.3, Algorithm amsSelect): any k in [kmin, kmax]
    u32 flexible;
    u64 kmin, kmax;
    u64* k_out;     // 1 (caller): the k chosen
};

constexpr u64 VOID_PIVOT = ~(u64)0; // a trial whose every run fell short (no estimate)

__device__ inline void runs_latch(const RunsArgs& a, u32 code) {
    atomicCAS(a.err, 0u, code);
    a.st->status = code;
    a.st->phase = RPH_ERROR;
}

// (key, g) < (vk, vg)
__device__ __forceinline__ bool pair_less(u64 key, u64 g, u64 vk, u64 vg) {
    return key < vk || (key == vk && g < vg);
}

// Number of positions q in [lo, hi) of run r whose object is below (vk, vg):
// the predicate is monotone in q because the run is sorted and g grows with q.
__device__ __forceinline__ u64 count_below(const u64* keys, u64 base, u64 lo, u64 hi, u64 vk, u64 vg) {
    while (lo < hi) {
        const u64 mid = lo + (hi - lo) / 2;
        if (pair_less(__ldg(keys + base + mid), base + mid, vk, vg)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Block-wide exclusive prefix of (hi_r - lo_r) into a.prefix; returns the total.
__device__ u64 block_prefix_brackets(const RunsArgs& a, u64* warp_sums, u64* carry_smem) {
    const u32 tid = threadIdx.x, lane = lane_id(), warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) *carry_smem = 0;
    __syncthreads();
    for (u32 base = 0; base < a.p; base += blockDim.x) {
        const u32 r = base + tid;
        const u64 v = r < a.p ? a.hi[r] - a.lo[r] : 0;
        u64 incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u64 y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (u32)o) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (tid == 0) {
            u64 acc = 0;
            for (u32 w = 0; w < nw; ++w) {
                const u64 t = warp_sums[w];
                warp_sums[w] = acc;
                acc += t;
            }
            warp_sums[nw] = acc;
        }
        __syncthreads();
        const u64 carry = *carry_smem;
        if (r < a.p) a.prefix[r] = carry + warp_sums[warp] + incl - v;
        __syncthreads();
        if (tid == 0) *carry_smem = carry + warp_sums[nw];
        __syncthreads();
    }
    const u64 total = *carry_smem;
    if (tid == 0) a.prefix[a.p] = total;
    __syncthreads();
    return total;
}

// Draws the d pivots of round `round` uniformly among the m undecided
// objects (prefix must be current).
__device__ void draw_pivots(const RunsArgs& a, u64 m, u32 round) {
    for (u32 j = threadIdx.x; j < a.d; j += blockDim.x) {
        const Philox4 rr = philox4x32_10(j, round, 0x52554E53u, 0, (u32)a.seed, (u32)(a.seed >> 32));
        const u64 u64r = ((u64)rr.v[1] << 32) | rr.v[0];
        const u64 u = (u64)(((u128)u64r * m) >> 64); // uniform in [0, m)
        // run r with prefix[r] <= u < prefix[r+1]
        u32 lo = 0, hi = a.p;
        while (hi - lo > 1) {
            const u32 mid = (lo + hi) / 2;
            if (a.prefix[mid] <= u) lo = mid;
            else hi = mid;
        }
        const u64 pos = a.lo[lo] + (u - a.prefix[lo]);
        const u64 g = a.off[lo] + pos;
        a.piv_key[j] = a.keys[g];
        a.piv_g[j] = g;
        a.piv_run[j] = lo;
    }
}

// Geometric deviate on {1, 2, ...} with ln(1 - q) = ln_keep (<= 0): the
// number of Bernoulli(q) trials up to the first success, from one uniform
// variate by inversion.  ln_keep = -inf (q = 1) gives 1.
__device__ __forceinline__ u64 geometric_deviate(u32 bits, float ln_keep) {
    if (isinf(ln_keep)) return 1;                  // q = 1
    if (!(ln_keep < 0.f)) return ~(u64)0;          // q = 0: never
    const float u = ((float)(bits >> 8) + 0.5f) * (1.0f / 16777216.0f); // (0, 1)
    const float x = floorf(logf(u) / ln_keep);
    return x >= 1.8e19f ? ~(u64)0 : (u64)x + 1;
}

// The d trials of a flexible round (Section 4.3, Algorithm amsSelect with
// "Multiple Concurrent Trials"): in every run r, trial j draws a geometric
// deviate x and takes the run's x-th smallest undecided object (min-based
// estimator) or its x-th largest (max-based estimator, used when the range
// sought lies in the upper half); the trial's estimate is the minimum
// (maximum) of those over all runs, an object whose rank is most likely in
// [kmin, kmax].  One warp per trial.
__device__ void draw_flexible(const RunsArgs& a, const RunsState& st, u32 round) {
    const u64 m = st.m, kmin = st.kmin, kmax = st.kmax;
    const bool min_based = kmin < m - (kmax < m ? kmax : m);
    // ln(1 - q): q = 1 - ((kmin-1)/kmax)^(1/(kmax-kmin+1)), or for the
    // max-based estimator q = 1 - ((m-kmax)/(m-kmin+1))^(1/(kmax-kmin+1))
    // (as log1p of the complement, accurate when the ratio is close to 1)
    const float span = (float)(kmax - kmin + 1);
    const float ln_keep = min_based ? log1pf(-span / (float)kmax) / span
                                    : log1pf(-span / (float)(m - kmin + 1)) / span;
    const u32 lane = lane_id(), nwarps = blockDim.x >> 5;
    for (u32 j = threadIdx.x >> 5; j < a.d; j += nwarps) {
        u64 bk = min_based ? ~(u64)0 : 0, bg = VOID_PIVOT;
        u32 br = 0;
        constexpr u32 B = 8; // runs per lane whose loads are in flight together
        for (u32 r0 = lane; r0 < a.p; r0 += 32 * B) {
            u64 gg[B], kk[B];
#pragma unroll
            for (u32 b = 0; b < B; ++b) {
                const u32 r = r0 + 32 * b;
                gg[b] = VOID_PIVOT;
                if (r < a.p) {
                    const u64 lo = a.lo[r], hi = a.hi[r];
                    const Philox4 rr = philox4x32_10(r, j, round, 0x414D5345u, (u32)a.seed, (u32)(a.seed >> 32));
                    const u64 x = geometric_deviate(rr.v[0], ln_keep);
                    if (x <= hi - lo) gg[b] = a.off[r] + (min_based ? lo + x - 1 : hi - x);
                }
            }
#pragma unroll
            for (u32 b = 0; b < B; ++b) kk[b] = gg[b] != VOID_PIVOT ? a.keys[gg[b]] : 0;
#pragma unroll
            for (u32 b = 0; b < B; ++b) {
                if (gg[b] == VOID_PIVOT) continue;
                const bool better = bg == VOID_PIVOT ||
                                    (min_based ? pair_less(kk[b], gg[b], bk, bg) : pair_less(bk, bg, kk[b], gg[b]));
                if (better) {
                    bk = kk[b];
                    bg = gg[b];
                    br = r0 + 32 * b;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const u64 ok = __shfl_xor_sync(0xffffffffu, bk, o), og = __shfl_xor_sync(0xffffffffu, bg, o);
            const u32 orr = __shfl_xor_sync(0xffffffffu, br, o);
            const bool take = og != VOID_PIVOT &&
                              (bg == VOID_PIVOT || (min_based ? pair_less(ok, og, bk, bg) : pair_less(bk, bg, ok, og)));
            if (take) {
                bk = ok;
                bg = og;
                br = orr;
            }
        }
        if (lane == 0) {
            a.piv_key[j] = bk;
            a.piv_g[j] = bg;
            a.piv_run[j] = br;
        }
    }
}

// Trial j's estimate, drawn by a whole block (the round kernel, one block
// per trial): every thread takes some runs, the block reduces to the
// minimum (maximum) pair.  Result in piv_*[j].
__device__ void draw_flexible_block(const RunsArgs& a, const RunsState& st, u32 j, u32 round, u64* red_k, u64* red_g,
                                    u32* red_r) {
    const u64 m = st.m, kmin = st.kmin, kmax = st.kmax;
    const bool min_based = kmin < m - (kmax < m ? kmax : m);
    const float span = (float)(kmax - kmin + 1);
    const float ln_keep = min_based ? log1pf(-span / (float)kmax) / span
                                    : log1pf(-span / (float)(m - kmin + 1)) / span;
    const u32 lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    u64 bk = min_based ? ~(u64)0 : 0, bg = VOID_PIVOT;
    u32 br = 0;
    auto consider = [&](u64 key, u64 g, u32 r) {
        if (g == VOID_PIVOT) return;
        if (bg == VOID_PIVOT || (min_based ? pair_less(key, g, bk, bg) : pair_less(bk, bg, key, g))) {
            bk = key;
            bg = g;
            br = r;
        }
    };
    for (u32 r = threadIdx.x; r < a.p; r += blockDim.x) {
        const u64 lo = a.lo[r], hi = a.hi[r];
        const Philox4 rr = philox4x32_10(r, j, round, 0x414D5345u, (u32)a.seed, (u32)(a.seed >> 32));
        const u64 x = geometric_deviate(rr.v[0], ln_keep);
        if (x > hi - lo) continue;
        const u64 g = a.off[r] + (min_based ? lo + x - 1 : hi - x);
        consider(a.keys[g], g, r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const u64 ok = __shfl_xor_sync(0xffffffffu, bk, o), og = __shfl_xor_sync(0xffffffffu, bg, o);
        const u32 orr = __shfl_xor_sync(0xffffffffu, br, o);
        consider(ok, og, orr);
    }
    if (lane == 0) {
        red_k[warp] = bk;
        red_g[warp] = bg;
        red_r[warp] = br;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (u32 w = 1; w < nw; ++w) consider(red_k[w], red_g[w], red_r[w]);
        a.piv_key[j] = bk;
        a.piv_g[j] = bg;
        a.piv_run[j] = br;
    }
    __syncthreads();
}

struct RunsSmem {
    u64 warp_sums[RUN_FIN_NT / 32 + 1];
    u64 carry;
    u64 red[RUN_FIN_NT / 32];
    int best_lo, best_hi, exact;
    u32 flag;
};

// The branch after a round: keep the tightest pivots (one block).
__device__ void runs_decide(const RunsArgs& a, RunsSmem& sm) {
    RunsState* st = a.st;
    const u32 tid = threadIdx.x;
    if (tid == 0) {
        // the undecided objects below the pivot sought: exactly k_rem - 1, or
        // (flexible) any number in [kmin - 1, kmax - 1]
        const u64 tlo = a.flexible ? st->kmin - 1 : st->k_rem - 1;
        const u64 thi = a.flexible ? st->kmax - 1 : st->k_rem - 1;
        int bl = -1, bh = -1, ex = -1;
        u64 rl = 0, rh = ~(u64)0;
        for (u32 j = 0; j < a.d; ++j) {
            if (__ldcg(a.piv_g + j) == VOID_PIVOT) continue;
            const u64 rj = __ldcg(a.piv_rank + j);
            if (rj >= tlo && rj <= thi) {
                if (ex < 0) ex = (int)j;
            } else if (rj < tlo && (bl < 0 || rj > rl)) {
                bl = (int)j;
                rl = rj;
            } else if (rj > thi && (bh < 0 || rj < rh)) {
                bh = (int)j;
                rh = rj;
            }
        }
        sm.best_lo = bl;
        sm.best_hi = bh;
        sm.exact = ex;
    }
    __syncthreads();
    const int ex = sm.exact, bl = sm.best_lo, bh = sm.best_hi;
    if (ex >= 0) { // pivot ex has rank k: everything below it is selected
        const u32 vr = a.piv_run[ex];
        for (u32 r = tid; r < a.p; r += blockDim.x)
            a.split[r] = a.lo[r] + __ldcg(a.cnt + (size_t)ex * a.p + r) + (r == vr ? 1 : 0);
        if (tid == 0) {
            *a.kth_key = a.piv_key[ex];
            *a.kth_run = vr;
            *a.kth_pos = a.piv_g[ex] - a.off[vr];
            if (a.k_out) *a.k_out = st->committed + __ldcg(a.piv_rank + ex) + 1;
            st->phase = RPH_DONE;
        }
        __syncthreads();
        return;
    }
    for (u32 r = tid; r < a.p; r += blockDim.x) {
        const u64 l = a.lo[r];
        if (bh >= 0) a.hi[r] = l + __ldcg(a.cnt + (size_t)bh * a.p + r);
        if (bl >= 0) a.lo[r] = l + __ldcg(a.cnt + (size_t)bl * a.p + r) + (r == a.piv_run[bl] ? 1 : 0);
    }
    __syncthreads();
    const u64 m = block_prefix_brackets(a, sm.warp_sums, &sm.carry);
    if (tid == 0) {
        if (bl >= 0) {
            const u64 below = __ldcg(a.piv_rank + bl) + 1; // now selected
            st->k_rem -= below;
            st->committed += below;
            if (a.flexible) {
                st->kmin -= below;
                st->kmax -= below;
            }
        }
        if (a.flexible) {
            if (st->kmax > m) st->kmax = m;
            st->k_rem = st->kmin; // what the one-block finish selects
        }
        st->m = m;
        st->round += 1;
        if (m <= RUN_T) st->phase = RPH_FINISH;
    }
    __syncthreads();
    // (flexible trials are drawn by the next round's blocks, one per trial)
    if (st->phase == RPH_RUN && !a.flexible) draw_pivots(a, m, st->round);
    __syncthreads();
}

__global__ void __launch_bounds__(RUN_FIN_NT) k_runs_init(RunsArgs a) {
    grid_dep_wait();
    grid_dep_release();
    __shared__ RunsSmem sm;
    RunsState* st = a.st;
    const u64 total = a.off[a.p];
    if (threadIdx.x == 0) {
        st->total = total;
        st->k_rem = a.flexible ? a.kmin : a.k;
        st->kmin = a.flexible ? a.kmin : a.k;
        st->kmax = a.flexible ? a.kmax : a.k;
        st->committed = 0;
        st->round = 0;
        st->status = 0;
        st->rounds_grid = 0;
        st->rounds_block = 0;
        st->phase = RPH_RUN;
        sm.flag = 1;
        if (a.off[0] != 0 || (a.flexible ? a.kmin : a.k) > total || total > 0xFFFFFFFFull) {
            runs_latch(a, ST_EINVAL);
            sm.flag = 0;
        }
    }
    __syncthreads();
    if (!sm.flag) return;
    for (u32 r = threadIdx.x; r < a.p; r += blockDim.x) {
        const u64 s = a.off[r], e = a.off[r + 1];
        const u64 len = e >= s ? e - s : 0;
        const u64 c = a.start ? a.start[r] : 0;
        const u64 kcap = a.flexible ? a.kmax : a.k;
        a.lo[r] = c < len ? c : len;
        // only the first k after the start of a run can be selected
        a.hi[r] = len - a.lo[r] < kcap ? len : a.lo[r] + kcap;
        if (e < s || c > len) runs_latch(a, ST_EINVAL);
    }
    __syncthreads();
    const u64 m = block_prefix_brackets(a, sm.warp_sums, &sm.carry);
    if (threadIdx.x == 0) {
        st->m = m;
        // (m holds every remaining object when fewer than k remain in total)
        if ((a.flexible ? a.kmin : a.k) > m && st->phase == RPH_RUN) runs_latch(a, ST_EINVAL);
        if (a.flexible && st->kmax > m) st->kmax = m;
        if (st->phase == RPH_RUN && m <= RUN_T) st->phase = RPH_FINISH;
    }
    __syncthreads();
    if (st->phase == RPH_RUN && !a.flexible) draw_pivots(a, m, 0);
}

// Optional order check: every run non-decreasing (one block per run).
__global__ void __launch_bounds__(RUN_NT) k_runs_check_sorted(RunsArgs a) {
    grid_dep_wait();
    grid_dep_release();
    const u32 r = blockIdx.x;
    const u64 s = a.off[r], e = a.off[r + 1];
    for (u64 i = s + 1 + threadIdx.x; i < e; i += blockDim.x)
        if (a.keys[i - 1] > a.keys[i]) {
            atomicCAS(a.err, 0u, (u32)ST_EINVAL);
            return;
        }
}

// One pivot per block: rank of v_j among the undecided objects.
__global__ void __launch_bounds__(RUN_NT) k_runs_round(RunsArgs a) {
    grid_dep_wait();
    grid_dep_release();
    __shared__ RunsSmem sm;
    __shared__ u32 is_last;
    __shared__ u64 red_k[RUN_NT / 32], red_g[RUN_NT / 32];
    __shared__ u32 red_r[RUN_NT / 32];
    RunsState* st = a.st;
    if (st->phase != RPH_RUN) return;
    const u32 j = blockIdx.x;
    if (a.flexible) draw_flexible_block(a, *st, j, st->round, red_k, red_g, red_r);
    const u64 vk = a.piv_key[j], vg = a.piv_g[j];
    u64 acc = 0;
    if (vg != VOID_PIVOT) // (a void trial has no estimate to rank)
        for (u32 r = threadIdx.x; r < a.p; r += blockDim.x) {
            const u64 lo = a.lo[r], hi = a.hi[r], base = a.off[r];
            const u64 c = count_below(a.keys, base, lo, hi, vk, vg) - lo;
            a.cnt[(size_t)j * a.p + r] = (u32)c;
            acc += c;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane_id() == 0) sm.red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 t = 0;
        for (u32 w = 0; w < blockDim.x / 32; ++w) t += sm.red[w];
        a.piv_rank[j] = t;
        __threadfence();
        is_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        *a.counter = 0;
        st->rounds_grid += 1;
    }
    runs_decide(a, sm);
}

// Remaining rounds inside one block (rare), then the final selection among
// at most T undecided objects.
__global__ void __launch_bounds__(RUN_FIN_NT) k_runs_finish(RunsArgs a) {
    grid_dep_wait();
    grid_dep_release();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typedef Comp<64> C;
    typedef C::t ct;
    ct* items = reinterpret_cast<ct*>(smem_raw);                    // RUN_T composites
    u32* run_cnt = reinterpret_cast<u32*>(items + RUN_T);          // per-run selected counts (chunked)
    __shared__ RunsSmem sm;
    __shared__ RadixSmem<64, 1> rs;
    RunsState* st = a.st;
    for (u32 it = 0; it < RUN_MAX_BLOCK_ROUNDS && st->phase == RPH_RUN; ++it) {
        if (a.flexible) {
            draw_flexible(a, *st, st->round);
            __syncthreads();
        }
        for (u32 j = 0; j < a.d; ++j) { // one block does every pivot
            const u64 vk = a.piv_key[j], vg = a.piv_g[j];
            u64 acc = 0;
            for (u32 r = threadIdx.x; r < a.p && vg != VOID_PIVOT; r += blockDim.x) {
                const u64 lo = a.lo[r];
                const u64 c = count_below(a.keys, a.off[r], lo, a.hi[r], vk, vg) - lo;
                a.cnt[(size_t)j * a.p + r] = (u32)c;
                acc += c;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane_id() == 0) sm.red[threadIdx.x >> 5] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                u64 t = 0;
                for (u32 w = 0; w < blockDim.x / 32; ++w) t += sm.red[w];
                a.piv_rank[j] = t;
            }
            __syncthreads();
        }
        __threadfence_block();
        if (threadIdx.x == 0) st->rounds_block += 1;
        runs_decide(a, sm);
    }
    if (st->phase == RPH_RUN) {
        if (threadIdx.x == 0) runs_latch(a, ST_EINTERNAL);
        return;
    }
    if (st->phase != RPH_FINISH) return; // done by an exact pivot, or error
    // gather the undecided objects (prefix is current)
    const u64 m = st->m;
    for (u64 i = threadIdx.x; i < m; i += blockDim.x) {
        u32 lo = 0, hi = a.p;
        while (hi - lo > 1) {
            const u32 mid = (lo + hi) / 2;
            if (a.prefix[mid] <= i) lo = mid;
            else hi = mid;
        }
        const u64 g = a.off[lo] + a.lo[lo] + (i - a.prefix[lo]);
        items[i] = C::make(a.keys[g], (u32)g);
    }
    __syncthreads();
    const u32 count = (u32)m;
    if (st->k_rem == 0 || st->k_rem > count) {
        if (threadIdx.x == 0) runs_latch(a, ST_EINTERNAL);
        return;
    }
    const u32 rk[1] = {(u32)(st->k_rem - 1)};
    block_select_ranks<64, 1>(items, count, rk, rs);
    const ct kth = rs.result[0];
    const u32 kg = C::idx(kth);
    // run of the rank-k object
    if (threadIdx.x == 0) {
        u32 lo = 0, hi = a.p;
        while (hi - lo > 1) {
            const u32 mid = (lo + hi) / 2;
            if (a.off[mid] <= kg) lo = mid;
            else hi = mid;
        }
        // skip empty runs that share the offset
        while (lo + 1 < a.p && a.off[lo + 1] <= kg) ++lo;
        *a.kth_key = C::key(kth);
        *a.kth_run = lo;
        *a.kth_pos = kg - a.off[lo];
        if (a.k_out) *a.k_out = st->committed + st->k_rem;
    }
    // splits: lo_r plus the undecided objects of run r not above the k-th,
    // counted in chunks of RUN_FIN_NT runs
    for (u32 r0 = 0; r0 < a.p; r0 += RUN_FIN_NT) {
        const u32 nr = min((u32)RUN_FIN_NT, a.p - r0);
        for (u32 r = threadIdx.x; r < nr; r += blockDim.x) run_cnt[r] = 0;
        __syncthreads();
        for (u32 i = threadIdx.x; i < count; i += blockDim.x) {
            const ct c = items[i];
            if (c > kth) continue;
            // run of item i by its rank among the brackets (prefix)
            u32 lo = 0, hi = a.p;
            while (hi - lo > 1) {
                const u32 mid = (lo + hi) / 2;
                if (a.prefix[mid] <= i) lo = mid;
                else hi = mid;
            }
            if (lo >= r0 && lo < r0 + nr) atomicAdd(&run_cnt[lo - r0], 1u);
        }
        __syncthreads();
        for (u32 r = threadIdx.x; r < nr; r += blockDim.x) a.split[r0 + r] = a.lo[r0 + r] + run_cnt[r];
        __syncthreads();
    }
    if (threadIdx.x == 0) st->phase = RPH_DONE;
}

static u32 runs_rounds_for(u64 p, u64 k, u32 d) {
    // undecided objects start at most p*k and shrink by about d/2 per round
    double m = (double)p * (double)k;
    const double shrink = std::max(2.0, d / 3.0);
    u32 r = 0;
    while (m > RUN_T && r < 12) {
        m /= shrink;
        ++r;
    }
    return r;
}

topk_status runs_last_stats(topk_ctx* ctx, topk_stats* out) {
    RunsState s;
    if (cudaMemcpy(&s, ctx->d_state, sizeof(RunsState), cudaMemcpyDeviceToHost) != cudaSuccess) return TOPK_ECUDA;
    out->levels_grid = s.rounds_grid;
    out->levels_block = s.rounds_block;
    return TOPK_OK;
}

} // namespace topk

using namespace topk;

namespace topk {

// Both entry points: exact k (flexible = false) or any k in [kmin, kmax].
static topk_status run_sorted_runs(topk_ctx* ctx, const void* d_keys, const uint64_t* d_run_off, uint32_t p,
                                   uint64_t k, bool flexible, uint64_t kmin, uint64_t kmax, topk_dtype dtype,
                                   uint64_t* d_split, void* d_kth_key, uint32_t* d_kth_run, uint64_t* d_kth_pos,
                                   uint64_t* d_k, const topk_params* params, void* stream,
                                   const uint64_t* d_start = nullptr) {
    if (!ctx || !d_keys || !d_run_off || !d_split || !d_kth_key || !d_kth_run || !d_kth_pos) return TOPK_EINVAL;
    if (flexible && (!d_k || kmin == 0 || kmin > kmax || kmax > 0xFFFFFFFFull)) return TOPK_EINVAL;
    if (!flexible && (k == 0 || k > 0xFFFFFFFFull)) return TOPK_EINVAL;
    if (dtype != TOPK_U64 || p == 0 || p > (1u << 24)) return TOPK_EINVAL;
    if (params && (params->flags & TOPK_FLAG_LARGEST)) return TOPK_EINVAL; // ascending runs only
    if (reinterpret_cast<uintptr_t>(d_keys) % 8 || reinterpret_cast<uintptr_t>(d_run_off) % 8) return TOPK_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return TOPK_ECUDA;
    topk_params prm{};
    if (params) prm = *params;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    RunsArgs a{};
    a.keys = static_cast<const u64*>(d_keys);
    a.off = d_run_off;
    a.p = p;
    a.k = flexible ? kmin : k;
    a.flexible = flexible ? 1u : 0u;
    a.kmin = kmin;
    a.kmax = kmax;
    a.k_out = flexible ? d_k : nullptr;
    a.start = d_start;
    a.d = prm.sample_size ? std::min<u32>(std::max<u32>(prm.sample_size, 1), RUN_MAX_D) : 64;
    a.seed = prm.seed ? prm.seed : 0x13198A2E03707344ull;
    a.flags = prm.flags;
    Carve cv;
    const size_t o_lo = cv.take(8ull * p), o_hi = cv.take(8ull * p), o_pre = cv.take(8ull * (p + 1));
    const size_t o_cnt = cv.take(4ull * a.d * p);
    const size_t o_pk = cv.take(8ull * a.d), o_pg = cv.take(8ull * a.d), o_pr = cv.take(4ull * a.d);
    const size_t o_prk = cv.take(8ull * a.d);
    topk_status rs = ensure_scratch(ctx, cv.off);
    if (rs != TOPK_OK) return rs;
    char* base = static_cast<char*>(ctx->scratch.base);
    a.lo = reinterpret_cast<u64*>(base + o_lo);
    a.hi = reinterpret_cast<u64*>(base + o_hi);
    a.prefix = reinterpret_cast<u64*>(base + o_pre);
    a.cnt = reinterpret_cast<u32*>(base + o_cnt);
    a.piv_key = reinterpret_cast<u64*>(base + o_pk);
    a.piv_g = reinterpret_cast<u64*>(base + o_pg);
    a.piv_run = reinterpret_cast<u32*>(base + o_pr);
    a.piv_rank = reinterpret_cast<u64*>(base + o_prk);
    a.st = static_cast<RunsState*>(ctx->d_state);
    a.counter = ctx->d_counter + 1;
    a.err = ctx->d_err;
    a.split = d_split;
    a.kth_key = static_cast<u64*>(d_kth_key);
    a.kth_run = d_kth_run;
    a.kth_pos = d_kth_pos;
    static_assert(sizeof(RunsState) <= 4096, "state region");
    ctx->last_kind = LAST_RUNS;

    static std::atomic<uint64_t> attr_mask{0};
    const uint64_t bit = 1ull << (ctx->device & 63);
    const size_t fin_smem = RUN_T * sizeof(u128) + RUN_FIN_NT * sizeof(u32);
    if (!(attr_mask.load() & bit)) {
        if (cudaFuncSetAttribute(k_runs_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fin_smem) !=
            cudaSuccess)
            return TOPK_ECUDA;
        attr_mask.fetch_or(bit);
    }
    // a flexible search usually ends within a round or two (each trial lands
    // in the range with constant probability); the spare rounds return at once
    const u32 rounds = flexible ? std::min<u32>(runs_rounds_for(p, kmax, a.d), 4u) : runs_rounds_for(p, k, a.d);
    cudaError_t e = launch_dep(k_runs_init, 1, RUN_FIN_NT, 0, st, a);
    if (e == cudaSuccess && (prm.flags & TOPK_FLAG_CHECK_SORTED))
        e = launch_dep(k_runs_check_sorted, (int)p, RUN_NT, 0, st, a);
    for (u32 r = 0; r < rounds && e == cudaSuccess; ++r) e = launch_dep(k_runs_round, (int)a.d, RUN_NT, 0, st, a);
    if (e == cudaSuccess) e = launch_dep(k_runs_finish, 1, RUN_FIN_NT, fin_smem, st, a);
    if (e != cudaSuccess) return cuda_status(e);
    count_launch(ctx, 2 + rounds + ((prm.flags & TOPK_FLAG_CHECK_SORTED) ? 1 : 0));
    return cuda_status(cudaGetLastError());
}

} // namespace topk

extern "C" topk_status topk_select_sorted_runs(topk_ctx* ctx, const void* d_keys, const uint64_t* d_run_off,
                                               uint32_t p, uint64_t k, topk_dtype dtype, uint64_t* d_split,
                                               void* d_kth_key, uint32_t* d_kth_run, uint64_t* d_kth_pos,
                                               const topk_params* params, void* stream) {
    return run_sorted_runs(ctx, d_keys, d_run_off, p, k, false, 0, 0, dtype, d_split, d_kth_key, d_kth_run, d_kth_pos,
                           nullptr, params, stream);
}

extern "C" topk_status topk_select_sorted_runs_flexible(topk_ctx* ctx, const void* d_keys, const uint64_t* d_run_off,
                                                        uint32_t p, uint64_t kmin, uint64_t kmax, topk_dtype dtype,
                                                        uint64_t* d_split, void* d_kth_key, uint32_t* d_kth_run,
                                                        uint64_t* d_kth_pos, uint64_t* d_k, const topk_params* params,
                                                        void* stream) {
    return run_sorted_runs(ctx, d_keys, d_run_off, p, 0, true, kmin, kmax, dtype, d_split, d_kth_key, d_kth_run,
                           d_kth_pos, d_k, params, stream);
}

extern "C" topk_status topk_runs_delete_min(topk_ctx* ctx, const void* d_keys, const uint64_t* d_run_off, uint32_t p,
                                            uint64_t* d_cursor, uint64_t k, topk_dtype dtype, void* d_kth_key,
                                            uint32_t* d_kth_run, uint64_t* d_kth_pos, const topk_params* params,
                                            void* stream) {
    if (!d_cursor) return TOPK_EINVAL;
    return run_sorted_runs(ctx, d_keys, d_run_off, p, k, false, 0, 0, dtype, d_cursor, d_kth_key, d_kth_run,
                           d_kth_pos, nullptr, params, stream, d_cursor);
}

extern "C" topk_status topk_runs_delete_min_flexible(topk_ctx* ctx, const void* d_keys, const uint64_t* d_run_off,
                                                     uint32_t p, uint64_t* d_cursor, uint64_t kmin, uint64_t kmax,
                                                     topk_dtype dtype, void* d_kth_key, uint32_t* d_kth_run,
                                                     uint64_t* d_kth_pos, uint64_t* d_k, const topk_params* params,
                                                     void* stream) {
    if (!d_cursor) return TOPK_EINVAL;
    return run_sorted_runs(ctx, d_keys, d_run_off, p, 0, true, kmin, kmax, dtype, d_cursor, d_kth_key, d_kth_run,
                           d_kth_pos, d_k, params, stream, d_cursor);
}
