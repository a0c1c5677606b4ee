// select_impl.cuh — topk_select: selection of the k smallest of n unsorted keys
// (paper, Section 2, Algorithm "select"; Section 4.1, Theorem "selectFR").
//
// Launch sequence of one call (all on the caller's stream, no host round
// trip), per recursion level:
//   k_sample (grid)     per-partition draws of the current window -> sample
//                       array + histogram over the window
//   k_pivots (1 block)  pivots = sample elements of ranks k|S|/n -/+ Delta,
//                       read off the histogram and refined in two bins
//   k_pass   (grid)     one read of the source: a -> output, b -> candidate
//                       buffer; the last block takes the branch
// then k_finish (1 block): remaining levels inside one block until at most T
// candidates are left, selection of rank k among them, the rest of the output
// and the rank-k pair.  The host predicts the number of grid levels; a level
// whose state is already small returns at once.
// k = 1 (the base case of Algorithm "select", a global minimum) and k = n
// (everything selected) take one reduction kernel instead.
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>

#include "internal.h"
#include "select_block.cuh"

namespace topk {

// ------------------------------------------------------------- kernels

// Read-after-atomics: the pass counters as the last block of the pass sees them.
__device__ __forceinline__ u64 atomic_read(u64* p) {
    return atomicAdd(reinterpret_cast<unsigned long long*>(p), 0ull);
}

// The branch of Algorithm "select", taken by the last block of a pass once
// every block's counts are in (block-done counter; nobody waits).  The calling
// thread must be the block's thread 0, after the block's own atomics.
__device__ __forceinline__ void pass_epilogue(const SelArgs& a) {
    __threadfence();
    const u32 prev = atomicAdd(a.pass_done, 1u);
    if (prev == gridDim.x - 1) {
        __threadfence();
        SelState* g = a.st;
        g->cnt_a = atomic_read(&g->cnt_a);
        g->cnt_b = atomic_read(&g->cnt_b);
        decide(*g);
        *a.pass_done = 0;
    }
}

// ---- pickPivots, part 1: the sample (whole grid)
// Every thread makes SMP_DRAWS per-partition draws of the current window,
// appends the kept ones to the sample array and counts them in a shared
// histogram over the window, added to the global histogram at the end.
constexpr int SMP_NT = 128;
constexpr int SMP_DRAWS = 4;        // one Philox block per thread
constexpr u32 SMP_MAX_SCALE = 4;    // extra draws for a narrowed window

template <int DT> __global__ void __launch_bounds__(SMP_NT) k_sample(SelArgs a, int first) {
    grid_dep_wait();
    grid_dep_release();
    typedef Key<DT> K;
    typedef typename K::key_t key_t;
    constexpr int KW = K::KW;
    typedef Comp<KW> C;
    typedef typename C::t ct;
    __shared__ u32 hist[HIST_BINS];
    for (u32 i = threadIdx.x; i < HIST_BINS; i += blockDim.x) hist[i] = 0;
    SelState s;
    if (first) {
        s.lo = 0;
        s.hi = key_domain_max<DT>();
        s.m_src = a.n;
        s.m_win = a.n;
        s.src = SRC_INPUT;
        s.level = 0;
        s.phase = PH_RUN;
    } else {
        s = *a.st;
    }
    __syncthreads();
    if (s.phase != PH_RUN || s.m_src <= a.grid_G || s.m_win <= a.finish_T) return;
    const ct lo = C::from128(s.lo), hi = C::from128(s.hi);
    const u32 sh = hist_shift(lo, hi);
    u32 draws = a.sample;
    if (s.m_win < s.m_src) { // narrowed window: draw more so that enough land inside
        u64 ratio = s.m_src / (s.m_win ? s.m_win : 1);
        ratio = ratio < 1 ? 1 : ratio > SMP_MAX_SCALE ? SMP_MAX_SCALE : ratio;
        draws = (u32)((u64)draws * ratio);
    }
    if (blockIdx.x * SMP_NT * SMP_DRAWS >= draws) return; // the whole block draws nothing
    const u32 m = (u32)s.m_src; // sources hold fewer than 2^32 elements
    const u32 p = a.parts < m ? a.parts : m;
    const u32 len = m / p, rem = m - len * p;
    const u32 j0 = (blockIdx.x * SMP_NT + threadIdx.x) * SMP_DRAWS;
    const Philox4 r = philox4x32_10(j0, s.level, 0x53414D50u, 0, (u32)a.seed, (u32)(a.seed >> 32));
    key_t kk[SMP_DRAWS];
    u32 ii[SMP_DRAWS];
    const InputSrc<DT> isrc = InputSrc<DT>::make(a.keys, m);
    const CandSrc<KW> csrc{static_cast<const key_t*>(a.cand_key[s.src == SRC_CAND1 ? 1 : 0]),
                           a.cand_idx[s.src == SRC_CAND1 ? 1 : 0], m};
    u32 keepm = 0; // bit q: draw q is inside the window
#pragma unroll
    for (int q = 0; q < SMP_DRAWS; ++q) {
        const u32 j = j0 + q;
        const u32 part = j % p; // draws dealt round-robin: an equal share per partition
        const u32 plo = part * len + (part < rem ? part : rem);
        const u32 psz = len + (part < rem ? 1 : 0);
        const u32 pos = plo + (u32)(((u64)r.v[q] * psz) >> 32);
        kk[q] = 0;
        ii[q] = 0;
        if (j < draws) {
            if (s.src == SRC_INPUT) isrc.at(pos, kk[q], ii[q]);
            else csrc.at(pos, kk[q], ii[q]);
            const ct c = C::make(kk[q], ii[q]);
            if (c >= lo && c <= hi) keepm |= 1u << q;
        }
    }
    // one slot reservation per warp for all its kept draws
    const u32 cnt = (u32)__popc(keepm);
    u32 incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane_id() >= (u32)o) incl += y;
    }
    const u32 tot = __shfl_sync(0xffffffffu, incl, 31);
    u32 slot0 = 0;
    if (lane_id() == 31 && tot) slot0 = atomicAdd(a.samp_count, tot);
    u32 slot = __shfl_sync(0xffffffffu, slot0, 31) + incl - cnt;
    ct* samp = static_cast<ct*>(a.samp);
#pragma unroll
    for (int q = 0; q < SMP_DRAWS; ++q) {
        if ((keepm >> q) & 1u) {
            const ct c = C::make(kk[q], ii[q]);
            if (slot < a.samp_cap) {
                samp[slot] = c;
                atomicAdd(&hist[hist_bin(c, lo, sh)], 1u);
            } else {
                keepm &= ~(1u << q);
            }
            ++slot;
        }
    }
    __syncthreads();
    // each touched bin is moved to the global histogram once (the first
    // thread to take it)
#pragma unroll
    for (int q = 0; q < SMP_DRAWS; ++q) {
        if (!((keepm >> q) & 1u)) continue;
        const u32 b = hist_bin(C::make(kk[q], ii[q]), lo, sh);
        const u32 v = atomicExch(&hist[b], 0u);
        if (v) atomicAdd(a.hist + b, v);
    }
}

// ---- pickPivots, part 2 (one block): pivots from the histogram and the
// sample.  The bins holding sample ranks k|S|/n -/+ Delta are found from the
// histogram's prefix sums; only the sample elements of those bins are
// gathered and ranked exactly.  Leaves the histogram and the sample count at
// zero for the next level.
constexpr int PIV_NT = 1024;

template <int KW> struct PivotSmem {
    typedef typename Comp<KW>::t ct;
    ct buf[Lim<KW>::ELEMS];
    u32 warp_sum[PIV_NT / 32];
    RadixSmem<KW, 2> rs2;
    RadixSmem<KW, 1> rs1;
    u32 bin[2], base[2], cnt[2], want[2];
    u32 flag, collect, kept;
    long long jl, jr;
    u32 whist[2][256];
    ct wres[2];
};

constexpr u32 WARP_SELECT_MAX = 512; // bins up to this size are ranked by one warp, larger ones by the block

template <int DT> __global__ void __launch_bounds__(PIV_NT) k_pivots(SelArgs a, int first) {
    grid_dep_wait();
    grid_dep_release();
    constexpr int KW = Key<DT>::KW;
    typedef Comp<KW> C;
    typedef typename C::t ct;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<PivotSmem<KW>*>(smem_raw);
    SelState* g = a.st;
    const u32 tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    // the histogram and the state are loaded at once (independent round trips)
    u32 h[4], t = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) h[q] = a.hist[tid * 4 + q];
    const SelState s = first ? initial_state<DT>(a) : *g;
    if (tid == 0) {
        if (first) *g = s;
        u32 go = s.phase == PH_RUN;
        if (go && s.m_src <= a.grid_G) {
            g->phase = PH_FINISH;
            go = 0;
        }
        sm.flag = go;
        sm.collect = s.m_win <= a.finish_T;
        const u32 c = *a.samp_count;
        sm.kept = c < a.samp_cap ? c : a.samp_cap;
        // pivot ranks once (the block shares them)
        long long jl = -1, jr = 0;
        if (go && sm.kept > 0)
            pivot_ranks(sm.kept, s.m_win, s.k_rem, a.z, (a.flags & TOPK_FLAG_RAW_DELTA) != 0, jl, jr);
        sm.jl = jl;
        sm.jr = jr;
        for (int q = 0; q < 2; ++q) {
            sm.bin[q] = 0xFFFFFFFFu;
            sm.base[q] = 0;
            sm.cnt[q] = 0;
        }
    }
    __syncthreads();
    if (sm.flag) {
        const ct lo = C::from128(s.lo), hi = C::from128(s.hi);
        ct pl = lo, pr = hi; // "collect": every window element becomes a candidate
        const u32 kept = sm.kept;
        const long long jl = sm.jl, jr = sm.jr;
        if (!sm.collect && kept > 0) {
            const long long top = (long long)kept - 1;
            const u32 rl = (u32)(jl < 0 ? 0 : jl > top ? top : jl);
            const u32 rr = (u32)(jr < 0 ? 0 : jr > top ? top : jr);
            // exclusive prefix of the histogram (4 bins per thread)
#pragma unroll
            for (int q = 0; q < 4; ++q) t += h[q];
            u32 incl = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (u32)o) incl += y;
            }
            if (lane == 31) sm.warp_sum[warp] = incl;
            __syncthreads();
            if (warp == 0) { // exclusive scan of the 32 warp totals
                const u32 v = sm.warp_sum[lane];
                u32 wi = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const u32 y = __shfl_up_sync(0xffffffffu, wi, o);
                    if (lane >= (u32)o) wi += y;
                }
                sm.warp_sum[lane] = wi - v;
            }
            __syncthreads();
            u32 run = sm.warp_sum[warp] + incl - t;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const u32 b = tid * 4 + q;
                // bin holding sample rank rl / rr
                if (h[q] && rl >= run && rl < run + h[q]) {
                    sm.bin[0] = b;
                    sm.base[0] = run;
                    sm.cnt[0] = h[q];
                }
                if (h[q] && rr >= run && rr < run + h[q]) {
                    sm.bin[1] = b;
                    sm.base[1] = run;
                    sm.cnt[1] = h[q];
                }
                run += h[q];
            }
            if (tid == 0) {
                sm.want[0] = 0;
                sm.want[1] = 0;
            }
            __syncthreads();
            // gather the two bins (one region if they coincide)
            const u32 sh = hist_shift(lo, hi);
            const u32 b0 = sm.bin[0], b1 = sm.bin[1];
            const bool same = b0 == b1;
            const u32 off1 = same ? 0 : sm.cnt[0];
            const ct* samp = static_cast<const ct*>(a.samp);
            constexpr int U = KW == 32 ? 8 : 4; // loads in flight per thread
            for (u32 base = 0; base < kept; base += PIV_NT * U) {
                ct cv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const u32 i = base + u * PIV_NT + tid;
                    cv[u] = i < kept ? samp[i] : (ct)0;
                }
                // one slot reservation per warp and bin for all U elements
                u32 m0 = 0, m1 = 0;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const u32 i = base + u * PIV_NT + tid;
                    const u32 b = i < kept ? hist_bin(cv[u], lo, sh) : 0xFFFFFFFFu;
                    m0 |= (u32)(b == b0) << u;
                    m1 |= (u32)(!same && b == b1) << u;
                }
                const u32 cnt = (u32)__popc(m0) | ((u32)__popc(m1) << 16);
                u32 incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= (u32)o) incl += y;
                }
                const u32 tot = __shfl_sync(0xffffffffu, incl, 31);
                u32 w0 = 0, w1 = 0;
                if (lane == 31) {
                    if (tot & 0xFFFFu) w0 = atomicAdd(&sm.want[0], tot & 0xFFFFu);
                    if (tot >> 16) w1 = atomicAdd(&sm.want[1], tot >> 16);
                }
                u32 s0 = __shfl_sync(0xffffffffu, w0, 31) + ((incl - cnt) & 0xFFFFu);
                u32 s1 = __shfl_sync(0xffffffffu, w1, 31) + ((incl - cnt) >> 16);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if ((m0 >> u) & 1u) {
                        if (s0 < sm.cnt[0] && s0 < Lim<KW>::ELEMS) sm.buf[s0] = cv[u];
                        ++s0;
                    }
                    if ((m1 >> u) & 1u) {
                        if (s1 < sm.cnt[1] && off1 + s1 < Lim<KW>::ELEMS) sm.buf[off1 + s1] = cv[u];
                        ++s1;
                    }
                }
            }
            __syncthreads();
            const bool consistent = sm.cnt[0] > 0 && sm.want[0] == sm.cnt[0] &&
                                    (same || (sm.cnt[1] > 0 && sm.want[1] == sm.cnt[1])) &&
                                    sm.cnt[0] + (same ? 0 : sm.cnt[1]) <= Lim<KW>::ELEMS;
            const bool small = sm.cnt[0] <= WARP_SELECT_MAX && (same || sm.cnt[1] <= WARP_SELECT_MAX);
            if (consistent && small) {
                // two warps select the two pivots concurrently
                if (warp < 2) {
                    const u32 t = warp;
                    const u32 region = (t == 1 && !same) ? 1 : 0;
                    const ct* base = sm.buf + (region ? off1 : 0);
                    const u32 rk = (t == 0 ? rl : rr) - sm.base[region];
                    const ct res = warp_select_rank<KW>(base, sm.cnt[region], rk, sm.whist[t]);
                    if (lane == 0) sm.wres[t] = res;
                }
                __syncthreads();
                if (jl >= 0) pl = sm.wres[0];
                if (jr <= top) pr = sm.wres[1];
            } else if (consistent) {
                if (same) {
                    const u32 rk[2] = {rl - sm.base[0], rr - sm.base[0]};
                    block_select_ranks<KW, 2>(sm.buf, sm.cnt[0], rk, sm.rs2);
                    if (jl >= 0) pl = sm.rs2.result[0];
                    if (jr <= top) pr = sm.rs2.result[1];
                } else {
                    const u32 rk0[1] = {rl - sm.base[0]};
                    block_select_ranks<KW, 1>(sm.buf, sm.cnt[0], rk0, sm.rs1);
                    if (jl >= 0) pl = sm.rs1.result[0];
                    const u32 rk1[1] = {rr - sm.base[1]};
                    block_select_ranks<KW, 1>(sm.buf + off1, sm.cnt[1], rk1, sm.rs1);
                    if (jr <= top) pr = sm.rs1.result[0];
                }
            } else if (tid == 0) {
                g->overflows++; // histogram and sample disagree: fall back to collecting the window
            }
        }
        if (tid == 0) {
            g->pl = (u128)pl;
            g->pr = (u128)pr;
            g->dst = s.src == SRC_CAND0 ? SRC_CAND1 : SRC_CAND0;
            g->cnt_a = 0;
            g->cnt_b = 0;
            g->pending = 1;
            g->level = s.level + 1;
            g->levels_grid++;
            if (s.level == 0) g->sample_kept = kept;
            // many a-elements expected: the pass compacts with block scans
            g->dense = (jl >= 0 && kept > 0 && (double)(jl + 1) > (double)kept / 16.0) ? 1u : 0u;
        }
    }
    __syncthreads();
    for (u32 i = tid; i < HIST_BINS; i += PIV_NT) a.hist[i] = 0;
    if (tid == 0) *a.samp_count = 0;
}

// ---- partition + reduction + branch (whole grid)

template <int DT>
__device__ __forceinline__ Sink<DT> make_sink(const SelArgs& a, const SelState& s) {
    typedef typename Key<DT>::raw_t raw_t;
    typedef typename Key<DT>::key_t key_t;
    Sink<DT> sink;
    sink.out_keys = static_cast<raw_t*>(a.out_keys);
    sink.out_idx = a.out_idx;
    sink.out_base = s.out_base;
    sink.cap_a = s.k_rem;
    sink.ck = static_cast<key_t*>(a.cand_key[s.dst - 1]);
    sink.ci = a.cand_idx[s.dst - 1];
    sink.cap_b = a.cap_b;
    sink.cnt_a = &a.st->cnt_a;
    sink.cnt_b = &a.st->cnt_b;
    return sink;
}

// Register-path pass (later levels; a first level on misaligned input).
template <int DT, bool INPUT_ONLY> __device__ void grid_pass(const SelArgs& a, const SelState& s) {
    typedef Key<DT> K;
    typedef typename K::key_t key_t;
    constexpr int KW = K::KW;
    typedef Comp<KW> C;
    typedef typename C::t ct;
    __shared__ PassSmem<PASS_NT> ps;
    __shared__ WarpQ<KW> wq[PASS_NT / 32];
    const Sink<DT> sink = make_sink<DT>(a, s);
    const ct lo = C::from128(s.lo), pl = C::from128(s.pl), pr = C::from128(s.pr);
    const bool dense = s.dense != 0, exact = lo != (ct)0, has_a = pl > lo;
    WarpQ<KW>& q = wq[threadIdx.x >> 5];
    if (INPUT_ONLY || s.src == SRC_INPUT) {
        const InputSrc<DT> src = InputSrc<DT>::make(a.keys, s.m_src);
        if (!dense) pass_tiles_sparse<PASS_NT, DT>(src, blockIdx.x, gridDim.x, lo, pl, pr, sink, q);
        else if (exact) pass_tiles<PASS_NT, true, true, DT>(src, blockIdx.x, gridDim.x, lo, pl, pr, sink, ps);
        else if (has_a) pass_tiles<PASS_NT, true, false, DT>(src, blockIdx.x, gridDim.x, lo, pl, pr, sink, ps);
        else pass_tiles<PASS_NT, false, false, DT>(src, blockIdx.x, gridDim.x, lo, pl, pr, sink, ps);
    } else if constexpr (!INPUT_ONLY) {
        const CandSrc<KW> src{static_cast<const key_t*>(a.cand_key[s.src - 1]), a.cand_idx[s.src - 1], s.m_src};
        if (!dense) pass_tiles_sparse<PASS_NT, DT>(src, blockIdx.x, gridDim.x, lo, pl, pr, sink, q);
        else if (exact) pass_tiles<PASS_NT, true, true, DT>(src, blockIdx.x, gridDim.x, lo, pl, pr, sink, ps);
        else if (has_a) pass_tiles<PASS_NT, true, false, DT>(src, blockIdx.x, gridDim.x, lo, pl, pr, sink, ps);
        else pass_tiles<PASS_NT, false, false, DT>(src, blockIdx.x, gridDim.x, lo, pl, pr, sink, ps);
    }
    __syncthreads();
    if (threadIdx.x == 0) pass_epilogue(a);
}

// First level: the source is always the input, so this variant carries no
// candidate-source code (fewer registers on the pass that reads all n keys).
template <int DT> __global__ void __launch_bounds__(PASS_NT) k_pass_first(SelArgs a) {
    grid_dep_wait();
    grid_dep_release();
    const SelState s = *a.st;
    if (s.phase != PH_RUN || !s.pending || s.src != SRC_INPUT) return;
    grid_pass<DT, true>(a, s);
}

template <int DT> __global__ void __launch_bounds__(PASS_NT) k_pass(SelArgs a) {
    grid_dep_wait();
    grid_dep_release();
    const SelState s = *a.st;
    if (s.phase != PH_RUN || !s.pending) return;
    grid_pass<DT, false>(a, s);
}

// First level, 16-byte-aligned input: a producer warp streams full tiles
// into a ring of shared-memory stages with bulk (TMA) copies while 8 consumer
// warps classify and compact, so HBM reads never wait for the compute.  Every
// wait is bounded; a timeout latches TOPK_ETIMEOUT and the block winds down
// without hanging.
constexpr int TMA_CONS = 256;
constexpr int TMA_NT = TMA_CONS + 32;
constexpr u64 WAIT_LIMIT_NS = 200ull * 1000 * 1000;

// Ring geometry.  A sparse pass is memory-bound: a deep ring, 2 blocks per
// SM.  A dense pass holds two stages per block (one counted, one being
// written out), so its ring is one or two stages deeper than that, with 3
// blocks (24 consumer warps) per SM, 2 for 64-bit keys.
template <int DT, bool DENSE = false> struct TmaCfg {
    static constexpr u32 W = sizeof(typename Key<DT>::raw_t);
    static constexpr u32 TILE = TMA_CONS * 16; // elements per stage
    static constexpr u32 BYTES = TILE * W;     // 8, 16 or 32 KiB
    static constexpr u32 STAGES = DENSE ? (W == 2 ? 8 : W == 4 ? 4 : 3) : (W == 2 ? 8 : W == 4 ? 5 : 3);
    static constexpr u32 SMEM = STAGES * BYTES;
    static constexpr int MIN_BLOCKS = DENSE ? (W == 8 ? 2 : 3) : 1;
};

// Raw key bits of this thread's 16 slots from a stage (slot q at vector
// q / EPV of the thread, element q % EPV).
template <int DT>
__device__ __forceinline__ void load_raw_stage(const unsigned char* stage, typename Key<DT>::raw_t (&rr)[16]) {
    uint4 v[InputSrc<DT>::NV];
    const uint4* sp = reinterpret_cast<const uint4*>(stage);
#pragma unroll
    for (int j = 0; j < InputSrc<DT>::NV; ++j) v[j] = sp[j * TMA_CONS + threadIdx.x];
    InputSrc<DT>::unpack_raw(v, rr);
}

// Sparse first level (few elements in a and b): the elements whose pair is
// at most pr are appended to the warp's queue (select_core.cuh); a tile that
// contains neither pivot's position finds them with one comparison of raw
// key bits per element (tile_bounds), the rare other tile on the pair.
template <int DT>
__device__ void tma_consume_sparse(const SelArgs& a, const SelState& s, const unsigned char* stages, uint64_t* full,
                                   uint64_t* empty, u64 my_n, u32* dead, WarpQ<Key<DT>::KW>& wq) {
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    typedef Comp<K::KW> C;
    typedef typename C::t ct;
    typedef TmaCfg<DT> Cfg;
    constexpr u32 EPV = InputSrc<DT>::EPV;
    const Sink<DT> sink = make_sink<DT>(a, s);
    const ct lo = C::from128(s.lo), pl = C::from128(s.pl), pr = C::from128(s.pr);
    const u32 lane = lane_id();
    const InputSrc<DT> isrc = InputSrc<DT>::make(a.keys, s.m_src); // head = 0: input is 16-byte aligned
    QState qs = QState::make();
    const TileBounds<DT> tbd = TileBounds<DT>::make(pl, pr);
    for (u64 i = 0; i < my_n; ++i) {
        const u32 stg = (u32)(i % Cfg::STAGES);
        const u32 parity = (u32)((i / Cfg::STAGES) & 1);
        bool ok = !*(volatile u32*)dead;
        if (ok && !mbar_wait_bounded(&full[stg], parity, WAIT_LIMIT_NS)) {
            ok = false;
            *(volatile u32*)dead = 1;
            if (lane == 0) latch(a.err, ST_ETIMEOUT);
        }
        ok = __all_sync(0xffffffffu, ok);
        // positions in 32 bits (inputs hold fewer than 2^32 keys): slot q of
        // this thread is ib + (q / EPV) * TMA_CONS * EPV + q % EPV
        const u32 tb = (u32)((blockIdx.x + i * gridDim.x) * (u64)Cfg::TILE);
        const u32 ib = tb + threadIdx.x * EPV;
        auto pos = [&](int q) -> u32 { return ib + (u32)(q / (int)EPV) * (TMA_CONS * EPV) + (u32)(q % (int)EPV); };
        raw_t rr[16];
        u32 hit = 0;
        if (ok) {
            load_raw_stage<DT>(stages + (size_t)stg * Cfg::BYTES, rr);
            RawBound<DT> ba, bb;
            bool any_a, any_l;
            if (tbd.get(tb, tb + Cfg::TILE - 1, ba, bb, any_a, any_l)) {
                hit = tile_le_dispatch<DT>(rr, bb, any_l);
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) hit |= (u32)(C::make(K::fwd(rr[q]), pos(q)) <= pr) << q;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) rr[q] = 0;
        }
        __syncwarp();
        if (ok && lane == 0) mbar_arrive(&empty[stg]); // keys are in registers: the stage may be refilled
        sparse_append_hits<DT>(hit, pos, [&](u32 sq) { return K::fwd(pick16(rr, sq)); }, lo, pl, pr, sink, wq, qs);
    }
    // the ragged last tile, read directly by the block that owns it
    const u64 nfull = s.m_src / Cfg::TILE;
    if (s.m_src % Cfg::TILE != 0 && nfull % gridDim.x == blockIdx.x) {
        key_t kk[16];
        u32 ii[16];
        const u64 tb = nfull * (u64)Cfg::TILE;
        const u32 valid = isrc.template load16<TMA_CONS>(tb, kk, ii);
        auto pos = [&](int q) -> u32 { return isrc.template idx_of<TMA_CONS>(tb, q); };
        classify_sparse<DT>(kk, pos, valid, lo, pl, pr, sink, wq, qs);
    }
    queue_drain<DT>(wq, qs, sink, lo, pl, pr);
}

// Dense first level (many elements in a; the window starts at the smallest
// pair).  Output room is reserved per tile with one atomic per class, but
// the reservation of tile i is issued right after the block's one barrier
// of iteration i and published before the barrier of iteration i+1, so its
// latency overlaps the work of a whole tile; tile i-1 is written after that
// barrier, re-read from its shared-memory stage, which is held until then.
// Two threads take turns issuing the atomics.
//
// A tile that contains neither pivot's position is classified with two
// comparisons of raw key bits per element (tile_bounds): ties with a pivot's
// key are decided for the whole tile by which side of the pivot's position
// it lies on.  a-elements leave by per-slot warp ballots: one store
// instruction per slot writes the warp's selected keys (and one their
// positions) to consecutive addresses, the run pointers advancing by the
// slot's count.  b-elements are few; each lane writes its own at an offset
// from one warp scan.
struct DenseSmem {
    u32 wa[2][TMA_CONS / 32], wb[2][TMA_CONS / 32]; // per-warp counts, by tile parity
    u64 oa[2][TMA_CONS / 32], ob[2][TMA_CONS / 32]; // per-warp offsets inside the tile
    u64 ba[2], bb[2];                               // tile bases in the output / candidates
};

template <int DT>
__device__ void tma_consume_dense(const SelArgs& a, const SelState& s, const unsigned char* stages, uint64_t* full,
                                  uint64_t* empty, u64 my_n, u32* dead, DenseSmem& ds, PassSmem<TMA_CONS>& ps) {
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    typedef Comp<K::KW> C;
    typedef typename C::t ct;
    typedef TmaCfg<DT, true> Cfg;
    typedef SyncNamed<1, TMA_CONS> Sync;
    constexpr int EPV = InputSrc<DT>::EPV;
    constexpr u32 STRIDE = TMA_CONS * EPV; // index distance between a thread's vectors
    const Sink<DT> sink = make_sink<DT>(a, s);
    const ct pl = C::from128(s.pl), pr = C::from128(s.pr);
    const u32 warp = threadIdx.x >> 5, lane = lane_id(), below = lanemask_lt();
    const InputSrc<DT> isrc = InputSrc<DT>::make(a.keys, s.m_src); // head = 0
    const key_t plk = (key_t)C::key(pl), prk = (key_t)C::key(pr);
    const u32 plx = C::idx(pl), prx = C::idx(pr);
    u32 ma_prev = 0, mb_prev = 0, stg_prev = 0, ib_prev = 0;
    bool ok_prev = false;
    u64 my_ra = 0, my_rb = 0;   // pending reservation of the issuing thread
    u32 ring = 0, ring_par = 0; // stage and phase parity of tile i
    for (u64 i = 0; i <= my_n; ++i) {
        const bool cur = i < my_n, have_prev = i > 0;
        const u32 par = (u32)(i & 1), ppar = par ^ 1u;
        u32 ma = 0, mb = 0, stg = 0, ib = 0;
        bool ok = false;
        if (cur) {
            stg = ring;
            const u32 fpar = ring_par;
            if (++ring == Cfg::STAGES) {
                ring = 0;
                ring_par ^= 1u;
            }
            ok = !*(volatile u32*)dead;
            if (ok && !mbar_wait_bounded(&full[stg], fpar, WAIT_LIMIT_NS)) {
                ok = false;
                *(volatile u32*)dead = 1;
                if (lane == 0) latch(a.err, ST_ETIMEOUT);
            }
            ok = __all_sync(0xffffffffu, ok);
            // position of slot q = ib + (q / EPV) * STRIDE + q % EPV (32-bit: positions < 2^32)
            const u32 tb = (u32)((blockIdx.x + i * gridDim.x) * (u64)Cfg::TILE);
            ib = tb + threadIdx.x * EPV;
            if (ok) {
                const u32 te = tb + Cfg::TILE - 1;
                u32 le = 0;
                if (!((plx >= tb && plx <= te) || (prx >= tb && prx <= te))) {
                    // the tile holds neither pivot's position: ties with a
                    // pivot's key are decided by the side it lies on
                    raw_t rr[16];
                    load_raw_stage<DT>(stages + (size_t)stg * Cfg::BYTES, rr);
                    const bool ta = te < plx, tl = te <= prx;
                    const RawBound<DT> ba = RawBound<DT>::le((key_t)(plk - (ta ? 0 : 1)));
                    const RawBound<DT> bb = RawBound<DT>::le((key_t)(prk - (tl ? 0 : 1)));
                    tile_masks_dispatch<DT>(rr, ba, bb, ta || plk != 0, tl || prk != 0, ma, le);
                } else {
                    key_t kk[16];
                    InputSrc<DT>::template load16_smem<TMA_CONS>(
                        reinterpret_cast<const uint4*>(stages + (size_t)stg * Cfg::BYTES), kk);
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const ct c = C::make(kk[q], ib + (u32)((q / EPV) * STRIDE + q % EPV));
                        ma |= (u32)(c < pl) << q;
                        le |= (u32)(c <= pr) << q;
                    }
                }
                mb = le & ~ma;
            }
            const u32 wa = __reduce_add_sync(0xffffffffu, (u32)__popc(ma));
            const u32 wb = __reduce_add_sync(0xffffffffu, (u32)__popc(mb));
            if (lane == 0) {
                ds.wa[par][warp] = wa;
                ds.wb[par][warp] = wb;
            }
        }
        // the issuer of tile i-1 publishes its reservation before the barrier
        const u32 issuer_cur = par ? 32u : 0u, issuer_prev = ppar ? 32u : 0u;
        if (have_prev && threadIdx.x == issuer_prev) {
            ds.ba[ppar] = my_ra;
            ds.bb[ppar] = my_rb;
        }
        Sync::sync(); // counts of tile i, base of tile i-1 in; writes of tile i-2 done
        if (cur && threadIdx.x == issuer_cur) {
            u64 ta = 0, tb2 = 0;
            for (int w = 0; w < TMA_CONS / 32; ++w) {
                ds.oa[par][w] = ta;
                ds.ob[par][w] = tb2;
                ta += ds.wa[par][w];
                tb2 += ds.wb[par][w];
            }
            my_ra = 0;
            my_rb = 0;
            if (ta) my_ra = atomicAdd((unsigned long long*)sink.cnt_a, (unsigned long long)ta);
            if (tb2) my_rb = atomicAdd((unsigned long long*)sink.cnt_b, (unsigned long long)tb2);
        }
        if (have_prev && ok_prev) {
            // this thread's element of slot q sits at a constant offset from `mine`
            const unsigned char* mine = stages + (size_t)stg_prev * Cfg::BYTES + threadIdx.x * 16u;
            auto elem = [&](u32 q) -> raw_t {
                return *reinterpret_cast<const raw_t*>(mine + (q / EPV) * (TMA_CONS * 16u) + (q % EPV) * sizeof(raw_t));
            };
            if (__any_sync(0xffffffffu, ma_prev)) {
                const u64 xa = ds.ba[ppar] + ds.oa[ppar][warp];
                if (xa + ds.wa[ppar][warp] <= sink.cap_a) { // the usual case: no per-element bound
                    raw_t* okp = sink.out_keys + sink.out_base + xa;
                    u32* oip = sink.out_idx + sink.out_base + xa;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const bool bit = (ma_prev >> q) & 1u;
                        const u32 bal = __ballot_sync(0xffffffffu, bit);
                        // operands computed on every lane so that the stores
                        // are predicated rather than branched around; the run
                        // pointers advance by the slot's count
                        const u32 r = (u32)__popc(bal & below);
                        const raw_t key = elem(q);
                        const u32 idx = ib_prev + (u32)((q / EPV) * STRIDE + q % EPV);
                        if (bit) {
                            okp[r] = key;
                            oip[r] = idx;
                        }
                        const u32 c = (u32)__popc(bal);
                        okp += c;
                        oip += c;
                    }
                } else {
                    u64 ra = xa;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const bool bit = (ma_prev >> q) & 1u;
                        const u32 bal = __ballot_sync(0xffffffffu, bit);
                        if (bit)
                            sink.put_a_raw(ra + __popc(bal & below), elem(q),
                                           ib_prev + (u32)((q / EPV) * STRIDE + q % EPV));
                        ra += (u32)__popc(bal);
                    }
                }
            }
            if (__any_sync(0xffffffffu, mb_prev)) { // b is sparse: each lane writes its own
                const u32 cnt = (u32)__popc(mb_prev);
                u32 incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= (u32)o) incl += y;
                }
                u64 xb = ds.bb[ppar] + ds.ob[ppar][warp] + (incl - cnt);
                u32 m = mb_prev;
                while (m) {
                    const u32 q = (u32)(__ffs(m) - 1);
                    m &= m - 1;
                    sink.put_b(xb++, K::fwd(elem(q)), ib_prev + (q / EPV) * STRIDE + q % EPV);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[stg_prev]); // stage may be refilled
        }
        ma_prev = ma;
        mb_prev = mb;
        stg_prev = stg;
        ib_prev = ib;
        ok_prev = ok;
    }
    // the ragged last tile, read directly by the block that owns it
    const u64 nfull = s.m_src / Cfg::TILE;
    if (s.m_src % Cfg::TILE != 0 && nfull % gridDim.x == blockIdx.x) {
        key_t kk[16];
        u32 ii[16];
        const u64 tb = nfull * (u64)Cfg::TILE;
        const u32 valid = isrc.template load16<TMA_CONS>(tb, kk, ii);
        auto pos = [&](int q) -> u32 { return isrc.template idx_of<TMA_CONS>(tb, q); };
        classify_emit<TMA_CONS, true, false, Sync>(kk, pos, valid, (ct)0, pl, pr, sink, ps);
    }
}

template <int DT, bool DENSE>
__global__ void __launch_bounds__(TMA_NT, (TmaCfg<DT, DENSE>::MIN_BLOCKS)) k_pass_tma(SelArgs a) {
    typedef TmaCfg<DT, DENSE> Cfg;
    typedef typename Key<DT>::raw_t raw_t;
    constexpr int KW = Key<DT>::KW;
    extern __shared__ __align__(128) unsigned char stages[];
    __shared__ __align__(8) uint64_t full[Cfg::STAGES];
    __shared__ __align__(8) uint64_t empty[Cfg::STAGES];
    __shared__ PassSmem<TMA_CONS> ps;
    __shared__ WarpQ<KW> wq[DENSE ? 1 : TMA_CONS / 32];
    __shared__ DenseSmem ds;
    __shared__ u32 dead;
    grid_dep_wait();
    const SelState s = *a.st;
    if (s.phase != PH_RUN || !s.pending || s.src != SRC_INPUT || (s.dense != 0) != DENSE) {
        grid_dep_release(); // the variant not needed lets the next launch proceed at once
        return;
    }
    // the tile thresholds of the dense variant assume a window starting at the
    // smallest pair, which holds on first levels (the only ones this kernel runs)
    if (DENSE && Comp<KW>::from128(s.lo) != (typename Comp<KW>::t)0) {
        if (threadIdx.x == 0) latch(a.err, ST_EINTERNAL);
        return;
    }
    // the working variant keeps the next kernel's blocks off its SMs until it ends
    if (threadIdx.x == 0) {
        for (u32 i = 0; i < Cfg::STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], TMA_CONS / 32);
        }
        dead = 0;
        mbar_fence_init();
    }
    __syncthreads();
    const u64 nfull = s.m_src / Cfg::TILE;
    const u64 my_n = nfull > blockIdx.x ? (nfull - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    if (threadIdx.x >= TMA_CONS) { // producer warp: one lane issues the copies
        if (threadIdx.x == TMA_CONS) {
            const raw_t* keys = static_cast<const raw_t*>(a.keys);
            u32 stg = 0, epar = 1; // the first pass over the ring waits for nothing
            for (u64 i = 0; i < my_n; ++i) {
                if (i >= Cfg::STAGES) {
                    const u32 parity = epar;
                    if (*(volatile u32*)&dead || !mbar_wait_bounded(&empty[stg], parity, WAIT_LIMIT_NS)) {
                        *(volatile u32*)&dead = 1;
                        latch(a.err, ST_ETIMEOUT);
                        break;
                    }
                }
                const u64 t = blockIdx.x + i * gridDim.x;
                mbar_arrive_expect_tx(&full[stg], Cfg::BYTES);
                bulk_g2s(stages + (size_t)stg * Cfg::BYTES, keys + t * Cfg::TILE, Cfg::BYTES, &full[stg]);
                if (++stg == Cfg::STAGES) {
                    stg = 0;
                    epar ^= 1u;
                }
            }
        }
        return;
    }
    WarpQ<KW>& q = wq[DENSE ? 0 : threadIdx.x >> 5];
    if constexpr (!DENSE) tma_consume_sparse<DT>(a, s, stages, full, empty, my_n, &dead, q);
    else tma_consume_dense<DT>(a, s, stages, full, empty, my_n, &dead, ds, ps);
    SyncNamed<1, TMA_CONS>::sync();
    if (threadIdx.x == 0) pass_epilogue(a);
}

// ---- one-launch selection of a small input: the first level's steps in
// one cooperative kernel of one block per SM, separated by a bounded grid
// barrier, then the exact finish in block 0.  For inputs of up to SMALL_MAX
// keys the separate launches of the grid levels cost more than their work.
constexpr u64 SMALL_MAX = 1ull << 22;
constexpr int SMALL_NT = 512;
constexpr u64 GRID_BARRIER_NS = 200ull * 1000 * 1000;
template <int KW> using SmallSmem = BlockSmem<KW, SMALL_NT>;

// Every block of the grid arrives, then waits (at most `limit_ns`) until all
// have: words[0] counts arrivals and is reset by the last one, which then
// advances the generation words[1].  False after a timeout.
__device__ __forceinline__ bool grid_barrier(u32* words, u64 limit_ns) {
    __shared__ u32 s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile u32* gen = words + 1;
        const u32 g0 = *gen;
        __threadfence();
        bool ok = true;
        if (atomicAdd(words, 1u) == gridDim.x - 1) {
            atomicExch(words, 0u);
            __threadfence();
            atomicAdd(words + 1, 1u);
        } else {
            u64 t0, t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            while (*gen == g0) {
                __nanosleep(64);
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                if (t - t0 > limit_ns) {
                    ok = false;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <int DT> __global__ void __launch_bounds__(SMALL_NT, 1) k_small(SelArgs a) {
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    constexpr int KW = K::KW;
    typedef Comp<KW> C;
    typedef typename C::t ct;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<SmallSmem<KW>*>(smem_raw);
    SelState* g = a.st;
    const u32 tid = threadIdx.x;
    const u32 m = (u32)a.n;
    const InputSrc<DT> isrc = InputSrc<DT>::make(a.keys, a.n);
    // 1. the sample: draw j falls in partition j mod p (an equal share per
    //    partition) at a position uniform in it (Philox4x32-10 word j mod 4 of
    //    counter (j / 4, 0, salt, 0)); every draw lies in the first window
    const u32 s = a.sample;
    const u32 p = a.parts < m ? a.parts : m;
    const u32 len = m / p, rem = m - len * p;
    ct* samp = static_cast<ct*>(a.samp);
    for (u32 j = blockIdx.x * SMALL_NT + tid; j < s; j += gridDim.x * SMALL_NT) {
        const Philox4 r = philox4x32_10(j >> 2, 0, 0x53414D50u, 0, (u32)a.seed, (u32)(a.seed >> 32));
        const u32 part = j % p;
        const u32 plo = part * len + (part < rem ? part : rem);
        const u32 psz = len + (part < rem ? 1 : 0);
        const u32 pos = plo + (u32)(((u64)r.v[j & 3] * psz) >> 32);
        key_t kq;
        u32 x;
        isrc.at(pos, kq, x);
        samp[j] = C::make(kq, x);
    }
    if (blockIdx.x == 0 && tid == 0) {
        *g = initial_state<DT>(a);
        g->phase = PH_RUN;
    }
    if (!grid_barrier(a.gbar, GRID_BARRIER_NS)) {
        if (tid == 0) latch(a.err, ST_ETIMEOUT);
        return;
    }
    // 2. the pivots, in every block alike: the sample elements of ranks
    //    k|S|/n -/+ Delta (the same rule as the grid levels)
    {
        // the whole sample into shared memory, 16-byte loads, all in flight
        // (s * sizeof(ct) is a multiple of 16 bytes: s is at least 64)
        constexpr u32 PER = (Lim<KW>::ELEMS * sizeof(ct) / 16 + SMALL_NT - 1) / SMALL_NT;
        const uint4* src4 = reinterpret_cast<const uint4*>(samp);
        uint4* dst4 = reinterpret_cast<uint4*>(sm.samp);
        const u32 n4 = (u32)((s * sizeof(ct)) / 16);
        uint4 v[PER];
#pragma unroll
        for (u32 q = 0; q < PER; ++q) {
            const u32 i = q * SMALL_NT + tid;
            if (i < n4) v[q] = __ldcg(src4 + i);
        }
#pragma unroll
        for (u32 q = 0; q < PER; ++q) {
            const u32 i = q * SMALL_NT + tid;
            if (i < n4) dst4[i] = v[q];
        }
    }
    if (tid == 0) {
        long long jl, jr;
        pivot_ranks(s, a.n, a.k, a.z, (a.flags & TOPK_FLAG_RAW_DELTA) != 0, jl, jr);
        sm.jl = jl;
        sm.jr = jr;
    }
    __syncthreads();
    const ct lo = 0, hi = C::from128(key_domain_max<DT>());
    const long long jl = sm.jl, jr = sm.jr, top = (long long)s - 1;
    ct pl = lo, pr = hi;
    if (jl >= 0) pl = block_select_hist<KW, SMALL_NT>(sm.samp, s, lo, hi, (u32)(jl > top ? top : jl), sm.hs);
    if (jr <= top) pr = block_select_hist<KW, SMALL_NT>(sm.samp, s, lo, hi, (u32)(jr < 0 ? 0 : jr), sm.hs);
    // 3. the pass: a to the output, b to the candidate buffer
    {
        Sink<DT> sink;
        sink.out_keys = static_cast<raw_t*>(a.out_keys);
        sink.out_idx = a.out_idx;
        sink.out_base = 0;
        sink.cap_a = a.k;
        sink.ck = static_cast<key_t*>(a.cand_key[0]);
        sink.ci = a.cand_idx[0];
        sink.cap_b = a.cap_b;
        sink.cnt_a = &g->cnt_a;
        sink.cnt_b = &g->cnt_b;
        if (pl > lo) pass_tiles<SMALL_NT, true, false, DT>(isrc, blockIdx.x, gridDim.x, lo, pl, pr, sink, sm.ps);
        else pass_tiles<SMALL_NT, false, false, DT>(isrc, blockIdx.x, gridDim.x, lo, pl, pr, sink, sm.ps);
    }
    if (!grid_barrier(a.gbar, GRID_BARRIER_NS)) {
        if (tid == 0) latch(a.err, ST_ETIMEOUT);
        return;
    }
    // 4. block 0: the branch of Algorithm "select", then the finish
    if (blockIdx.x != 0) return;
    if (tid == 0) {
        g->pl = (u128)pl;
        g->pr = (u128)pr;
        g->dst = SRC_CAND0;
        g->pending = 1;
        g->level = 1;
        g->levels_grid = 1;
        g->sample_kept = s;
        g->cnt_a = *(volatile u64*)&g->cnt_a;
        g->cnt_b = *(volatile u64*)&g->cnt_b;
        decide(*g);
    }
    __syncthreads();
    block_levels_and_finish<DT, true, true>(a, sm);
}

// Remaining levels in one block, then the exact finish.
template <int DT> __global__ void __launch_bounds__(BLK_NT) k_finish(SelArgs a, int first) {
    grid_dep_wait();
    grid_dep_release();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<BlockSmem<Key<DT>::KW>*>(smem_raw);
    SelState* g = a.st;
    if (threadIdx.x == 0) {
        if (first) init_state<DT>(g, a);
        if (g->phase == PH_RUN) g->phase = PH_FINISH;
        sm.flag = g->phase == PH_FINISH;
    }
    __syncthreads();
    if (!sm.flag) return;
    block_levels_and_finish<DT, true, true>(a, sm);
}

// k = 1: the minimum pair (base case of Algorithm "select");
// k = n: every pair, plus the maximum as the rank-n pair.
template <int KW> __device__ __forceinline__ typename Comp<KW>::t shfl_xor_ct(typename Comp<KW>::t v, int o);
template <> __device__ __forceinline__ u64 shfl_xor_ct<32>(u64 v, int o) {
    return __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
}
template <> __device__ __forceinline__ u128 shfl_xor_ct<64>(u128 v, int o) {
    const u64 lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)(u64)v, o);
    const u64 hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(u64)(v >> 64), o);
    return ((u128)hi << 64) | lo;
}

template <int KW>
__device__ typename Comp<KW>::t block_extreme(typename Comp<KW>::t v, bool want_max, typename Comp<KW>::t* red) {
    typedef typename Comp<KW>::t ct;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const ct w = shfl_xor_ct<KW>(v, o);
        v = want_max ? (w > v ? w : v) : (w < v ? w : v);
    }
    const u32 warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane_id() == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        ct b = red[0];
        for (u32 w = 1; w < nw; ++w) b = want_max ? (red[w] > b ? red[w] : b) : (red[w] < b ? red[w] : b);
        red[0] = b;
    }
    __syncthreads();
    const ct out = red[0];
    __syncthreads();
    return out;
}

template <int DT>
__global__ void __launch_bounds__(EXT_NT) k_extreme(SelArgs a, int want_max, u32* counter, void* partials_v) {
    grid_dep_wait();
    grid_dep_release();
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    constexpr int KW = K::KW;
    typedef Comp<KW> C;
    typedef typename C::t ct;
    __shared__ ct red[EXT_NT / 32];
    __shared__ u32 is_last;
    ct* partials = static_cast<ct*>(partials_v);
    const InputSrc<DT> src = InputSrc<DT>::make(a.keys, a.n);
    const bool copy = want_max != 0; // k = n also copies every pair out
    raw_t* ok_out = static_cast<raw_t*>(a.out_keys);
    ct best = want_max ? (ct)0 : C::max_value();
    constexpr u64 TILE = (u64)EXT_NT * 16;
    const u64 ntiles = (a.n + TILE - 1) / TILE;
    for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
        typename K::key_t kk[16];
        u32 ii[16];
        const u32 valid = src.template load16<EXT_NT>(t * TILE, kk, ii);
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            if (!((valid >> s) & 1u)) continue;
            const ct c = C::make(kk[s], ii[s]);
            best = want_max ? (c > best ? c : best) : (c < best ? c : best);
            if (copy) {
                ok_out[ii[s]] = K::inv(kk[s]);
                a.out_idx[ii[s]] = ii[s];
            }
        }
    }
    best = block_extreme<KW>(best, want_max, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = best;
        __threadfence();
        const u32 prev = atomicAdd(counter, 1u);
        is_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    ct v = want_max ? (ct)0 : C::max_value();
    for (u32 i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
        const volatile ct* p = partials;
        const ct w = p[i];
        v = want_max ? (w > v ? w : v) : (w < v ? w : v);
    }
    v = block_extreme<KW>(v, want_max, red);
    if (threadIdx.x == 0) {
        static_cast<raw_t*>(a.kth_key)[0] = K::inv((typename K::key_t)C::key(v));
        a.kth_idx[0] = C::idx(v);
        if (!copy) {
            ok_out[0] = K::inv((typename K::key_t)C::key(v));
            a.out_idx[0] = C::idx(v);
        }
        SelState* g = a.st;
        init_state<DT>(g, a);
        g->phase = PH_DONE;
        g->out_base = a.k;
        atomicExch(counter, 0u);
    }
}

// ----------------------------------------------------------- host side

struct Tuning {
    u32 sample, parts, T, G;
    float z;
    u32 flags;
    u64 seed;
};

template <int KW> static Tuning make_tuning(const topk_params* prm, int sms) {
    constexpr u32 ELEMS = Lim<KW>::ELEMS;
    topk_params p{};
    if (prm) p = *prm;
    Tuning tu;
    tu.sample = p.sample_size ? std::min<u32>(std::max<u32>(p.sample_size, 64), ELEMS) : ELEMS;
    tu.parts = p.partitions ? p.partitions : (u32)sms;
    tu.T = p.finish_threshold ? std::min<u32>(std::max<u32>(p.finish_threshold, 64), ELEMS) : ELEMS;
    tu.G = tu.T; // grid levels run until the one-block finish can take over
    tu.z = p.delta_factor > 0.f ? p.delta_factor : 4.0f;
    tu.flags = p.flags;
    tu.seed = p.seed ? p.seed : 0x243F6A8885A308D3ull;
    return tu;
}

static SelArgs make_args(const void* keys, u64 n, u64 k, void* out_keys, u32* out_idx, void* kth_key,
                         u32* kth_idx, const Tuning& tu) {
    SelArgs a{};
    a.keys = keys;
    a.n = n;
    a.k = k;
    a.out_keys = out_keys;
    a.out_idx = out_idx;
    a.kth_key = kth_key;
    a.kth_idx = kth_idx;
    a.seed = tu.seed;
    a.parts = tu.parts;
    a.sample = tu.sample;
    a.finish_T = tu.T;
    a.grid_G = tu.G;
    a.z = tu.z;
    a.flags = tu.flags;
    a.aligned = (reinterpret_cast<uintptr_t>(keys) & 15u) == 0;
    return a;
}

// Host copy of the device pivot-rank rule, for sizing buffers and predicting
// the number of grid levels.
static double est_bracket(u64 m, u64 k_rem, u32 s, float z) {
    const double kept = (double)std::min<u64>(s, m);
    const double mu_le = kept * (double)k_rem / (double)m;
    const double mu_lt = kept * (double)(k_rem - 1) / (double)m;
    const double v = std::max(0.0, mu_le * (1.0 - mu_le / kept));
    const double d = z * std::sqrt(v) + z * z / 3.0 + 1.0;
    const double jl = std::max(-1.0, std::floor(mu_le - d) - 1.0);
    const double jr = std::min(kept, std::ceil(mu_lt + d));
    return std::min((double)m, (jr - jl + 1.0) * (double)m / kept);
}

// Kernel attributes, set once per device.
template <int DT> static topk_status set_smem_attrs() {
    static std::atomic<uint64_t> done_mask{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TOPK_ECUDA;
    const uint64_t bit = 1ull << (dev & 63);
    if (done_mask.load() & bit) return TOPK_OK;
    if (cudaFuncSetAttribute(k_pass_tma<DT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TmaCfg<DT, false>::SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k_pass_tma<DT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TmaCfg<DT, true>::SMEM) != cudaSuccess)
        return TOPK_ECUDA;
    const int bytes = (int)sizeof(BlockSmem<Key<DT>::KW>);
    if (cudaFuncSetAttribute(k_pivots<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(PivotSmem<Key<DT>::KW>)) != cudaSuccess)
        return TOPK_ECUDA;
    if (cudaFuncSetAttribute(k_finish<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
        cudaFuncSetAttribute(k_small<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(SmallSmem<Key<DT>::KW>)) != cudaSuccess)
        return TOPK_ECUDA;
    done_mask.fetch_or(bit);
    return TOPK_OK;
}

// Resident blocks per SM of each pass variant: the grid is one full wave.
template <int DT, bool DENSE> static int tma_grid(int sms) {
    static int occ = 0;
    if (occ == 0) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_pass_tma<DT, DENSE>, TMA_NT,
                                                          TmaCfg<DT, DENSE>::SMEM) != cudaSuccess)
            o = 1;
        occ = std::max(1, o);
    }
    return sms * occ;
}

template <int DT> static int pass_grid(int sms, bool first) {
    static int occ_first = 0, occ_rest = 0;
    if (occ_first == 0) {
        int o1 = 0, o2 = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_pass_first<DT>, PASS_NT, 0) != cudaSuccess) o1 = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_pass<DT>, PASS_NT, 0) != cudaSuccess) o2 = 1;
        occ_rest = std::max(1, o2);
        occ_first = std::max(1, o1);
    }
    return sms * (first ? occ_first : occ_rest);
}

// Whether one block of k_small fits on every SM (the cooperative launch
// needs the whole grid resident).
template <int DT> static bool small_fits(int sms) {
    static int occ = -1;
    if (occ < 0) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_small<DT>, SMALL_NT, sizeof(SmallSmem<Key<DT>::KW>)) !=
            cudaSuccess) {
            cudaGetLastError();
            o = 0;
        }
        occ = o;
    }
    (void)sms;
    return occ >= 1;
}

// Candidate capacity for a first level over n keys: twice the expected
// bracket, at least the finisher's range.
static u64 candidate_capacity(u64 n, u64 k, const Tuning& tu) {
    u64 cap = (u64)(2.0 * est_bracket(n, k, tu.sample, tu.z)) + 4ull * tu.T;
    if (tu.flags & TOPK_FLAG_TINY_CAND) cap = tu.T;
    cap = std::max<u64>(cap, tu.T);
    cap = std::min<u64>(cap, std::max<u64>(n, tu.T));
    return (cap + 4095) & ~(u64)4095;
}

// Enqueues one selection whose state, error word and buffers `a` already
// points to.  k = 1 and k = n need `counter` (zero) and `partials`
// (EXT grid composites).  `ctx` (may be null) receives the measurement hooks.
template <int DT>
static topk_status enqueue_select(topk_ctx* ctx, SelArgs a, const Tuning& tu, int sms, u32* counter,
                                  void* partials, cudaStream_t st) {
    constexpr int KW = Key<DT>::KW;
    const u64 n = a.n, k = a.k;
    if (k == 1 || k == n) {
        if (ctx) profile_pass_begin(ctx, st);
        const cudaError_t e = launch_dep(k_extreme<DT>, sms * EXT_BLOCKS_PER_SM, EXT_NT, 0, st, a,
                                         k == n && n > 1 ? 1 : 0, counter, partials);
        if (e != cudaSuccess) return cuda_status(e);
        if (ctx) {
            profile_pass_end(ctx, st);
            count_launch(ctx);
        }
        return cuda_status(cudaGetLastError());
    }
    topk_status rs = set_smem_attrs<DT>();
    if (rs != TOPK_OK) return rs;
    // the first level's expected bracket fits the finishing block
    if (n <= SMALL_MAX && n > tu.G && a.gbar != nullptr && (!ctx || ctx->one_launch) && small_fits<DT>(sms) &&
        1.2 * est_bracket(n, k, tu.sample, tu.z) <= (double)tu.T) {
        // one launch: sample, pivots, pass and finish (cooperative, one block per SM)
        if (ctx) profile_pass_begin(ctx, st);
        cudaError_t e = cudaMemsetAsync(a.gbar, 0, 2 * sizeof(u32), st);
        if (e == cudaSuccess) e = launch_coop(k_small<DT>, sms, SMALL_NT, sizeof(SmallSmem<KW>), st, a);
        if (e != cudaSuccess) return cuda_status(e);
        if (ctx) {
            profile_pass_end(ctx, st);
            count_launch(ctx);
        }
        return cuda_status(cudaGetLastError());
    }
    // grid levels until the candidates fit the block finisher's range
    int levels = 0;
    {
        double m = (double)n, kr = (double)k;
        while (m > tu.G && levels < 8) {
            m = 1.2 * est_bracket((u64)m, (u64)std::max(1.0, std::min(kr, m)), tu.sample, tu.z);
            kr = m / 2;
            ++levels;
        }
    }
    const size_t smem = sizeof(BlockSmem<KW>);
    const int smp_blocks = (int)((tu.sample * SMP_MAX_SCALE + SMP_NT * SMP_DRAWS - 1) / (SMP_NT * SMP_DRAWS));
    for (int l = 0; l < levels; ++l) {
        cudaError_t e = launch_dep(k_sample<DT>, smp_blocks, SMP_NT, 0, st, a, l == 0 ? 1 : 0);
        if (e == cudaSuccess) e = launch_dep(k_pivots<DT>, 1, PIV_NT, sizeof(PivotSmem<KW>), st, a, l == 0 ? 1 : 0);
        if (e != cudaSuccess) return cuda_status(e);
        if (l == 0 && ctx) profile_pass_begin(ctx, st);
        if (l == 0 && a.aligned && !(tu.flags & TOPK_FLAG_NO_BULK_COPY)) {
            // the mode is chosen on the device: the variant that does not match returns at once
            e = launch_dep(k_pass_tma<DT, false>, tma_grid<DT, false>(sms), TMA_NT, TmaCfg<DT, false>::SMEM, st, a);
            if (e == cudaSuccess)
                e = launch_dep(k_pass_tma<DT, true>, tma_grid<DT, true>(sms), TMA_NT, TmaCfg<DT, true>::SMEM, st, a);
        }
        else if (l == 0) e = launch_dep(k_pass_first<DT>, pass_grid<DT>(sms, true), PASS_NT, 0, st, a);
        else e = launch_dep(k_pass<DT>, pass_grid<DT>(sms, false), PASS_NT, 0, st, a);
        if (e != cudaSuccess) return cuda_status(e);
        if (l == 0 && ctx) profile_pass_end(ctx, st);
    }
    const cudaError_t e = launch_dep(k_finish<DT>, 1, BLK_NT, smem, st, a, levels == 0 ? 1 : 0);
    if (e != cudaSuccess) return cuda_status(e);
    if (ctx) count_launch(ctx, 3 * (uint64_t)levels + 1 + (levels > 0 && a.aligned ? 1 : 0));
    return cuda_status(cudaGetLastError());
}

// Scratch regions of one selection: reduction partials, the sample, and the
// two candidate buffers (keys, then positions) of `cap` pairs each.
struct SelectCarve {
    size_t part, samp, k0, k1, i0, i1;
};
template <int KW> static Carve select_carve(u64 cap, int sms, SelectCarve& sc) {
    const size_t kbytes = KW / 8;
    Carve cv;
    sc.part = cv.take(sizeof(typename Comp<KW>::t) * (size_t)sms * EXT_BLOCKS_PER_SM);
    sc.samp = cv.take(sizeof(typename Comp<KW>::t) * (size_t)Lim<KW>::ELEMS);
    sc.k0 = cv.take(cap * kbytes);
    sc.k1 = cv.take(cap * kbytes);
    sc.i0 = cv.take(cap * 4);
    sc.i1 = cv.take(cap * 4);
    return cv;
}

template <int DT>
topk_status run_select(topk_ctx* ctx, const void* keys, u64 n, u64 k, void* out_keys, u32* out_idx,
                              void* kth_key, u32* kth_idx, const topk_params* prm, cudaStream_t st) {
    constexpr int KW = Key<DT>::KW;
    const Tuning tu = make_tuning<KW>(prm, ctx->sms);
    SelArgs a = make_args(keys, n, k, out_keys, out_idx, kth_key, kth_idx, tu);
    a.st = static_cast<SelState*>(ctx->d_state);
    a.err = ctx->d_err;
    ctx->last_kind = LAST_SELECT;

    const u64 cap = (k == 1 || k == n) ? 0 : candidate_capacity(n, k, tu);
    a.cap_b = cap;
    SelectCarve sc;
    const Carve cv = select_carve<KW>(cap, ctx->sms, sc);
    const size_t off_part = sc.part, off_samp = sc.samp, off_k0 = sc.k0, off_k1 = sc.k1, off_i0 = sc.i0,
                 off_i1 = sc.i1;
    topk_status rs = ensure_scratch(ctx, cv.off);
    if (rs != TOPK_OK) return rs;
    char* base = static_cast<char*>(ctx->scratch.base);
    a.samp = base + off_samp;
    a.samp_cap = Lim<KW>::ELEMS;
    a.samp_count = ctx->d_counter + 3;
    a.pass_done = ctx->d_counter + 2;
    a.gbar = ctx->d_counter + 8;
    a.hist = ctx->d_hist;
    a.cand_key[0] = base + off_k0;
    a.cand_key[1] = base + off_k1;
    a.cand_idx[0] = reinterpret_cast<u32*>(base + off_i0);
    a.cand_idx[1] = reinterpret_cast<u32*>(base + off_i1);
    return enqueue_select<DT>(ctx, a, tu, ctx->sms, ctx->d_counter, base + off_part, st);
}

// ------------------------------------------ entry point without allocation
// topk_select_noalloc runs the same kernels as topk_select, with every piece
// of scratch (state, error word, block-done counter, reduction partials and
// the two candidate buffers) in one file-scope device array instead of a
// context's cudaMalloc'd block.  The array lives in every GPU that loads the
// library until the process exits.  Host code must not pass the array's name
// to a kernel (in host code it is only a stand-in for the symbol); its device
// address is looked up once per device with cudaGetSymbolAddress.

constexpr u64 NOALLOC_MAX_N = 1ull << 22;  // largest n accepted (4 Mi keys)
// Candidate pairs per buffer.  The context path sizes its buffers as
// candidate_capacity(n, k): twice the expected first bracket plus 4 T, which
// is largest at k = n/2 and, for n = 2^22 with the default tuning, is about
// 3.4e5 pairs for 32-bit keys (s = 16384) and 4.2e5 for 64-bit keys
// (s = 8192).  2^19 covers both, so no accepted call overflows more often
// than the same call through a context; the set-up checks this relation.
constexpr u64 NOALLOC_CAP = 1ull << 19;
constexpr size_t NA_OFF_STATE = 0;         // SelState
constexpr size_t NA_OFF_WORDS = 4096;      // [0] error, [1] reduction done, [2] pass done, [3] sample count
constexpr size_t NA_OFF_HIST = 8192;       // HIST_BINS u32
constexpr size_t NA_OFF_PART = NA_OFF_HIST + HIST_BINS * 4; // per-block composites of the k = 1 / k = n reduction
constexpr size_t NA_PART_BYTES = 64 * 1024;
constexpr size_t NA_OFF_SAMP = NA_OFF_PART + NA_PART_BYTES; // sample, Lim<32>::ELEMS * 8 = Lim<64>::ELEMS * 16 bytes
constexpr size_t NA_SAMP_BYTES = 128 * 1024;
constexpr size_t NA_OFF_CAND = NA_OFF_SAMP + NA_SAMP_BYTES;
constexpr size_t NA_BYTES = NA_OFF_CAND + 2 * NOALLOC_CAP * (8 + 4); // about 12.2 MiB

// Kernel attributes and the launch-geometry queries of every key type, so
// that no later call on this device makes them (they are made once per
// process and key type otherwise, on the first call with 1 < k < n).
template <int DT> topk_status noalloc_prepare_dt(int sms) {
    topk_status rs = set_smem_attrs<DT>();
    if (rs != TOPK_OK) return rs;
    (void)tma_grid<DT, false>(sms);
    (void)tma_grid<DT, true>(sms);
    (void)pass_grid<DT>(sms, true);
    (void)small_fits<DT>(sms);
    return cudaGetLastError() == cudaSuccess ? TOPK_OK : TOPK_ECUDA;
}

template <int DT>
topk_status run_select_noalloc(char* base, int sms, const void* keys, u64 n, u64 k, void* out_keys,
                                      u32* out_idx, void* kth_key, u32* kth_idx, u32* d_status,
                                      cudaStream_t st) {
    constexpr int KW = Key<DT>::KW;
    static_assert(sizeof(SelState) <= NA_OFF_WORDS, "state region too small");
    if ((size_t)sms * EXT_BLOCKS_PER_SM * sizeof(typename Comp<KW>::t) > NA_PART_BYTES) return TOPK_EINVAL;
    const Tuning tu = make_tuning<KW>(nullptr, sms);
    SelArgs a = make_args(keys, n, k, out_keys, out_idx, kth_key, kth_idx, tu);
    u32* words = reinterpret_cast<u32*>(base + NA_OFF_WORDS);
    a.st = reinterpret_cast<SelState*>(base + NA_OFF_STATE);
    a.err = d_status ? d_status : words;
    a.cap_b = NOALLOC_CAP;
    char* cand = base + NA_OFF_CAND;
    a.cand_key[0] = cand;
    a.cand_key[1] = cand + NOALLOC_CAP * 8;
    a.cand_idx[0] = reinterpret_cast<u32*>(cand + 2 * NOALLOC_CAP * 8);
    a.cand_idx[1] = reinterpret_cast<u32*>(cand + 2 * NOALLOC_CAP * 8 + NOALLOC_CAP * 4);
    static_assert(sizeof(typename Comp<KW>::t) * Lim<KW>::ELEMS <= NA_SAMP_BYTES, "sample region too small");
    a.samp = base + NA_OFF_SAMP;
    a.samp_cap = Lim<KW>::ELEMS;
    a.pass_done = words + 2;
    a.samp_count = words + 3;
    a.gbar = words + 8;
    a.hist = reinterpret_cast<u32*>(base + NA_OFF_HIST);
    // the error word, the block-done counters, the sample count and the
    // histogram must start at zero (a call that failed may have left them set)
    if (cudaMemsetAsync(words, 0, 4 * sizeof(u32), st) != cudaSuccess) return TOPK_ECUDA;
    if (cudaMemsetAsync(a.hist, 0, HIST_BINS * sizeof(u32), st) != cudaSuccess) return TOPK_ECUDA;
    if (d_status && cudaMemsetAsync(d_status, 0, sizeof(u32), st) != cudaSuccess) return TOPK_ECUDA;
    return enqueue_select<DT>(nullptr, a, tu, sms, words + 1, base + NA_OFF_PART, st);
}

// Explicit instantiation (one translation unit per key type) and the
// matching declarations for the translation unit of the C entry points.
#define TOPK_SELECT_TEMPLATES(PREFIX, DT)                                                                  \
    PREFIX template topk_status run_select<DT>(topk_ctx*, const void*, u64, u64, void*, u32*, void*, u32*,    \
                                               const topk_params*, cudaStream_t);                            \
    PREFIX template topk_status run_select<DT_DESC + DT>(topk_ctx*, const void*, u64, u64, void*, u32*, void*, \
                                                         u32*, const topk_params*, cudaStream_t);            \
    PREFIX template topk_status run_select_noalloc<DT>(char*, int, const void*, u64, u64, void*, u32*, void*,  \
                                                       u32*, u32*, cudaStream_t);                            \
    PREFIX template topk_status noalloc_prepare_dt<DT>(int);

} // namespace topk
