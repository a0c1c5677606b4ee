// select_block.cuh — one thread block runs whole recursion levels of the
// selection: planning (sample + pivots), a block-wide pass, the branch, and
// the final exact selection among at most T candidates.  Used by the
// single-selection finish (select_impl.cuh: k_finish) and by the batched
// kernels (batched.cu), where every block selects whole rows.
#pragma once

#include "select_core.cuh"

namespace topk {

constexpr int BLK_NT = 1024;  // planning / finishing block
constexpr int PASS_NT = 256;  // grid pass block
constexpr int EXT_NT = 256;   // min / max reduction block
constexpr int EXT_BLOCKS_PER_SM = 4;
constexpr u32 MAX_BLOCK_LEVELS = 256;

template <int KW> struct Lim {
    // sample and finish capacity of one block (128 KiB of composites)
    static constexpr u32 ELEMS = KW == 32 ? 16384u : 8192u;
};

// Shared memory of a block that runs whole levels: NT threads, room for CAP
// composites (the sample, then the finisher's candidates; CAP >= T).
template <int KW, int NT = BLK_NT, u32 CAP = Lim<KW>::ELEMS> struct BlockSmem {
    typedef typename Comp<KW>::t ct;
    static constexpr int THREADS = NT;
    static constexpr u32 ELEMS = CAP;
    ct samp[CAP];
    HistSelSmem<KW> hs;
    PassSmem<NT> ps;
    u32 kept;
    u32 flag;
    long long jl, jr;
};

__device__ inline void latch(u32* err, u32 code) { atomicCAS(err, 0u, code); }

// All 32 lanes call with their element counts; returns this lane's first
// slot of a contiguous run reserved for the warp with one atomic.
__device__ __forceinline__ u32 warp_reserve(u32 cnt, u32* counter) {
    u32 incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane_id() >= (u32)o) incl += y;
    }
    const u32 tot = __shfl_sync(0xffffffffu, incl, 31);
    u32 base = 0;
    if (lane_id() == 31 && tot) base = atomicAdd(counter, tot);
    return __shfl_sync(0xffffffffu, base, 31) + incl - cnt;
}

// All 32 lanes call; returns the slot of this lane's element when `keep`.
__device__ __forceinline__ u32 warp_append(bool keep, u32* counter) {
    const u32 bal = __ballot_sync(0xffffffffu, keep);
    u32 base = 0;
    if (lane_id() == 0 && bal) base = atomicAdd(counter, (u32)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    return base + __popc(bal & lanemask_lt());
}

// The state of a call before its first level.
template <int DT> __device__ SelState initial_state(const SelArgs& a) {
    SelState s;
    s.lo = 0;
    s.hi = key_domain_max<DT>();
    s.pl = 0;
    s.pr = 0;
    s.m_src = a.n;
    s.m_win = a.n;
    s.k_rem = a.k;
    s.out_base = 0;
    s.cnt_a = 0;
    s.cnt_b = 0;
    s.cap_b = a.cap_b;
    s.first_cand = 0;
    s.level = 0;
    s.phase = PH_RUN;
    s.src = SRC_INPUT;
    s.dst = SRC_CAND0;
    s.pending = 0;
    s.status = ST_OK;
    s.levels_grid = 0;
    s.levels_block = 0;
    s.failures = 0;
    s.overflows = 0;
    s.sample_kept = 0;
    s.dense = 0;
    return s;
}
template <int DT> __device__ void init_state(SelState* g, const SelArgs& a) { *g = initial_state<DT>(a); }

// ------------------------------------------------------------ one pass

// One pass over the source of state `s` (tiles tile0, tile0 + step, ...):
// a to the output, b to candidate buffer s.dst, the counts reserved on
// *cnt_a and *cnt_b.
template <int NT, int DT, bool INPUT_ONLY = false, bool ONLY_EXACT = false>
__device__ void run_pass_to(const SelArgs& a, const SelState& s, u64 tile0, u64 step, PassSmem<NT>& ps, u64* cnt_a,
                            u64* cnt_b) {
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    constexpr int KW = K::KW;
    typedef Comp<KW> C;
    typedef typename C::t ct;
    Sink<DT> sink;
    sink.out_keys = static_cast<raw_t*>(a.out_keys);
    sink.out_idx = a.out_idx;
    sink.out_base = s.out_base;
    sink.cap_a = s.k_rem;
    sink.ck = static_cast<key_t*>(a.cand_key[s.dst - 1]);
    sink.ci = a.cand_idx[s.dst - 1];
    sink.cap_b = a.cap_b;
    sink.cnt_a = cnt_a;
    sink.cnt_b = cnt_b;
    const ct lo = C::from128(s.lo), pl = C::from128(s.pl), pr = C::from128(s.pr);
    const bool has_a = pl > lo, exact = ONLY_EXACT || lo != (ct)0;
    if (INPUT_ONLY || s.src == SRC_INPUT) {
        const InputSrc<DT> src = InputSrc<DT>::make(a.keys, s.m_src);
        if (exact) pass_tiles<NT, true, true, DT>(src, tile0, step, lo, pl, pr, sink, ps);
        else if constexpr (!ONLY_EXACT) {
            if (has_a) pass_tiles<NT, true, false, DT>(src, tile0, step, lo, pl, pr, sink, ps);
            else pass_tiles<NT, false, false, DT>(src, tile0, step, lo, pl, pr, sink, ps);
        }
    } else if constexpr (!INPUT_ONLY) {
        CandSrc<KW> src{static_cast<const key_t*>(a.cand_key[s.src - 1]), a.cand_idx[s.src - 1], s.m_src};
        if (exact) pass_tiles<NT, true, true, DT>(src, tile0, step, lo, pl, pr, sink, ps);
        else if constexpr (!ONLY_EXACT) {
            if (has_a) pass_tiles<NT, true, false, DT>(src, tile0, step, lo, pl, pr, sink, ps);
            else pass_tiles<NT, false, false, DT>(src, tile0, step, lo, pl, pr, sink, ps);
        }
    }
}

template <int NT, int DT, bool INPUT_ONLY = false, bool ONLY_EXACT = false>
__device__ __forceinline__ void run_pass(const SelArgs& a, const SelState& s, u64 tile0, u64 step,
                                         PassSmem<NT>& ps) {
    run_pass_to<NT, DT, INPUT_ONLY, ONLY_EXACT>(a, s, tile0, step, ps, &a.st->cnt_a, &a.st->cnt_b);
}

// ------------------------------------------------------- pickPivots
// Samples the window, reads the pivots off the sample and arms the next pass.

template <int DT, class SM> __device__ void plan_level(const SelArgs& a, SM& sm, bool grid_level) {
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    constexpr int KW = K::KW;
    typedef Comp<KW> C;
    typedef typename C::t ct;
    SelState* g = a.st;
    const SelState s = *g;
    const ct lo = C::from128(s.lo), hi = C::from128(s.hi);
    ct pl = lo, pr = hi; // "collect": every window element becomes a candidate
    u32 kept = 0;
    if (s.m_win > a.finish_T) {
        u32 draws = grid_level ? a.sample : (u32)min((u64)a.sample, max((u64)1024, s.m_src / 4));
        if (s.m_win < s.m_src) { // narrowed window: draw more so enough land inside
            u64 ratio = s.m_src / (s.m_win ? s.m_win : 1);
            ratio = ratio < 2 ? 2 : ratio > 64 ? 64 : ratio;
            draws = (u32)min((u64)draws * ratio / 2, (u64)a.sample * 32);
        }
        if (s.src == SRC_INPUT) {
            const InputSrc<DT> src = InputSrc<DT>::make(a.keys, s.m_src);
            kept = block_sample(src, lo, hi, draws, a.parts, a.seed, s.level, 0, sm.samp, SM::ELEMS, &sm.kept);
        } else {
            CandSrc<KW> src{static_cast<const key_t*>(a.cand_key[s.src - 1]), a.cand_idx[s.src - 1], s.m_src};
            kept = block_sample(src, lo, hi, draws, a.parts, a.seed, s.level, 0, sm.samp, SM::ELEMS, &sm.kept);
        }
        if (kept > 0) {
            // pivot ranks once (the block shares them)
            if (threadIdx.x == 0) {
                long long l, r;
                pivot_ranks(kept, s.m_win, s.k_rem, a.z, (a.flags & TOPK_FLAG_RAW_DELTA) != 0, l, r);
                sm.jl = l;
                sm.jr = r;
            }
            __syncthreads();
            const long long jl = sm.jl, jr = sm.jr;
            const long long top = (long long)kept - 1;
            const u32 r0 = (u32)(jl < 0 ? 0 : jl > top ? top : jl), r1 = (u32)(jr < 0 ? 0 : jr > top ? top : jr);
            ct x0, x1;
            block_select_two<KW, SM::THREADS>(sm.samp, kept, lo, hi, r0, r1, sm.hs, x0, x1);
            if (jl >= 0) pl = x0;
            if (jr <= top) pr = x1;
        }
    }
    if (threadIdx.x == 0) {
        g->pl = (u128)pl;
        g->pr = (u128)pr;
        g->dst = s.src == SRC_CAND0 ? SRC_CAND1 : SRC_CAND0;
        g->cnt_a = 0;
        g->cnt_b = 0;
        g->pending = 1;
        g->level = s.level + 1;
        if (grid_level) g->levels_grid++;
        else g->levels_block++;
        if (s.level == 0) g->sample_kept = kept;
    }
    __syncthreads();
}

// ------------------------------------------------- finish in one block
// At most T undecided elements remain in the source: gather them, select the
// one of rank k_rem, emit every element not above it.

template <int DT, class SM> __device__ void block_finish(const SelArgs& a, SM& sm) {
    constexpr int NT = SM::THREADS;
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    constexpr int KW = K::KW;
    typedef Comp<KW> C;
    typedef typename C::t ct;
    SelState* g = a.st;
    const SelState s = *g;
    const ct lo = C::from128(s.lo), hi = C::from128(s.hi);
    if (threadIdx.x == 0) sm.kept = 0;
    __syncthreads();
    const InputSrc<DT> isrc = InputSrc<DT>::make(a.keys, s.m_src);
    const CandSrc<KW> csrc{static_cast<const key_t*>(a.cand_key[s.src == SRC_CAND1 ? 1 : 0]),
                           a.cand_idx[s.src == SRC_CAND1 ? 1 : 0], s.m_src};
    constexpr int U = 8; // loads in flight per thread; one slot reservation per warp for all of them
    for (u64 base = 0; base < s.m_src; base += (u64)NT * U) {
        ct cv[U];
        u32 keepm = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const u64 i = base + (u64)u * NT + threadIdx.x;
            key_t kv = 0;
            u32 x = 0;
            if (i < s.m_src) {
                if (s.src == SRC_INPUT) isrc.at(i, kv, x);
                else csrc.at(i, kv, x);
            }
            cv[u] = C::make(kv, x);
            keepm |= (u32)(i < s.m_src && cv[u] >= lo && cv[u] <= hi) << u;
        }
        u32 slot = warp_reserve((u32)__popc(keepm), &sm.kept);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if ((keepm >> u) & 1u) {
                if (slot < SM::ELEMS) sm.samp[slot] = cv[u];
                ++slot;
            }
        }
    }
    __syncthreads();
    const u32 count = sm.kept;
    if (count != s.m_win || s.k_rem == 0 || s.k_rem > count || count > SM::ELEMS) {
        if (threadIdx.x == 0) {
            g->status = ST_EINTERNAL;
            g->phase = PH_ERROR;
            latch(a.err, ST_EINTERNAL);
        }
        return;
    }
    const ct kth = block_select_hist<KW, NT>(sm.samp, count, lo, hi, (u32)(s.k_rem - 1), sm.hs);
    if (threadIdx.x == 0) sm.kept = 0;
    __syncthreads();
    raw_t* ok_out = static_cast<raw_t*>(a.out_keys);
    for (u32 base = 0; base < count; base += NT * U) {
        u32 selm = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const u32 i = base + u * NT + threadIdx.x;
            selm |= (u32)(i < count && sm.samp[i] <= kth) << u;
        }
        u32 slot = warp_reserve((u32)__popc(selm), &sm.kept);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if ((selm >> u) & 1u) {
                const ct c = sm.samp[base + u * NT + threadIdx.x];
                ok_out[s.out_base + slot] = K::inv((key_t)C::key(c));
                a.out_idx[s.out_base + slot] = C::idx(c);
                ++slot;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        static_cast<raw_t*>(a.kth_key)[0] = K::inv((key_t)C::key(kth));
        a.kth_idx[0] = C::idx(kth);
        if (sm.kept != s.k_rem) {
            g->status = ST_EINTERNAL;
            g->phase = PH_ERROR;
            latch(a.err, ST_EINTERNAL);
        } else {
            g->out_base = s.out_base + s.k_rem;
            g->phase = PH_DONE;
        }
    }
}


// One recursion level run by this block alone: plan, pass, branch.
template <int DT, bool ONLY_EXACT, class SM>
__device__ __forceinline__ void block_level(const SelArgs& a, SM& sm) {
    SelState* g = a.st;
    plan_level<DT>(a, sm, false);
    {
        const SelState s = *g;
        run_pass<SM::THREADS, DT, false, ONLY_EXACT>(a, s, 0, 1, sm.ps);
    }
    __syncthreads();
    if (threadIdx.x == 0) decide(*g);
    __syncthreads();
}

// The same, out of line: its register demand then does not weigh on a
// caller that seldom needs it.
template <int DT, bool ONLY_EXACT, class SM>
__device__ __noinline__ void block_level_outlined(const SelArgs& a, SM& sm) {
    block_level<DT, ONLY_EXACT>(a, sm);
}

// Recursion levels run by this block alone until at most T elements remain in
// the source, then the exact finish.  Precondition: no pass pending.
// OUTLINED keeps the level code out of line (for callers whose source is
// usually at most T already).
template <int DT, bool ONLY_EXACT, bool OUTLINED = false, class SM>
__device__ void block_levels_and_finish(const SelArgs& a, SM& sm) {
    SelState* g = a.st;
    for (u32 it = 0; it < MAX_BLOCK_LEVELS; ++it) {
        if (g->m_src <= a.finish_T) {
            block_finish<DT>(a, sm);
            return;
        }
        if (OUTLINED) block_level_outlined<DT, ONLY_EXACT>(a, sm);
        else block_level<DT, ONLY_EXACT>(a, sm);
    }
    if (threadIdx.x == 0) {
        g->status = ST_EINTERNAL;
        g->phase = PH_ERROR;
        latch(a.err, ST_EINTERNAL);
    }
}

} // namespace topk
