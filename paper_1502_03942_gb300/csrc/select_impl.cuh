// select_impl.cuh — topk_select: selection of the k smallest of n unsorted keys
// (paper, Section 2, Algorithm "select"; Section 4.1, Theorem "selectFR").
//
// Launch sequence of one call (all on the caller's stream, no host round
// trip), per recursion level:
//   k_sample (grid)     per-partition draws of the current window -> sample
//                       array (draw j at slot j)
//   k_pivots (1 block)  pivots = sample elements of ranks k|S|/n -/+ Delta:
//                       the sample into shared memory, one histogram over
//                       its range, the two rank bins ranked exactly
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

// ---- pickPivots: the sample (k_sample, whole grid) and the pivots
// (k_pivots, one block), defined with the sampling routines further down.
constexpr int SMP_NT = 128;
constexpr int SMP_DRAWS = 4;        // one Philox block per thread
constexpr u32 SMP_MAX_SCALE = 4;    // extra draws for a narrowed window
constexpr int PIV_NT = 1024;

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
    LQState qs = LQState::make();
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
        // the hits' keys come from the stage, which is released after them
        const unsigned char* mine = stages + (size_t)stg * Cfg::BYTES + threadIdx.x * 16u;
        lq_append<DT>(hit, pos, [&](u32 sq) {
            return K::fwd(*reinterpret_cast<const raw_t*>(mine + (sq / EPV) * (TMA_CONS * 16u) + (sq % EPV) * sizeof(raw_t)));
        }, lo, pl, pr, sink, wq, qs);
        __syncwarp();
        if (ok && lane == 0) mbar_arrive(&empty[stg]); // the stage may be refilled
    }
    // the ragged last tile, read directly by the block that owns it
    const u64 nfull = s.m_src / Cfg::TILE;
    if (s.m_src % Cfg::TILE != 0 && nfull % gridDim.x == blockIdx.x) {
        key_t kk[16];
        u32 ii[16];
        const u64 tb = nfull * (u64)Cfg::TILE;
        const u32 valid = isrc.template load16<TMA_CONS>(tb, kk, ii);
        auto pos = [&](int q) -> u32 { return isrc.template idx_of<TMA_CONS>(tb, q); };
        u32 tail_hit = 0;
#pragma unroll
        for (int q = 0; q < 16; ++q) tail_hit |= (u32)(C::make(kk[q], pos(q)) <= pr) << q;
        lq_append<DT>(tail_hit & valid, pos, [&](u32 sq) { return pick16(kk, sq); }, lo, pl, pr, sink, wq, qs);
    }
    lq_drain<DT>(wq, qs, sink, lo, pl, pr);
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
        grid_dep_release(); // nothing to do (an earlier failure, or the other mode): the next launch proceeds
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

// Number of draws of a level: the sample size, more for a narrowed window
// (proportionally, at most SMP_MAX_SCALE times), so that about as many land
// inside it.
__device__ __forceinline__ u32 level_draws(const SelArgs& a, const SelState& s) {
    u32 draws = a.sample;
    if (s.m_win < s.m_src) {
        u64 ratio = s.m_src / (s.m_win ? s.m_win : 1);
        ratio = ratio < 1 ? 1 : ratio > SMP_MAX_SCALE ? SMP_MAX_SCALE : ratio;
        draws = (u32)((u64)draws * ratio);
    }
    return draws;
}

// Slots of the sample array a level fills: every draw when they all fit
// (draw j at slot j), else the draws inside the window (appended, up to the
// capacity).  `count` is the append counter.
__device__ __forceinline__ u32 sample_stored(const SelArgs& a, u32 draws, const u32* count) {
    if (draws <= a.samp_cap) return draws;
    const u32 c = *(const volatile u32*)count;
    return c < a.samp_cap ? c : a.samp_cap;
}

// The sample of one level, drawn by a grid of NT-thread blocks: draw j falls
// in partition j mod p at a position uniform in it (Philox4x32-10 of counter
// (4 floor(j / 4), level, salt, 0), word j mod 4).  When the draws fit the
// sample array, draw j is stored at slot j (a draw outside the window as the
// all-ones composite, which no element has); otherwise the draws inside the
// window are appended (one reservation per warp on `count`).  The four draws
// of one Philox block go to one thread; consecutive blocks of draws go to
// consecutive thread blocks.
template <int DT, int NT>
__device__ void sample_draws(const SelArgs& a, const SelState& s, typename Comp<Key<DT>::KW>::t lo,
                             typename Comp<Key<DT>::KW>::t hi, u32 draws, u32* count) {
    typedef Key<DT> K;
    typedef typename K::key_t key_t;
    constexpr int KW = K::KW;
    typedef Comp<KW> C;
    typedef typename C::t ct;
    const bool direct = draws <= a.samp_cap;
    const u32 m = (u32)s.m_src; // sources hold fewer than 2^32 elements
    const u32 p = a.parts < m ? a.parts : m;
    const u32 len = m / p, rem = m - len * p;
    const InputSrc<DT> isrc = InputSrc<DT>::make(a.keys, m);
    const CandSrc<KW> csrc{static_cast<const key_t*>(a.cand_key[s.src == SRC_CAND1 ? 1 : 0]),
                           a.cand_idx[s.src == SRC_CAND1 ? 1 : 0], m};
    ct* samp = static_cast<ct*>(a.samp);
    const u32 blocks4 = (draws + 3) / 4; // Philox blocks
    // Philox block b = (round * NT + t) * gridDim.x + blockIdx.x for thread t
    const u32 rounds = (blocks4 + gridDim.x * NT - 1) / (gridDim.x * NT);
    for (u32 rd = 0; rd < rounds; ++rd) {
        const u32 b = (rd * NT + threadIdx.x) * gridDim.x + blockIdx.x;
        // warps whose blocks of draws all lie beyond the last stop here
        const u32 warp_b0 = (rd * NT + (threadIdx.x & ~31u)) * gridDim.x + blockIdx.x;
        if (warp_b0 >= blocks4) break;
        ct c[4];
        u32 keepm = 0;
        const u32 j0 = b * 4;
        if (b < blocks4) {
            const Philox4 r = philox4x32_10(j0, s.level, 0x53414D50u, 0, (u32)a.seed, (u32)(a.seed >> 32));
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const u32 j = j0 + q;
                const u32 part = j % p;
                const u32 plo = part * len + (part < rem ? part : rem);
                const u32 psz = len + (part < rem ? 1 : 0);
                const u32 pos = plo + (u32)(((u64)r.v[q] * psz) >> 32);
                key_t kq = 0;
                u32 x = 0;
                if (j < draws) {
                    if (s.src == SRC_INPUT) isrc.at(pos, kq, x);
                    else csrc.at(pos, kq, x);
                }
                c[q] = C::make(kq, x);
                keepm |= (u32)(j < draws && c[q] >= lo && c[q] <= hi) << q;
            }
        }
        if (direct) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (b < blocks4 && j0 + q < draws) samp[j0 + q] = ((keepm >> q) & 1u) ? c[q] : ~(ct)0;
        } else {
            u32 slot = warp_reserve((u32)__popc(keepm), count);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if ((keepm >> q) & 1u) {
                    if (slot < a.samp_cap) samp[slot] = c[q];
                    ++slot;
                }
            }
        }
    }
}

// Pivots from the sample (one block of NT threads): the sample array
// (`stored` slots) into shared memory `buf` by one bulk copy (completion on
// the block's mbarrier `mb`, phase `mphase`), the number `kept` of draws in
// the window and their smallest and largest composite; then the sample
// elements of ranks k|S|/n -/+ Delta (pivot_ranks), selected with a histogram
// over [smallest, largest].  Returns kept; pl / pr stay as given when a rank
// falls outside the sample; *jl_out receives the lower rank.  `ok` turns
// false if the copy did not complete in time.
template <int DT, int NT>
__device__ u32 sample_pivots(const SelArgs& a, const SelState& s, u32 stored, typename Comp<Key<DT>::KW>::t lo,
                             typename Comp<Key<DT>::KW>::t hi, typename Comp<Key<DT>::KW>::t* buf,
                             HistSelSmem<Key<DT>::KW>& hs, uint64_t* mb, u32& mphase, bool& ok,
                             typename Comp<Key<DT>::KW>::t& pl, typename Comp<Key<DT>::KW>::t& pr,
                             long long* jl_out) {
    constexpr int KW = Key<DT>::KW;
    typedef Comp<KW> C;
    typedef typename C::t ct;
    __shared__ ct s_mn[NT / 32], s_mx[NT / 32];
    __shared__ u32 s_cnt[NT / 32];
    __shared__ long long s_jl, s_jr;
    __shared__ u32 s_kept;
    const u32 tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    // the sample array holds a whole number of 16-byte words and starts on
    // a 16-byte boundary, as does the shared copy
    const u32 bytes = (u32)((stored * sizeof(ct) + 15) & ~(size_t)15);
    __syncthreads(); // earlier readers of the shared sample are done
    if (tid == 0 && bytes > 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(mb, bytes);
        bulk_g2s(buf, a.samp, bytes, mb);
    }
    if (bytes > 0) {
        if (!mbar_wait_bounded(mb, mphase, WAIT_LIMIT_NS)) {
            ok = false;                                          // reported, and once more
            (void)mbar_wait_bounded(mb, mphase, WAIT_LIMIT_NS); // for the copy in flight
        }
        mphase ^= 1u;
    }
    if (__syncthreads_or(ok ? 0 : 1)) ok = false; // the same answer in every thread
    ct mn = ~(ct)0, mx = 0;
    u32 cnt = 0;
    for (u32 i = tid; i < stored; i += NT) {
        const ct c = buf[i];
        // (a window's upper end may be the all-ones composite itself, so the
        // stand-in for a draw outside it is excluded by value)
        const bool in = c != ~(ct)0 && c >= lo && c <= hi;
        cnt += (u32)in;
        if (in && c < mn) mn = c;
        if (in && c > mx) mx = c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const ct omn = shfl_comp(mn, lane ^ (u32)o), omx = shfl_comp(mx, lane ^ (u32)o);
        mn = omn < mn ? omn : mn;
        mx = omx > mx ? omx : mx;
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
        s_mn[warp] = mn;
        s_mx[warp] = mx;
        s_cnt[warp] = cnt;
    }
    __syncthreads();
    if (tid == 0) {
        ct a_mn = s_mn[0], a_mx = s_mx[0];
        u32 a_cnt = s_cnt[0];
        for (u32 w = 1; w < NT / 32; ++w) {
            a_mn = s_mn[w] < a_mn ? s_mn[w] : a_mn;
            a_mx = s_mx[w] > a_mx ? s_mx[w] : a_mx;
            a_cnt += s_cnt[w];
        }
        long long jl = -1, jr = 0;
        if (a_cnt > 0) pivot_ranks(a_cnt, s.m_win, s.k_rem, a.z, (a.flags & TOPK_FLAG_RAW_DELTA) != 0, jl, jr);
        s_jl = jl;
        s_jr = jr;
        s_kept = a_cnt;
        s_mn[0] = a_mn;
        s_mx[0] = a_mx;
    }
    __syncthreads();
    const u32 kept = s_kept;
    const long long jl = s_jl, jr = s_jr, top = (long long)kept - 1;
    if (jl_out) *jl_out = jl;
    if (kept > 0 && ok) {
        ct x0, x1;
        block_select_two<KW, NT>(buf, stored, s_mn[0], s_mx[0], (u32)(jl < 0 ? 0 : jl > top ? top : jl),
                                 (u32)(jr < 0 ? 0 : jr > top ? top : jr), hs, x0, x1);
        if (jl >= 0) pl = x0;
        if (jr <= top) pr = x1;
    }
    return kept;
}

// ---- pickPivots, part 1 (whole grid): the level's draws into the sample
// array (sample_draws).
template <int DT> __global__ void __launch_bounds__(SMP_NT) k_sample(SelArgs a, int first) {
    grid_dep_wait();
    grid_dep_release();
    typedef Comp<Key<DT>::KW> C;
    const SelState s = first ? initial_state<DT>(a) : *a.st;
    if (s.phase != PH_RUN || s.m_src <= a.grid_G || s.m_win <= a.finish_T) return;
    sample_draws<DT, SMP_NT>(a, s, C::from128(s.lo), C::from128(s.hi), level_draws(a, s), a.samp_count);
}

// ---- pickPivots, part 2 (one block): the pivots from the sample
// (sample_pivots), then the next pass armed; the sample count is left at zero
// for the next level.  A window of at most T elements is collected whole.
template <int KW> struct PivotSmem {
    typedef typename Comp<KW>::t ct;
    ct buf[Lim<KW>::ELEMS];
    HistSelSmem<KW> hs;
};

template <int DT> __global__ void __launch_bounds__(PIV_NT) k_pivots(SelArgs a, int first) {
    grid_dep_wait();
    grid_dep_release();
    constexpr int KW = Key<DT>::KW;
    typedef Comp<KW> C;
    typedef typename C::t ct;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<PivotSmem<KW>*>(smem_raw);
    __shared__ __align__(8) uint64_t mb; // completion of the sample's bulk copy
    __shared__ u32 s_go;
    SelState* g = a.st;
    const u32 tid = threadIdx.x;
    const SelState s = first ? initial_state<DT>(a) : *g;
    if (tid == 0) {
        if (first) *g = s;
        u32 go = s.phase == PH_RUN;
        if (go && s.m_src <= a.grid_G) {
            g->phase = PH_FINISH;
            go = 0;
        }
        s_go = go;
        mbar_init(&mb, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (!s_go) return;
    const ct lo = C::from128(s.lo), hi = C::from128(s.hi);
    ct pl = lo, pr = hi; // "collect": every window element becomes a candidate
    u32 kept = 0, mphase = 0;
    long long jl = -1;
    bool ok = true;
    if (s.m_win > a.finish_T) {
        const u32 stored = sample_stored(a, level_draws(a, s), a.samp_count);
        kept = sample_pivots<DT, PIV_NT>(a, s, stored, lo, hi, sm.buf, sm.hs, &mb, mphase, ok, pl, pr, &jl);
    }
    if (tid == 0) {
        if (!ok) {
            latch(a.err, ST_ETIMEOUT);
            g->phase = PH_ERROR;
        }
        g->pl = (u128)pl;
        g->pr = (u128)pr;
        g->dst = s.src == SRC_CAND0 ? SRC_CAND1 : SRC_CAND0;
        g->cnt_a = 0;
        g->cnt_b = 0;
        g->pending = 1;
        g->level = s.level + 1;
        g->levels_grid++;
        if (s.level == 0) g->sample_kept = kept;
        // many a-elements expected: the pass compacts with block scans (on
        // the first level the host has chosen, by the same rule, the one
        // variant it launches)
        g->dense = (s.level == 0 && a.first_dense >= 0)
                       ? (u32)a.first_dense
                       : (jl >= 0 && kept > 0 && (double)(jl + 1) > (double)kept / 16.0) ? 1u : 0u;
        *a.samp_count = 0;
    }
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
    a.first_dense = -1; // decided on the device unless the host fixes it
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
    if (cudaFuncSetAttribute(k_finish<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
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

// Pass mode of the first level: dense when more than 1/16 of the sample is
// expected below the lower pivot.  The first level's sample is `s` draws, all
// inside its window, so its pivot ranks are known before the launch; the
// mode only steers the pass (both modes give the same result).
static bool first_level_dense(u64 n, u64 k, u32 s, float z, bool raw) {
    const double mu = (double)s * (double)k / (double)n;
    const double d = raw ? z : z * std::sqrt(std::max(0.0, mu * (1.0 - mu / s))) + z * z / 3.0 + 1.0;
    const double jl = std::floor(mu - d) - 1.0;
    return jl >= 0.0 && jl + 1.0 > (double)s / 16.0;
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
    // the first level's pass mode, fixed here so that one variant is launched
    const bool bulk = a.aligned && !(tu.flags & TOPK_FLAG_NO_BULK_COPY);
    a.first_dense =
        bulk ? (first_level_dense(n, k, tu.sample, tu.z, (tu.flags & TOPK_FLAG_RAW_DELTA) != 0) ? 1 : 0) : -1;
    auto first_pass = [&]() -> cudaError_t {
        if (!bulk) return launch_dep(k_pass_first<DT>, pass_grid<DT>(sms, true), PASS_NT, 0, st, a);
        if (a.first_dense)
            return launch_dep(k_pass_tma<DT, true>, tma_grid<DT, true>(sms), TMA_NT, TmaCfg<DT, true>::SMEM, st, a);
        return launch_dep(k_pass_tma<DT, false>, tma_grid<DT, false>(sms), TMA_NT, TmaCfg<DT, false>::SMEM, st, a);
    };
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
        if (l == 0) e = first_pass();
        else e = launch_dep(k_pass<DT>, pass_grid<DT>(sms, false), PASS_NT, 0, st, a);
        if (e != cudaSuccess) return cuda_status(e);
        if (l == 0 && ctx) profile_pass_end(ctx, st);
    }
    const cudaError_t e = launch_dep(k_finish<DT>, 1, BLK_NT, smem, st, a, levels == 0 ? 1 : 0);
    if (e != cudaSuccess) return cuda_status(e);
    if (ctx) count_launch(ctx, 3 * (uint64_t)levels + 1);
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
constexpr size_t NA_OFF_PART = 8192;       // per-block composites of the k = 1 / k = n reduction
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
    // the error word, the block-done counters and the sample count must
    // start at zero (a call that failed may have left them set)
    if (cudaMemsetAsync(words, 0, 4 * sizeof(u32), st) != cudaSuccess) return TOPK_ECUDA;
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
