// select.cu — topk_select: selection of the k smallest of n unsorted keys
// (paper, Section 2, Algorithm "select"; Section 4.1, Theorem "selectFR").
//
// Launch sequence of one call (all on the caller's stream, no host round
// trip):
//   k_plan   (1 block)  level 1: initialise the state, sample, pivots
//   k_pass   (grid)     level 1: stream the input once, a -> output,
//                       b -> candidate buffer 0, block sums -> n_a, n_b
//   k_plan / k_pass     levels 2..L on the candidate buffers (L predicted on
//                       the host; a level whose state is already small
//                       returns at once)
//   k_finish (1 block)  remaining levels inside one block until at most T
//                       candidates are left, then selects rank k among them,
//                       writes the rest of the output and the rank-k pair.
// k = 1 (the base case of Algorithm "select", a global minimum) and k = n
// (everything selected) take one reduction kernel instead.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>

#include "internal.h"
#include "select_block.cuh"

namespace topk {

// ------------------------------------------------------------- kernels

template <int DT> __global__ void __launch_bounds__(BLK_NT) k_plan(SelArgs a, int first) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<BlockSmem<Key<DT>::KW>*>(smem_raw);
    SelState* g = a.st;
    if (threadIdx.x == 0) {
        if (first) init_state<DT>(g, a);
        else decide(*g);
        u32 go = g->phase == PH_RUN;
        if (go && g->m_src <= a.grid_G) {
            g->phase = PH_FINISH;
            go = 0;
        }
        sm.flag = go;
    }
    __syncthreads();
    if (!sm.flag) return;
    plan_level<DT>(a, sm, true);
}

// First level: the source is always the input, so this variant carries no
// candidate-source code (fewer registers on the pass that reads all n keys).
template <int DT> __global__ void __launch_bounds__(PASS_NT) k_pass_first(SelArgs a) {
    __shared__ PassSmem<PASS_NT> ps;
    const SelState s = *a.st;
    if (s.phase != PH_RUN || !s.pending || s.src != SRC_INPUT) return;
    run_pass<PASS_NT, DT, true>(a, s, blockIdx.x, gridDim.x, ps);
}

// First level, 16-byte-aligned input: a producer warp streams full tiles
// into a ring of shared-memory stages with bulk (TMA) copies while 8 consumer
// warps classify and compact, so HBM reads continue through the consumers'
// barriers.  Every wait is bounded; a timeout latches TOPK_ETIMEOUT and the
// block winds down without hanging.
constexpr int TMA_CONS = 256;
constexpr int TMA_NT = TMA_CONS + 32;
constexpr u64 WAIT_LIMIT_NS = 200ull * 1000 * 1000;

template <int DT> struct TmaCfg {
    static constexpr u32 W = sizeof(typename Key<DT>::raw_t);
    static constexpr u32 TILE = TMA_CONS * 16; // elements per stage
    static constexpr u32 BYTES = TILE * W;     // 8, 16 or 32 KiB
    static constexpr u32 STAGES = W == 2 ? 8 : W == 4 ? 6 : 3;
    static constexpr u32 SMEM = STAGES * BYTES;
};

template <int DT, bool HAS_A, bool EXACT>
__device__ void tma_consume(const SelArgs& a, const SelState& s, const unsigned char* stages, uint64_t* full,
                            uint64_t* empty, u64 my_n, u32* dead, PassSmem<TMA_CONS>& ps) {
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    typedef Comp<K::KW> C;
    typedef typename C::t ct;
    typedef TmaCfg<DT> Cfg;
    typedef SyncNamed<1, TMA_CONS> Sync;
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
    const ct lo = C::from128(s.lo), pl = C::from128(s.pl), pr = C::from128(s.pr);
    const u32 lane = lane_id();
    const InputSrc<DT> isrc = InputSrc<DT>::make(a.keys, s.m_src); // head = 0: input is 16-byte aligned
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
        key_t kk[16];
        if (ok) {
            InputSrc<DT>::template load16_smem<TMA_CONS>(
                reinterpret_cast<const uint4*>(stages + (size_t)stg * Cfg::BYTES), kk);
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) kk[q] = 0;
        }
        __syncwarp();
        if (ok && lane == 0) mbar_arrive(&empty[stg]); // stage may be refilled
        const u64 tb = (blockIdx.x + i * gridDim.x) * (u64)Cfg::TILE;
        auto pos = [&](int q) -> u32 { return isrc.template idx_of<TMA_CONS>(tb, q); };
        classify_emit<TMA_CONS, HAS_A, EXACT, Sync>(kk, pos, ok ? 0xFFFFu : 0u, lo, pl, pr, sink, ps);
    }
    // the ragged last tile, read directly by the block that owns it
    const u64 nfull = s.m_src / Cfg::TILE;
    if (s.m_src % Cfg::TILE != 0 && nfull % gridDim.x == blockIdx.x) {
        const InputSrc<DT> src = InputSrc<DT>::make(a.keys, s.m_src);
        key_t kk[16];
        u32 ii[16];
        const u64 tb = nfull * (u64)Cfg::TILE;
        const u32 valid = src.template load16<TMA_CONS>(tb, kk, ii);
        auto pos = [&](int q) -> u32 { return src.template idx_of<TMA_CONS>(tb, q); };
        classify_emit<TMA_CONS, HAS_A, EXACT, Sync>(kk, pos, valid, lo, pl, pr, sink, ps);
    }
}

template <int DT> __global__ void __launch_bounds__(TMA_NT) k_pass_tma(SelArgs a) {
    typedef TmaCfg<DT> Cfg;
    typedef typename Key<DT>::raw_t raw_t;
    extern __shared__ __align__(128) unsigned char stages[];
    __shared__ __align__(8) uint64_t full[Cfg::STAGES];
    __shared__ __align__(8) uint64_t empty[Cfg::STAGES];
    __shared__ PassSmem<TMA_CONS> ps;
    __shared__ u32 dead;
    const SelState s = *a.st;
    if (s.phase != PH_RUN || !s.pending || s.src != SRC_INPUT) return;
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
            for (u64 i = 0; i < my_n; ++i) {
                const u32 stg = (u32)(i % Cfg::STAGES);
                if (i >= Cfg::STAGES) {
                    const u32 parity = (u32)(((i / Cfg::STAGES) - 1) & 1);
                    if (*(volatile u32*)&dead || !mbar_wait_bounded(&empty[stg], parity, WAIT_LIMIT_NS)) {
                        *(volatile u32*)&dead = 1;
                        latch(a.err, ST_ETIMEOUT);
                        break;
                    }
                }
                const u64 t = blockIdx.x + i * gridDim.x;
                mbar_arrive_expect_tx(&full[stg], Cfg::BYTES);
                bulk_g2s(stages + (size_t)stg * Cfg::BYTES, keys + t * Cfg::TILE, Cfg::BYTES, &full[stg]);
            }
        }
        return;
    }
    typedef Comp<Key<DT>::KW> C;
    typedef typename C::t ct;
    const ct lo = C::from128(s.lo), pl = C::from128(s.pl);
    if (lo != (ct)0) tma_consume<DT, true, true>(a, s, stages, full, empty, my_n, &dead, ps);
    else if (pl > lo) tma_consume<DT, true, false>(a, s, stages, full, empty, my_n, &dead, ps);
    else tma_consume<DT, false, false>(a, s, stages, full, empty, my_n, &dead, ps);
}

template <int DT> __global__ void __launch_bounds__(PASS_NT) k_pass(SelArgs a) {
    __shared__ PassSmem<PASS_NT> ps;
    const SelState s = *a.st;
    if (s.phase != PH_RUN || !s.pending) return;
    run_pass<PASS_NT, DT>(a, s, blockIdx.x, gridDim.x, ps);
}

template <int DT> __global__ void __launch_bounds__(BLK_NT) k_finish(SelArgs a, int first) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<BlockSmem<Key<DT>::KW>*>(smem_raw);
    SelState* g = a.st;
    if (threadIdx.x == 0) {
        if (first) init_state<DT>(g, a);
        else decide(*g);
        if (g->phase == PH_RUN) g->phase = PH_FINISH;
        sm.flag = g->phase == PH_FINISH;
    }
    __syncthreads();
    if (!sm.flag) return;
    block_levels_and_finish<DT, true>(a, sm);
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
    tu.G = 4 * tu.T;
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
    if (cudaFuncSetAttribute(k_pass_tma<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TmaCfg<DT>::SMEM) != cudaSuccess)
        return TOPK_ECUDA;
    const int bytes = (int)sizeof(BlockSmem<Key<DT>::KW>);
    if (cudaFuncSetAttribute(k_plan<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
        return TOPK_ECUDA;
    if (cudaFuncSetAttribute(k_finish<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
        return TOPK_ECUDA;
    done_mask.fetch_or(bit);
    return TOPK_OK;
}

// Resident blocks per SM of each pass variant: the grid is one full wave.
template <int DT> static int tma_grid(int sms) {
    static int occ = 0;
    if (occ == 0) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_pass_tma<DT>, TMA_NT, TmaCfg<DT>::SMEM) !=
            cudaSuccess)
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
        k_extreme<DT><<<sms * EXT_BLOCKS_PER_SM, EXT_NT, 0, st>>>(a, k == n && n > 1 ? 1 : 0, counter, partials);
        if (ctx) {
            profile_pass_end(ctx, st);
            count_launch(ctx);
        }
        return cuda_status(cudaGetLastError());
    }
    topk_status rs = set_smem_attrs<DT>();
    if (rs != TOPK_OK) return rs;
    // grid levels until the candidates fit the block finisher's range
    int levels = 0;
    {
        double m = (double)n, kr = (double)k;
        while (m > tu.G && levels < 8) {
            m = 1.5 * est_bracket((u64)m, (u64)std::max(1.0, std::min(kr, m)), tu.sample, tu.z);
            kr = m / 2;
            ++levels;
        }
    }
    const size_t smem = sizeof(BlockSmem<KW>);
    for (int l = 0; l < levels; ++l) {
        k_plan<DT><<<1, BLK_NT, smem, st>>>(a, l == 0 ? 1 : 0);
        if (l == 0 && ctx) profile_pass_begin(ctx, st);
        if (l == 0 && a.aligned && !(tu.flags & TOPK_FLAG_NO_BULK_COPY))
            k_pass_tma<DT><<<tma_grid<DT>(sms), TMA_NT, TmaCfg<DT>::SMEM, st>>>(a);
        else if (l == 0) k_pass_first<DT><<<pass_grid<DT>(sms, true), PASS_NT, 0, st>>>(a);
        else k_pass<DT><<<pass_grid<DT>(sms, false), PASS_NT, 0, st>>>(a);
        if (l == 0 && ctx) profile_pass_end(ctx, st);
    }
    k_finish<DT><<<1, BLK_NT, smem, st>>>(a, levels == 0 ? 1 : 0);
    if (ctx) count_launch(ctx, 2 * (uint64_t)levels + 1);
    return cuda_status(cudaGetLastError());
}

template <int DT>
static topk_status run_select(topk_ctx* ctx, const void* keys, u64 n, u64 k, void* out_keys, u32* out_idx,
                              void* kth_key, u32* kth_idx, const topk_params* prm, cudaStream_t st) {
    constexpr int KW = Key<DT>::KW;
    const Tuning tu = make_tuning<KW>(prm, ctx->sms);
    SelArgs a = make_args(keys, n, k, out_keys, out_idx, kth_key, kth_idx, tu);
    a.st = static_cast<SelState*>(ctx->d_state);
    a.err = ctx->d_err;
    ctx->last_kind = LAST_SELECT;

    const u64 cap = (k == 1 || k == n) ? 0 : candidate_capacity(n, k, tu);
    a.cap_b = cap;
    const size_t kbytes = KW / 8;
    Carve cv;
    const size_t off_part = cv.take(sizeof(typename Comp<KW>::t) * (size_t)ctx->sms * EXT_BLOCKS_PER_SM);
    const size_t off_k0 = cv.take(cap * kbytes), off_k1 = cv.take(cap * kbytes);
    const size_t off_i0 = cv.take(cap * 4), off_i1 = cv.take(cap * 4);
    topk_status rs = ensure_scratch(ctx, cv.off);
    if (rs != TOPK_OK) return rs;
    char* base = static_cast<char*>(ctx->scratch.base);
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
constexpr u64 NOALLOC_CAP = 1ull << 18;    // candidate pairs per buffer
constexpr size_t NA_OFF_STATE = 0;         // SelState
constexpr size_t NA_OFF_WORDS = 4096;      // [0] error word, [1] block-done counter
constexpr size_t NA_OFF_PART = 8192;       // per-block composites of the k = 1 / k = n reduction
constexpr size_t NA_PART_BYTES = 64 * 1024;
constexpr size_t NA_OFF_CAND = NA_OFF_PART + NA_PART_BYTES;
constexpr size_t NA_BYTES = NA_OFF_CAND + 2 * NOALLOC_CAP * (8 + 4); // about 6 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64] = {};

// Device address of the array on the current device `dev` (set-up on first use).
static topk_status noalloc_base(int dev, char** out) {
    if (dev < 0 || dev >= 64) return TOPK_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return TOPK_ECUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<char*>(g_noalloc_addr[dev]);
    return TOPK_OK;
}

template <int DT>
static topk_status run_select_noalloc(char* base, int sms, const void* keys, u64 n, u64 k, void* out_keys,
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
    // the error word and the block-done counter must start at zero
    if (cudaMemsetAsync(words, 0, 2 * sizeof(u32), st) != cudaSuccess) return TOPK_ECUDA;
    if (d_status && cudaMemsetAsync(d_status, 0, sizeof(u32), st) != cudaSuccess) return TOPK_ECUDA;
    return enqueue_select<DT>(nullptr, a, tu, sms, words + 1, base + NA_OFF_PART, st);
}

} // namespace topk

using namespace topk;

extern "C" {

topk_status topk_select(topk_ctx* ctx, const void* d_keys, uint64_t n, uint64_t k, topk_dtype dtype,
                        void* d_out_keys, uint32_t* d_out_idx, void* d_kth_key, uint32_t* d_kth_idx,
                        const topk_params* params, void* stream) {
    if (!ctx || !d_keys || !d_out_keys || !d_out_idx || !d_kth_key || !d_kth_idx) return TOPK_EINVAL;
    const int w = dtype_bytes(dtype);
    if (w == 0) return TOPK_EINVAL;
    if (k < 1 || k > n || n > 0xFFFFFFFFull) return TOPK_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_keys) % (uintptr_t)w) return TOPK_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_out_keys) % (uintptr_t)w) return TOPK_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return TOPK_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (dtype) {
    case TOPK_U32: return run_select<DT_U32>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
    case TOPK_I32: return run_select<DT_I32>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
    case TOPK_F32: return run_select<DT_F32>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
    case TOPK_BF16: return run_select<DT_BF16>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
    case TOPK_U64: return run_select<DT_U64>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
    default: return TOPK_EINVAL;
    }
}

topk_status topk_select_noalloc(const void* d_keys, uint64_t n, uint64_t k, topk_dtype dtype,
                                void* d_out_keys, uint32_t* d_out_idx, void* d_kth_key,
                                uint32_t* d_kth_idx, uint32_t* d_status, void* stream) {
    if (!d_keys || !d_out_keys || !d_out_idx || !d_kth_key || !d_kth_idx) return TOPK_EINVAL;
    const int w = dtype_bytes(dtype);
    if (w == 0) return TOPK_EINVAL;
    if (k < 1 || k > n || n > NOALLOC_MAX_N) return TOPK_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_keys) % (uintptr_t)w) return TOPK_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_out_keys) % (uintptr_t)w) return TOPK_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TOPK_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TOPK_ECUDA;
    char* base = nullptr;
    topk_status rs = noalloc_base(dev, &base);
    if (rs != TOPK_OK) return rs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (dtype) {
    case TOPK_U32: return run_select_noalloc<DT_U32>(base, sms, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, d_status, st);
    case TOPK_I32: return run_select_noalloc<DT_I32>(base, sms, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, d_status, st);
    case TOPK_F32: return run_select_noalloc<DT_F32>(base, sms, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, d_status, st);
    case TOPK_BF16: return run_select_noalloc<DT_BF16>(base, sms, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, d_status, st);
    case TOPK_U64: return run_select_noalloc<DT_U64>(base, sms, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, d_status, st);
    default: return TOPK_EINVAL;
    }
}

topk_status topk_ctx_reserve(topk_ctx* ctx, uint64_t n, topk_dtype dtype) {
    if (!ctx) return TOPK_EINVAL;
    const int w = dtype_bytes(dtype);
    if (w == 0 || n == 0) return TOPK_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return TOPK_ECUDA;
    const u32 ELEMS = w == 8 ? Lim<64>::ELEMS : Lim<32>::ELEMS;
    const size_t kbytes = w == 8 ? 8 : 4;
    // worst first bracket over k (k = n/2), default tuning
    u64 cap = (u64)(2.0 * est_bracket(n, std::max<u64>(1, n / 2), ELEMS, 4.0f)) + 4ull * ELEMS;
    cap = std::min<u64>(cap, std::max<u64>(n, ELEMS));
    cap = (cap + 4095) & ~(u64)4095;
    Carve cv;
    cv.take(cap * kbytes);
    cv.take(cap * kbytes);
    cv.take(cap * 4);
    cv.take(cap * 4);
    return ensure_scratch(ctx, cv.off);
}

topk_status topk_last_stats(topk_ctx* ctx, topk_stats* out) {
    if (!ctx || !out) return TOPK_EINVAL;
    *out = topk_stats{};
    if (ctx->last_kind != LAST_SELECT) return TOPK_OK;
    SelState s;
    if (cudaMemcpy(&s, ctx->d_state, sizeof(SelState), cudaMemcpyDeviceToHost) != cudaSuccess) return TOPK_ECUDA;
    out->levels_grid = s.levels_grid;
    out->levels_block = s.levels_block;
    out->pivot_failures = s.failures;
    out->overflows = s.overflows;
    out->first_candidates = s.first_cand;
    out->sample_kept = s.sample_kept;
    return TOPK_OK;
}

} // extern "C"
