// batched.cu — topk_select_batched: many independent selections (rows of
// uneven length, each with its own k) in one persistent launch.
//
// The paper has no batched form; each row is the selection of Section 2
// (Algorithm "select").  A row up to the split length is selected whole by
// one thread block: sample, pivots, a block-wide partitioning pass into the
// block's candidate buffer, the branch, and the exact finish among at most T
// candidates (select_block.cuh).  A longer ("wide") row takes its first
// level as topk_select does, over the whole GPU: one block samples the row
// and picks its pivots (k_wide_plan), one grid-wide pass streams the tiles
// of all wide rows and classifies each against its own row's pivots, the
// last block to finish a row taking the branch (k_wide_pass), and the
// persistent kernel then finishes the wide rows from their candidates while
// it selects the short rows whole.  Rows are handed out longest first from a
// device work queue, so the blocks that finish early take the short rows at
// the end.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>

#include "internal.h"
#include "select_block.cuh"

namespace topk {

constexpr u64 BATCH_CAP = 1ull << 16; // candidate pairs per buffer per block
constexpr u32 BATCH_SAMPLE = 2048;    // draws per level (rows are short)
constexpr u32 WIDE_NONE = 0xFFFFFFFFu;  // split length that makes no row wide
constexpr u32 WIDE_SPLIT = 1u << 15;    // default split length
constexpr u32 WIDE_SAMPLE = 2048;       // draws of a wide row's first level
constexpr u32 WIDE_TILE = PASS_NT * 16; // keys per tile of the wide pass
constexpr u64 WIDE_POOL_PAIRS = 1ull << 23; // candidate pairs of all wide rows together

// Block variants: NT threads, a sample / finish buffer of CAP composites
// (T <= CAP), at least MINB resident blocks per SM.  1024 threads are capped
// at 64 registers (some spill in the level code); 512 and 256 threads get
// 128 and hold half and a quarter of the composites, so smaller blocks run
// more rows at once per SM.
template <int KW, int NT> struct BatchVariant;
template <int KW> struct BatchVariant<KW, 1024> {
    static constexpr u32 CAP = Lim<KW>::ELEMS;
    static constexpr int MINB = 1;
};
template <int KW> struct BatchVariant<KW, 512> {
    static constexpr u32 CAP = Lim<KW>::ELEMS / 2;
    static constexpr int MINB = 1;
};
template <int KW> struct BatchVariant<KW, 256> {
    static constexpr u32 CAP = Lim<KW>::ELEMS / 4;
    static constexpr int MINB = 2;
};
template <int KW, int NT> using BatchSmem = BlockSmem<KW, NT, BatchVariant<KW, NT>::CAP>;

struct BatchArgs {
    const void* keys;
    const u64* row_off; // rows + 1
    const u32* row_k;   // rows
    u32 rows;
    void* out_keys;
    u32* out_idx;
    const u64* out_off; // rows + 1
    void* kth_keys;
    u32* kth_idx;
    // Rows given by pointers instead (used by the serving loop; when set, the
    // arrays above are ignored): row i has keys row_keys[i][0..row_n[i]),
    // outputs row_out_keys[i] / row_out_idx[i] (row_k[i] entries) and
    // row_kth_key[i] / row_kth_idx[i] (one entry).
    const void* const* row_keys;
    const u64* row_n;
    void* const* row_out_keys;
    u32* const* row_out_idx;
    void* const* row_kth_key;
    u32* const* row_kth_idx;
    u32* order;         // rows: row ids, longest first
    u32* queue;         // next index into order
    SelState* states;   // one per block
    char* cand;         // per block: key'[2][CAP], idx[2][CAP]
    u64 seed;
    u32 parts, sample, finish_T;
    float z;
    u32 flags;
    u32* err;
    // wide rows (row arrays only; WIDE_NONE: none)
    u32 key_bytes;      // width of a key
    u32 split;          // rows longer than this are wide
    u32* wide;          // rows: ids of the wide rows, longest first
    u32* words;         // [0] wide rows, [1] planning queue
    u64* tile_pre;      // rows + 1: tiles of the wide rows before the j-th
    u32* done;          // rows: tiles of the row classified by the wide pass
    SelState* rstate;   // rows: state of each wide row
    u64* rcand;         // rows: the row's candidate buffer in the pool (pairs), ~0 = none
    char* pool;         // key'[pool_pairs], then idx[pool_pairs]
    u64 pool_pairs;
    u64* pool_next;     // pairs of the pool handed out
};

__device__ __forceinline__ bool is_wide(const BatchArgs& b, u64 len) {
    return b.split != WIDE_NONE && b.row_keys == nullptr && len > (u64)b.split;
}

// Tiles of the wide pass over a row: tile coordinates start at the 16-byte
// boundary at or below the row's first key (InputSrc), so the first tile
// holds `head` slots before it.
__device__ __forceinline__ u64 wide_tiles(const void* keys, u64 len, u32 key_bytes) {
    const u64 head = (u64)((reinterpret_cast<uintptr_t>(keys) & 15u) / (uintptr_t)key_bytes);
    return (len + head + WIDE_TILE - 1) / WIDE_TILE;
}

// Exclusive scan of one value per thread over a block of NT threads; *total
// receives the sum.  `ws` holds NT / 32 words.
template <int NT> __device__ __forceinline__ u32 block_excl_scan(u32 v, u32* ws, u32* total) {
    const u32 lane = lane_id(), warp = threadIdx.x >> 5;
    u32 incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (u32)o) incl += y;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const u32 x = lane < NT / 32 ? ws[lane] : 0u;
        u32 wi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= (u32)o) wi += y;
        }
        if (lane < NT / 32) ws[lane] = wi - x;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    const u32 r = ws[warp] + incl - v;
    __syncthreads();
    return r;
}

// Orders the rows by floor(log2(length)), longest first (one block).
__global__ void __launch_bounds__(1024) k_batch_order(BatchArgs b) {
    grid_dep_wait();
    grid_dep_release();
    __shared__ u32 hist[66], start[66];
    for (u32 i = threadIdx.x; i < 66; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (u32 i = threadIdx.x; i < b.rows; i += blockDim.x) {
        const u64 len = b.row_keys ? b.row_n[i] : b.row_off[i + 1] - b.row_off[i];
        atomicAdd(&hist[len ? 64 - __clzll((long long)len) : 0], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        u32 run = 0;
        for (int k = 65; k >= 0; --k) {
            start[k] = run;
            run += hist[k];
        }
        *b.queue = 0;
    }
    __syncthreads();
    for (u32 i = threadIdx.x; i < b.rows; i += blockDim.x) {
        const u64 len = b.row_keys ? b.row_n[i] : b.row_off[i + 1] - b.row_off[i];
        const u32 pos = atomicAdd(&start[len ? 64 - __clzll((long long)len) : 0], 1u);
        b.order[pos] = i;
    }
    if (b.split == WIDE_NONE || b.row_keys != nullptr) return;
    // the wide rows in queue order, with the prefix of their tile counts
    __syncthreads();
    __shared__ u32 ws[32], tot;
    __shared__ u64 carry_rows, carry_tiles;
    if (threadIdx.x == 0) {
        carry_rows = 0;
        carry_tiles = 0;
        *b.pool_next = 0;
        b.words[1] = 0;
    }
    __syncthreads();
    const unsigned char* base = static_cast<const unsigned char*>(b.keys);
    for (u32 c0 = 0; c0 < b.rows; c0 += 1024) {
        const u32 i = c0 + threadIdx.x;
        u32 row = 0, flag = 0, tiles = 0;
        if (i < b.rows) {
            row = b.order[i];
            const u64 len = b.row_off[row + 1] - b.row_off[row];
            if (is_wide(b, len)) {
                flag = 1;
                tiles = (u32)wide_tiles(base + b.row_off[row] * (u64)b.key_bytes, len, b.key_bytes);
            }
        }
        const u32 rpos = block_excl_scan<1024>(flag, ws, &tot);
        const u32 nr = tot;
        const u32 tpos = block_excl_scan<1024>(tiles, ws, &tot);
        const u32 nt = tot;
        if (flag) {
            const u64 j = carry_rows + rpos;
            b.wide[j] = row;
            b.tile_pre[j] = carry_tiles + tpos;
            b.done[row] = 0;
            b.rcand[row] = ~0ull;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_rows += nr;
            carry_tiles += nt;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        b.words[0] = (u32)carry_rows;
        b.tile_pre[carry_rows] = carry_tiles;
    }
}

// Arguments of row `row` (keys at r0, n keys, rank k) for the selection
// code of select_block.cuh; state and candidate buffers set by the caller.
template <int DT>
__device__ __forceinline__ SelArgs row_args(const BatchArgs& b, u32 row, u64 r0, u64 n, u64 k) {
    typedef typename Key<DT>::raw_t raw_t;
    SelArgs a{};
    a.keys = static_cast<const raw_t*>(b.keys) + r0;
    a.out_keys = static_cast<raw_t*>(b.out_keys) + b.out_off[row];
    a.out_idx = b.out_idx + b.out_off[row];
    a.kth_key = static_cast<raw_t*>(b.kth_keys) + row;
    a.kth_idx = b.kth_idx + row;
    a.n = n;
    a.k = k;
    a.seed = b.seed ^ ((u64)row * 0x9E3779B97F4A7C15ull);
    a.parts = b.parts;
    a.sample = b.sample;
    a.finish_T = b.finish_T;
    a.grid_G = b.finish_T;
    a.z = b.z;
    a.flags = b.flags;
    a.aligned = 0;
    a.err = b.err;
    return a;
}

template <int KW> __device__ __forceinline__ typename Comp<KW>::key_t* pool_keys(const BatchArgs& b, u64 off) {
    return reinterpret_cast<typename Comp<KW>::key_t*>(b.pool) + off;
}
template <int KW> __device__ __forceinline__ u32* pool_idx(const BatchArgs& b, u64 off) {
    return reinterpret_cast<u32*>(b.pool + ((b.pool_pairs * sizeof(typename Comp<KW>::key_t) + 255) & ~(u64)255)) +
           off;
}

// First level of the wide rows, part 1 (one block of 256 threads per row,
// persistent over a queue, several blocks per SM): the row's sample and pivots (plan_level, with
// the larger sample of a first level), then a candidate buffer from the
// pool: twice the bracket the pivots' sample ranks predict plus a margin, at
// most BATCH_CAP pairs.  A row the pool cannot serve is left whole to the
// persistent kernel.
constexpr int WIDE_PLAN_NT = 256;

template <int DT> __global__ void __launch_bounds__(WIDE_PLAN_NT) k_wide_plan(BatchArgs b) {
    grid_dep_wait();
    constexpr int KW = Key<DT>::KW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<BatchSmem<KW, WIDE_PLAN_NT>*>(smem_raw);
    __shared__ u32 s_row;
    const u32 nwide = b.words[0];
    while (true) {
        if (threadIdx.x == 0) {
            const u32 j = atomicAdd(&b.words[1], 1u);
            s_row = j < nwide ? b.wide[j] : 0xFFFFFFFFu;
        }
        __syncthreads();
        const u32 row = s_row;
        __syncthreads();
        if (row == 0xFFFFFFFFu) break;
        const u64 r0 = b.row_off[row], n = b.row_off[row + 1] - r0, k = b.row_k[row];
        if (k == 0 || k > n || n > 0xFFFFFFFFull) continue; // reported by the persistent kernel
        SelArgs a = row_args<DT>(b, row, r0, n, k);
        SelState* g = b.rstate + row;
        a.st = g;
        a.sample = WIDE_SAMPLE < BatchSmem<KW, WIDE_PLAN_NT>::ELEMS ? WIDE_SAMPLE : BatchSmem<KW, WIDE_PLAN_NT>::ELEMS;
        a.cap_b = 0;
        if (threadIdx.x == 0) init_state<DT>(g, a);
        __syncthreads();
        plan_level<DT>(a, sm, true);
        if (threadIdx.x == 0) {
            double est = (double)n;
            const long long top = (long long)sm.kept - 1;
            if (sm.kept > 0) {
                const long long l = sm.jl < 0 ? 0 : sm.jl, r = sm.jr > top ? top : sm.jr;
                est = (double)(r - l + 1) / (double)sm.kept * (double)n;
            }
            u64 cap = (u64)(2.0 * est) + 2048;
            cap = cap < n ? cap : n;
            cap = cap < BATCH_CAP ? cap : BATCH_CAP;
            cap = (cap + 255) & ~(u64)255;
            const u64 off = atomicAdd(reinterpret_cast<unsigned long long*>(b.pool_next), (unsigned long long)cap);
            if (off + cap <= b.pool_pairs) {
                g->cap_b = cap;
                b.rcand[row] = off;
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ u64 atomic_read_u64(u64* p) {
    return atomicAdd(reinterpret_cast<unsigned long long*>(p), 0ull);
}

// First level of the wide rows, part 2: the tiles of all wide rows, in
// order, split into one contiguous run per block.  Every element is
// classified against its own row's pivots (the window is the whole row:
// a below pl, b from pl to pr); a- and b-elements leave with one reservation
// per warp and class on the row's counters.  Each warp adds its part of the
// tiles it classified of a row to the row's done count when it leaves the
// row (no block barrier); the warp that completes a row takes the branch of
// Algorithm "select" for it.
template <int DT> struct WideRow {
    typedef Comp<Key<DT>::KW> C;
    u32 row;
    u64 t0, t1;      // the row's tiles [t0, t1)
    bool live;       // the row has a candidate buffer
    typename C::t pl, pr;
    TileBounds<DT> tbd; // bounds on raw key bits for tiles away from the pivots' positions
    SelState* g;
    InputSrc<DT> src;
    Sink<DT> sink;
};

template <int DT> __device__ __forceinline__ void wide_row_open(const BatchArgs& b, u32 j, WideRow<DT>& w) {
    typedef Key<DT> K;
    typedef Comp<K::KW> C;
    w.row = b.wide[j];
    w.t0 = b.tile_pre[j];
    w.t1 = b.tile_pre[j + 1];
    const u64 off = b.rcand[w.row];
    w.live = off != ~0ull;
    if (!w.live) return;
    w.g = b.rstate + w.row;
    w.pl = C::from128(w.g->pl);
    w.pr = C::from128(w.g->pr);
    w.tbd = TileBounds<DT>::make(w.pl, w.pr);
    const u64 r0 = b.row_off[w.row];
    w.src = InputSrc<DT>::make(static_cast<const typename K::raw_t*>(b.keys) + r0, b.row_off[w.row + 1] - r0);
    w.sink.out_keys = static_cast<typename K::raw_t*>(b.out_keys) + b.out_off[w.row];
    w.sink.out_idx = b.out_idx + b.out_off[w.row];
    w.sink.out_base = 0;
    w.sink.cap_a = w.g->k_rem;
    w.sink.ck = pool_keys<K::KW>(b, off);
    w.sink.ci = pool_idx<K::KW>(b, off);
    w.sink.cap_b = w.g->cap_b;
    w.sink.cnt_a = &w.g->cnt_a;
    w.sink.cnt_b = &w.g->cnt_b;
}

// A warp leaves row w after classifying its part of `n` of the row's tiles
// (one lane; every tile is classified by `parts` warps): the warp that
// completes the row's count takes the branch.
template <int DT>
__device__ __forceinline__ void wide_row_close(const BatchArgs& b, const WideRow<DT>& w, u32 n, u32 parts) {
    if (!w.live || n == 0) return;
    __threadfence();
    const u32 prev = atomicAdd(&b.done[w.row], n);
    if ((u64)prev + n == (w.t1 - w.t0) * parts) { // all of the row's tiles: the branch
        __threadfence();
        w.g->cnt_a = atomic_read_u64(&w.g->cnt_a);
        w.g->cnt_b = atomic_read_u64(&w.g->cnt_b);
        decide(*w.g);
    }
}

// The wide pass streams with the bulk-copy engine: one producer warp copies
// the block's tiles, in order, into a ring of shared-memory stages and
// records each tile's wide row and extent; eight consumer warps classify.  A
// tile is copied from the 16-byte boundary at or below its first slot up to
// the last 16-byte boundary inside its row (so no copy reads past the row);
// the few keys after that boundary are read directly.
constexpr int WIDE_CONS = 256;               // consumer threads
constexpr int WIDE_NT = WIDE_CONS + 32;      // plus the producer warp
constexpr u64 WIDE_WAIT_NS = 200ull * 1000 * 1000;
static_assert(WIDE_CONS * 16 == (int)WIDE_TILE, "a tile is 16 keys per consumer thread");

template <int DT> struct WideCfg {
    static constexpr u32 W = sizeof(typename Key<DT>::raw_t);
    static constexpr u32 BYTES = WIDE_TILE * W;
    static constexpr u32 STAGES = W == 2 ? 8 : W == 4 ? 5 : 3;
    static constexpr u32 SMEM = STAGES * BYTES;
};

struct WideMeta {
    u32 j;      // index into the wide rows
    u32 bytes;  // bytes copied into the stage
    u64 tb;     // tile coordinate of the stage's first slot
};

template <int DT> __global__ void __launch_bounds__(WIDE_NT, 2) k_wide_pass(BatchArgs b) {
    grid_dep_wait();
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    constexpr int KW = K::KW;
    typedef Comp<KW> C;
    typedef typename C::t ct;
    typedef WideCfg<DT> Cfg;
    constexpr int EPV = InputSrc<DT>::EPV;
    extern __shared__ __align__(128) unsigned char stages[];
    __shared__ __align__(8) uint64_t full[Cfg::STAGES];
    __shared__ __align__(8) uint64_t empty[Cfg::STAGES];
    __shared__ WideMeta meta[Cfg::STAGES];
    __shared__ WarpQ<KW> wqs[WIDE_CONS / 32];
    __shared__ u32 dead;
    const u32 nwide = b.words[0];
    if (nwide == 0) return;
    const u64 total = b.tile_pre[nwide];
    const u64 per = (total + gridDim.x - 1) / gridDim.x;
    const u64 t0 = (u64)blockIdx.x * per;
    const u64 t1 = t0 + per < total ? t0 + per : total;
    if (t0 >= t1) return;
    if (threadIdx.x == 0) {
        for (u32 i = 0; i < Cfg::STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], WIDE_CONS / 32);
        }
        dead = 0;
        mbar_fence_init();
    }
    __syncthreads();
    // the wide row holding tile t0: tile_pre[j] <= t0 < tile_pre[j + 1]
    u32 lo = 0, hi = nwide;
    while (hi - lo > 1) {
        const u32 mid = (lo + hi) >> 1;
        if (b.tile_pre[mid] <= t0) lo = mid;
        else hi = mid;
    }
    const unsigned char* kbase = static_cast<const unsigned char*>(b.keys);
    if (threadIdx.x >= WIDE_CONS) { // producer warp: one lane issues the copies
        if (threadIdx.x == WIDE_CONS) {
            u32 j = lo, stg = 0, epar = 1; // the first pass over the ring waits for nothing
            for (u64 t = t0; t < t1; ++t) {
                while (b.tile_pre[j + 1] <= t) ++j;
                if (t - t0 >= Cfg::STAGES) {
                    if (*(volatile u32*)&dead || !mbar_wait_bounded(&empty[stg], epar, WIDE_WAIT_NS)) {
                        *(volatile u32*)&dead = 1;
                        latch(b.err, ST_ETIMEOUT);
                        break;
                    }
                }
                const u32 row = b.wide[j];
                const u64 tb = (t - b.tile_pre[j]) * (u64)WIDE_TILE;
                const unsigned char* first = kbase + b.row_off[row] * Cfg::W;
                const unsigned char* abase = reinterpret_cast<const unsigned char*>(
                    reinterpret_cast<uintptr_t>(first) & ~(uintptr_t)15);
                const unsigned char* src = abase + tb * Cfg::W;
                const unsigned char* row_end = kbase + b.row_off[row + 1] * Cfg::W;
                const uintptr_t lim = reinterpret_cast<uintptr_t>(row_end) & ~(uintptr_t)15;
                u32 bytes = 0;
                if (reinterpret_cast<uintptr_t>(src) < lim) {
                    const uintptr_t avail = lim - reinterpret_cast<uintptr_t>(src);
                    bytes = avail < Cfg::BYTES ? (u32)avail : Cfg::BYTES;
                }
                meta[stg].j = j;
                meta[stg].bytes = bytes;
                meta[stg].tb = tb;
                mbar_arrive_expect_tx(&full[stg], bytes);
                if (bytes) bulk_g2s(stages + (size_t)stg * Cfg::BYTES, src, bytes, &full[stg]);
                if (++stg == Cfg::STAGES) {
                    stg = 0;
                    epar ^= 1u;
                }
            }
        }
        return;
    }
    // consumers: the hits (pair <= pr) go to the warp's per-lane queue,
    // classified and reserved in batches (select_core.cuh), drained when the
    // warp leaves the row
    const u32 lane = lane_id();
    WarpQ<KW>& wq = wqs[threadIdx.x >> 5];
    LQState qs = LQState::make();
    const ct lo0 = 0;
    WideRow<DT> w;
    w.row = 0xFFFFFFFFu;
    w.live = false;
    u32 j_cur = 0xFFFFFFFFu, ndone = 0;
    for (u64 t = t0; t < t1; ++t) {
        const u32 i = (u32)(t - t0);
        const u32 stg = i % Cfg::STAGES;
        const u32 par = (i / Cfg::STAGES) & 1u;
        bool ok = !*(volatile u32*)&dead;
        if (ok && !mbar_wait_bounded(&full[stg], par, WIDE_WAIT_NS)) {
            ok = false;
            *(volatile u32*)&dead = 1;
            if (lane == 0) latch(b.err, ST_ETIMEOUT);
        }
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) continue; // timed out: latched; the remaining waits return at once
        const WideMeta m = meta[stg];
        if (m.j != j_cur) { // a new row: this warp leaves the previous one
            if (w.live) lq_drain<DT>(wq, qs, w.sink, lo0, w.pl, w.pr);
            __syncwarp();
            if (lane == 0 && j_cur != 0xFFFFFFFFu) wide_row_close<DT>(b, w, ndone, WIDE_CONS / 32);
            ndone = 0;
            j_cur = m.j;
            wide_row_open<DT>(b, j_cur, w);
        }
        if (w.live) {
            // slot q of this thread: tile element tb + (q / EPV) * 256 * EPV + tid * EPV + q % EPV
            const unsigned char* mine = stages + (size_t)stg * Cfg::BYTES + threadIdx.x * 16u;
            const u64 ext = w.src.extent();
            // row position of the tile's slot 0 (32 bits: rows are shorter than 2^32)
            const u32 pbase = (u32)(m.tb - w.src.head);
            auto pos = [&](int q) -> u32 {
                return pbase + (u32)((q / EPV) * WIDE_CONS * EPV) + threadIdx.x * EPV + (u32)(q % EPV);
            };
            key_t kk[16];
            u32 hit = 0;
            if (m.tb >= w.src.head && m.tb + WIDE_TILE <= ext && m.bytes == Cfg::BYTES) {
                // a tile inside the row, wholly in the stage
                raw_t rr[16];
                {
                    uint4 v[InputSrc<DT>::NV];
#pragma unroll
                    for (int jj = 0; jj < InputSrc<DT>::NV; ++jj)
                        v[jj] = *reinterpret_cast<const uint4*>(mine + jj * (WIDE_CONS * 16u));
                    InputSrc<DT>::unpack_raw(v, rr);
                }
                RawBound<DT> ba, bb;
                bool any_a, any_l;
                if (w.tbd.get(pbase, pbase + WIDE_TILE - 1, ba, bb, any_a, any_l)) {
                    hit = tile_le_dispatch<DT>(rr, bb, any_l);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) hit |= (u32)(C::make(K::fwd(rr[q]), pos(q)) <= w.pr) << q;
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) kk[q] = K::fwd(rr[q]);
            } else {
                // the row's first or last tile: slots outside the row, keys past the stage
                const u32 in_stage = m.bytes / Cfg::W; // slots held by the stage
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const u32 so = (u32)((q / EPV) * WIDE_CONS * EPV) + threadIdx.x * EPV + (u32)(q % EPV);
                    const u64 e = m.tb + so;
                    kk[q] = 0;
                    if (e >= w.src.head && e < ext) {
                        raw_t r;
                        if (so < in_stage)
                            r = *reinterpret_cast<const raw_t*>(mine + (q / EPV) * (WIDE_CONS * 16u) +
                                                                (q % EPV) * sizeof(raw_t));
                        else r = w.src.keys[e]; // past the last 16-byte boundary of the row
                        kk[q] = K::fwd(r);
                        hit |= (u32)(C::make(kk[q], pos(q)) <= w.pr) << q;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[stg]); // keys are in registers
            lq_append<DT>(hit, pos, [&](u32 sq) { return pick16(kk, sq); }, lo0, w.pl, w.pr, w.sink, wq, qs);
            ++ndone;
        } else {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[stg]);
        }
    }
    if (w.live) lq_drain<DT>(wq, qs, w.sink, lo0, w.pl, w.pr);
    __syncwarp();
    if (lane == 0 && j_cur != 0xFFFFFFFFu) wide_row_close<DT>(b, w, ndone, WIDE_CONS / 32);
}

template <int DT, int NT>
__global__ void __launch_bounds__(NT, (BatchVariant<Key<DT>::KW, NT>::MINB)) k_batched(BatchArgs b) {
    grid_dep_wait();
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    constexpr int KW = K::KW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<BatchSmem<KW, NT>*>(smem_raw);
    __shared__ u32 s_row;
    SelState* g = b.states + blockIdx.x;
    char* cand = b.cand + (size_t)blockIdx.x * 2 * BATCH_CAP * (sizeof(key_t) + 4);
    while (true) {
        if (threadIdx.x == 0) {
            const u32 idx = atomicAdd(b.queue, 1u);
            s_row = idx < b.rows ? b.order[idx] : 0xFFFFFFFFu;
        }
        __syncthreads();
        const u32 row = s_row;
        __syncthreads();
        if (row == 0xFFFFFFFFu) break;
        const bool by_ptr = b.row_keys != nullptr;
        const u64 r0 = by_ptr ? 0 : b.row_off[row];
        const u64 n = by_ptr ? b.row_n[row] : b.row_off[row + 1] - r0;
        const u64 k = b.row_k[row];
        if (k == 0 || k > n || n > 0xFFFFFFFFull) {
            if (threadIdx.x == 0) latch(b.err, ST_EINVAL);
            continue;
        }
        if (!by_ptr && is_wide(b, n) && b.rcand[row] != ~0ull) {
            // a wide row whose first level ran over the grid: finish it from
            // its candidates (further levels alternate between the row's
            // buffer and this block's second buffer)
            SelArgs a = row_args<DT>(b, row, r0, n, k);
            SelState* gw = b.rstate + row;
            const u64 off = b.rcand[row];
            a.cand_key[0] = pool_keys<KW>(b, off);
            a.cand_idx[0] = pool_idx<KW>(b, off);
            a.cand_key[1] = cand + BATCH_CAP * sizeof(key_t);
            a.cand_idx[1] = reinterpret_cast<u32*>(cand + 2 * BATCH_CAP * sizeof(key_t) + BATCH_CAP * 4);
            a.st = gw;
            a.cap_b = gw->cap_b;
            block_levels_and_finish<DT, false>(a, sm);
            __syncthreads();
            continue;
        }
        SelArgs a{};
        if (by_ptr) {
            a.keys = b.row_keys[row];
            a.out_keys = b.row_out_keys[row];
            a.out_idx = b.row_out_idx[row];
            a.kth_key = b.row_kth_key[row];
            a.kth_idx = b.row_kth_idx[row];
        } else {
            a.keys = static_cast<const raw_t*>(b.keys) + r0;
            a.out_keys = static_cast<raw_t*>(b.out_keys) + b.out_off[row];
            a.out_idx = b.out_idx + b.out_off[row];
            a.kth_key = static_cast<raw_t*>(b.kth_keys) + row;
            a.kth_idx = b.kth_idx + row;
        }
        a.n = n;
        a.k = k;
        a.cand_key[0] = cand;
        a.cand_key[1] = cand + BATCH_CAP * sizeof(key_t);
        a.cand_idx[0] = reinterpret_cast<u32*>(cand + 2 * BATCH_CAP * sizeof(key_t));
        a.cand_idx[1] = reinterpret_cast<u32*>(cand + 2 * BATCH_CAP * sizeof(key_t) + BATCH_CAP * 4);
        a.st = g;
        a.cap_b = BATCH_CAP;
        a.seed = b.seed ^ ((u64)row * 0x9E3779B97F4A7C15ull);
        a.parts = b.parts;
        a.sample = b.sample;
        a.finish_T = b.finish_T;
        a.grid_G = b.finish_T;
        a.z = b.z;
        a.flags = b.flags;
        a.aligned = 0;
        a.err = b.err;
        if (threadIdx.x == 0) {
            init_state<DT>(g, a);
            g->phase = PH_FINISH;
        }
        __syncthreads();
        block_levels_and_finish<DT, false>(a, sm);
        __syncthreads();
    }
}

// Resident blocks per SM of one variant (once per device and variant).
template <int DT, int NT> static int batched_blocks_per_sm(int device, topk_status& rs) {
    constexpr int KW = Key<DT>::KW;
    static std::atomic<int> occ[64];
    int& o0 = *reinterpret_cast<int*>(&occ[device & 63]);
    int o = occ[device & 63].load();
    rs = TOPK_OK;
    if (o == 0) {
        if (cudaFuncSetAttribute(k_batched<DT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(BatchSmem<KW, NT>)) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_batched<DT, NT>, NT, sizeof(BatchSmem<KW, NT>)) !=
                cudaSuccess) {
            rs = TOPK_ECUDA;
            return 0;
        }
        o = std::max(1, o);
        occ[device & 63].store(o);
    }
    (void)o0;
    return o;
}

// Resident blocks per SM of the wide pass, and the planning kernel's
// shared-memory attribute (once per device and key type).
template <int DT> static topk_status wide_setup(int device, int& pass_per_sm, int& plan_per_sm) {
    constexpr int KW = Key<DT>::KW;
    static std::atomic<int> occ[64];
    int o = occ[device & 63].load();
    if (o == 0) {
        int op = 0;
        if (cudaFuncSetAttribute(k_wide_plan<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(BatchSmem<KW, WIDE_PLAN_NT>)) != cudaSuccess ||
            cudaFuncSetAttribute(k_wide_pass<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)WideCfg<DT>::SMEM) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_wide_pass<DT>, WIDE_NT, WideCfg<DT>::SMEM) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&op, k_wide_plan<DT>, WIDE_PLAN_NT,
                                                          sizeof(BatchSmem<KW, WIDE_PLAN_NT>)) != cudaSuccess)
            return TOPK_ECUDA;
        o = std::max(1, o) | (std::max(1, op) << 16);
        occ[device & 63].store(o);
    }
    pass_per_sm = o & 0xFFFF;
    plan_per_sm = o >> 16;
    return TOPK_OK;
}

template <int DT, int NT>
static topk_status launch_batched(topk_ctx* ctx, const BatchArgs& b, cudaStream_t st) {
    constexpr int KW = Key<DT>::KW;
    topk_status rs;
    const int per_sm = batched_blocks_per_sm<DT, NT>(ctx->device, rs);
    if (rs != TOPK_OK) return rs;
    int pass_per_sm = 1, plan_per_sm = 1;
    if (b.split != WIDE_NONE && (rs = wide_setup<DT>(ctx->device, pass_per_sm, plan_per_sm)) != TOPK_OK) return rs;
    cudaError_t e = launch_dep(k_batch_order, 1, 1024, 0, st, b);
    if (e == cudaSuccess && b.split != WIDE_NONE) {
        e = launch_dep(k_wide_plan<DT>, ctx->sms * plan_per_sm, WIDE_PLAN_NT, sizeof(BatchSmem<KW, WIDE_PLAN_NT>), st,
                       b);
        if (e == cudaSuccess)
            e = launch_dep(k_wide_pass<DT>, ctx->sms * pass_per_sm, WIDE_NT, WideCfg<DT>::SMEM, st, b);
    }
    if (e == cudaSuccess) e = launch_dep(k_batched<DT, NT>, ctx->sms * per_sm, NT, sizeof(BatchSmem<KW, NT>), st, b);
    if (e != cudaSuccess) return cuda_status(e);
    count_launch(ctx, b.split != WIDE_NONE ? 4 : 2);
    return cuda_status(cudaGetLastError());
}

// Largest resident grid over the variants: the number of per-block states
// and candidate buffers the scratch must hold.
template <int DT> static int batched_max_grid(topk_ctx* ctx, topk_status& rs) {
    int m = 0;
    for (int v : {batched_blocks_per_sm<DT, 1024>(ctx->device, rs), batched_blocks_per_sm<DT, 512>(ctx->device, rs),
                  batched_blocks_per_sm<DT, 256>(ctx->device, rs)})
        m = std::max(m, v);
    return ctx->sms * m;
}

// Scratch regions of one batched launch over `rows` rows with `grid` blocks
// (and, with wide rows, the per-row arrays and the candidate pool).
struct BatchCarve {
    size_t order, queue, states, cand;
    size_t wide, words, tile_pre, done, rstate, rcand, pool_next, pool;
};
template <int DT> static Carve batch_carve(u32 rows, int grid, bool wide, BatchCarve& bc) {
    typedef typename Key<DT>::key_t key_t;
    Carve cv;
    bc.order = cv.take(4ull * rows);
    bc.queue = cv.take(256);
    bc.states = cv.take(sizeof(SelState) * (size_t)grid);
    bc.cand = cv.take((size_t)grid * 2 * BATCH_CAP * (sizeof(key_t) + 4));
    if (wide) {
        bc.wide = cv.take(4ull * rows);
        bc.words = cv.take(256);
        bc.tile_pre = cv.take(8ull * (rows + 1));
        bc.done = cv.take(4ull * rows);
        bc.rstate = cv.take(sizeof(SelState) * (size_t)rows);
        bc.rcand = cv.take(8ull * rows);
        bc.pool_next = cv.take(256);
        bc.pool = cv.take(((WIDE_POOL_PAIRS * sizeof(key_t) + 255) & ~(size_t)255) + WIDE_POOL_PAIRS * 4);
    }
    return cv;
}

template <int DT>
static topk_status run_batched(topk_ctx* ctx, BatchArgs b, int threads, cudaStream_t st) {
    typedef typename Key<DT>::key_t key_t;
    constexpr int KW = Key<DT>::KW;
    topk_status rs = TOPK_OK;
    const int grid = batched_max_grid<DT>(ctx, rs);
    if (rs != TOPK_OK) return rs;
    const u32 cap = threads == 256 ? BatchVariant<KW, 256>::CAP
                                   : threads == 512 ? BatchVariant<KW, 512>::CAP : BatchVariant<KW, 1024>::CAP;
    b.finish_T = std::min(b.finish_T, cap);
    b.sample = std::min(b.sample, cap);
    b.key_bytes = (u32)sizeof(typename Key<DT>::raw_t);
    if (b.row_keys != nullptr) b.split = WIDE_NONE;
    if (b.split != WIDE_NONE) b.split = std::max(b.split, b.finish_T); // a wide row has more than T keys
    const bool wide = b.split != WIDE_NONE;
    BatchCarve bc;
    const Carve cv = batch_carve<DT>(b.rows, grid, wide, bc);
    rs = ensure_scratch(ctx, cv.off);
    if (rs != TOPK_OK) return rs;
    char* base = static_cast<char*>(ctx->scratch.base);
    b.order = reinterpret_cast<u32*>(base + bc.order);
    b.queue = reinterpret_cast<u32*>(base + bc.queue);
    b.states = reinterpret_cast<SelState*>(base + bc.states);
    b.cand = base + bc.cand;
    if (wide) {
        b.wide = reinterpret_cast<u32*>(base + bc.wide);
        b.words = reinterpret_cast<u32*>(base + bc.words);
        b.tile_pre = reinterpret_cast<u64*>(base + bc.tile_pre);
        b.done = reinterpret_cast<u32*>(base + bc.done);
        b.rstate = reinterpret_cast<SelState*>(base + bc.rstate);
        b.rcand = reinterpret_cast<u64*>(base + bc.rcand);
        b.pool_next = reinterpret_cast<u64*>(base + bc.pool_next);
        b.pool = base + bc.pool;
        b.pool_pairs = WIDE_POOL_PAIRS;
    }
    if (threads == 256) return launch_batched<DT, 256>(ctx, b, st);
    if (threads == 512) return launch_batched<DT, 512>(ctx, b, st);
    return launch_batched<DT, 1024>(ctx, b, st);
}

static topk_status run_batched_dt(topk_ctx* ctx, topk_dtype dtype, const BatchArgs& b, int threads,
                                  cudaStream_t st) {
    switch (dtype) {
    case TOPK_U32: return run_batched<DT_U32>(ctx, b, threads, st);
    case TOPK_I32: return run_batched<DT_I32>(ctx, b, threads, st);
    case TOPK_F32: return run_batched<DT_F32>(ctx, b, threads, st);
    case TOPK_BF16: return run_batched<DT_BF16>(ctx, b, threads, st);
    case TOPK_U64: return run_batched<DT_U64>(ctx, b, threads, st);
    default: return TOPK_EINVAL;
    }
}

// Rows given by device pointer arrays (serving).  `ptrs` is one device
// block laid out as: row_keys[rows], row_out_keys[rows], row_out_idx[rows],
// row_kth_key[rows], row_kth_idx[rows] (pointers), row_n[rows], row_k[rows].
topk_status batched_by_pointers(topk_ctx* ctx, topk_dtype dtype, u32 rows, const void* ptrs, cudaStream_t st) {
    const char* p = static_cast<const char*>(ptrs);
    BatchArgs b{};
    b.rows = rows;
    b.row_keys = reinterpret_cast<const void* const*>(p);
    b.row_out_keys = reinterpret_cast<void* const*>(p + 8ull * rows);
    b.row_out_idx = reinterpret_cast<u32* const*>(p + 16ull * rows);
    b.row_kth_key = reinterpret_cast<void* const*>(p + 24ull * rows);
    b.row_kth_idx = reinterpret_cast<u32* const*>(p + 32ull * rows);
    b.row_n = reinterpret_cast<const u64*>(p + 40ull * rows);
    b.row_k = reinterpret_cast<const u32*>(p + 48ull * rows);
    b.split = WIDE_NONE; // rows are short (at most BATCH_ROW_MAX keys)
    b.seed = 0xA4093822299F31D0ull;
    b.parts = 16;
    b.z = 4.0f;
    b.flags = 0;
    b.err = ctx->d_err;
    ctx->last_kind = LAST_BATCHED;
    // the context's tuned setting for this dtype and row count, else the
    // setting the tuner picks for batches of short rows
    int threads = 256;
    b.sample = 1024;
    b.finish_T = dtype == TOPK_U64 ? Lim<64>::ELEMS : Lim<32>::ELEMS;
    auto it = ctx->tuned.find({(int)dtype, rows ? 63 - __builtin_clzll((u64)rows) : 0});
    if (it != ctx->tuned.end()) {
        threads = (int)it->second.block_threads;
        b.sample = it->second.sample_size;
        b.finish_T = it->second.finish_threshold;
    }
    return run_batched_dt(ctx, dtype, b, threads, st);
}

static int log2_floor(u64 v) { return v ? 63 - __builtin_clzll(v) : 0; }

template <int DT> static topk_status batched_reserve_dt(topk_ctx* ctx, uint32_t rows) {
    topk_status rs = TOPK_OK;
    const int grid = batched_max_grid<DT>(ctx, rs);
    if (rs != TOPK_OK) return rs;
    BatchCarve bc;
    return ensure_scratch(ctx, batch_carve<DT>(rows, grid, false, bc).off);
}

topk_status batched_reserve(topk_ctx* ctx, topk_dtype dtype, uint32_t rows) {
    if (cudaSetDevice(ctx->device) != cudaSuccess) return TOPK_ECUDA;
    switch (dtype) {
    case TOPK_U32: return batched_reserve_dt<DT_U32>(ctx, rows);
    case TOPK_I32: return batched_reserve_dt<DT_I32>(ctx, rows);
    case TOPK_F32: return batched_reserve_dt<DT_F32>(ctx, rows);
    case TOPK_BF16: return batched_reserve_dt<DT_BF16>(ctx, rows);
    case TOPK_U64: return batched_reserve_dt<DT_U64>(ctx, rows);
    default: return TOPK_EINVAL;
    }
}

// Arguments of one topk_select_batched call (after validation) with the
// settings of `p`; `threads` receives the block size.
static BatchArgs batch_args(topk_ctx* ctx, const void* d_keys, const uint64_t* d_row_off, const uint32_t* d_row_k,
                            uint32_t rows, topk_dtype dtype, void* d_out_keys, uint32_t* d_out_idx,
                            const uint64_t* d_out_off, void* d_kth_keys, uint32_t* d_kth_idx, const topk_params& p,
                            int& threads) {
    BatchArgs b{};
    b.keys = d_keys;
    b.row_off = d_row_off;
    b.row_k = d_row_k;
    b.rows = rows;
    b.out_keys = d_out_keys;
    b.out_idx = d_out_idx;
    b.out_off = d_out_off;
    b.kth_keys = d_kth_keys;
    b.kth_idx = d_kth_idx;
    b.seed = p.seed ? p.seed : 0xA4093822299F31D0ull;
    b.parts = p.partitions ? p.partitions : 16;
    const u32 elems = dtype == TOPK_U64 ? Lim<64>::ELEMS : Lim<32>::ELEMS;
    b.sample = p.sample_size ? std::min<u32>(std::max<u32>(p.sample_size, 64), elems) : BATCH_SAMPLE;
    b.finish_T = p.finish_threshold ? std::min<u32>(std::max<u32>(p.finish_threshold, 64), elems) : elems;
    b.z = p.delta_factor > 0.f ? p.delta_factor : 4.0f;
    b.flags = p.flags;
    b.err = ctx->d_err;
    b.split = p.split_rows ? p.split_rows : WIDE_SPLIT;
    threads = p.block_threads == 256 || p.block_threads == 512 ? (int)p.block_threads : 1024;
    return b;
}

static bool batch_ptrs_ok(topk_ctx* ctx, const void* d_keys, const uint64_t* d_row_off, const uint32_t* d_row_k,
                          uint32_t rows, topk_dtype dtype, void* d_out_keys, uint32_t* d_out_idx,
                          const uint64_t* d_out_off, void* d_kth_keys, uint32_t* d_kth_idx) {
    if (!ctx || !d_keys || !d_row_off || !d_row_k || !d_out_keys || !d_out_idx || !d_out_off || !d_kth_keys ||
        !d_kth_idx || rows == 0)
        return false;
    const int w = dtype_bytes(dtype);
    if (w == 0) return false;
    return reinterpret_cast<uintptr_t>(d_keys) % (uintptr_t)w == 0 &&
           reinterpret_cast<uintptr_t>(d_out_keys) % (uintptr_t)w == 0;
}

} // namespace topk

using namespace topk;

extern "C" topk_status topk_select_batched(topk_ctx* ctx, const void* d_keys, const uint64_t* d_row_off,
                                           const uint32_t* d_row_k, uint32_t rows, topk_dtype dtype,
                                           void* d_out_keys, uint32_t* d_out_idx, const uint64_t* d_out_off,
                                           void* d_kth_keys, uint32_t* d_kth_idx, const topk_params* params,
                                           void* stream) {
    if (!batch_ptrs_ok(ctx, d_keys, d_row_off, d_row_k, rows, dtype, d_out_keys, d_out_idx, d_out_off, d_kth_keys,
                       d_kth_idx))
        return TOPK_EINVAL;
    if (params && (params->flags & TOPK_FLAG_LARGEST)) return TOPK_EINVAL; // k smallest only
    if (cudaSetDevice(ctx->device) != cudaSuccess) return TOPK_ECUDA;
    topk_params p{};
    if (params) p = *params;
    if (p.block_threads == 0 && p.sample_size == 0 && p.finish_threshold == 0 && p.split_rows == 0) {
        auto it = ctx->tuned.find({(int)dtype, log2_floor(rows)});
        if (it != ctx->tuned.end()) {
            p.block_threads = it->second.block_threads;
            p.sample_size = it->second.sample_size;
            p.finish_threshold = it->second.finish_threshold;
            p.split_rows = it->second.split_rows;
        }
    }
    int threads = 1024;
    const BatchArgs b = batch_args(ctx, d_keys, d_row_off, d_row_k, rows, dtype, d_out_keys, d_out_idx, d_out_off,
                                   d_kth_keys, d_kth_idx, p, threads);
    ctx->last_kind = LAST_BATCHED;
    return run_batched_dt(ctx, dtype, b, threads, static_cast<cudaStream_t>(stream));
}

extern "C" topk_status topk_tune_batched(topk_ctx* ctx, const void* d_keys, const uint64_t* d_row_off,
                                         const uint32_t* d_row_k, uint32_t rows, topk_dtype dtype, void* d_out_keys,
                                         uint32_t* d_out_idx, const uint64_t* d_out_off, void* d_kth_keys,
                                         uint32_t* d_kth_idx, const topk_params* base, topk_params* best,
                                         void* stream) {
    if (!batch_ptrs_ok(ctx, d_keys, d_row_off, d_row_k, rows, dtype, d_out_keys, d_out_idx, d_out_off, d_kth_keys,
                       d_kth_idx))
        return TOPK_EINVAL;
    if (base && (base->flags & TOPK_FLAG_LARGEST)) return TOPK_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return TOPK_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    topk_params b0{};
    if (base) b0 = *base;
    const u32 full = dtype == TOPK_U64 ? Lim<64>::ELEMS : Lim<32>::ELEMS;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return TOPK_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return TOPK_ECUDA;
    }
    topk_status rs = TOPK_OK;
    topk_params choice = b0;
    float best_ms = 0.f;
    bool have = false;
    for (u32 threads : {256u, 512u, 1024u}) {
        const u32 cap = threads == 1024 ? full : threads == 512 ? full / 2 : full / 4;
        for (u32 sample : {512u, 1024u, 2048u, 4096u}) {
            for (u32 T : {cap, cap / 2}) {
                topk_params p = b0;
                p.block_threads = threads;
                p.sample_size = std::min(sample, cap);
                p.finish_threshold = T;
                int nt = 1024;
                const BatchArgs b = batch_args(ctx, d_keys, d_row_off, d_row_k, rows, dtype, d_out_keys, d_out_idx,
                                               d_out_off, d_kth_keys, d_kth_idx, p, nt);
                float ms = 0.f;
                for (int rep = 0; rep < 4 && rs == TOPK_OK; ++rep) { // one warm-up, best of three
                    if (cudaEventRecord(e0, st) != cudaSuccess) rs = TOPK_ECUDA;
                    if (rs == TOPK_OK) rs = run_batched_dt(ctx, dtype, b, nt, st);
                    if (rs == TOPK_OK && cudaEventRecord(e1, st) != cudaSuccess) rs = TOPK_ECUDA;
                    if (rs == TOPK_OK && cudaEventSynchronize(e1) != cudaSuccess) rs = TOPK_ECUDA;
                    float t = 0.f;
                    if (rs == TOPK_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rs = TOPK_ECUDA;
                    if (rs == TOPK_OK && rep > 0) ms = rep == 1 ? t : std::min(ms, t);
                }
                if (rs == TOPK_OK) rs = topk_status_sync(ctx, stream);
                if (rs != TOPK_OK) break;
                if (!have || ms < best_ms) {
                    best_ms = ms;
                    choice = p;
                    have = true;
                }
            }
            if (rs != TOPK_OK) break;
        }
        if (rs != TOPK_OK) break;
    }
    // then the split length of wide rows, with the chosen block settings
    if (rs == TOPK_OK) {
        const topk_params blockwise = choice;
        for (u32 split : {1u << 13, 1u << 15, 1u << 17, WIDE_NONE}) {
            topk_params p = blockwise;
            p.split_rows = split;
            int nt = 1024;
            const BatchArgs b = batch_args(ctx, d_keys, d_row_off, d_row_k, rows, dtype, d_out_keys, d_out_idx,
                                           d_out_off, d_kth_keys, d_kth_idx, p, nt);
            float ms = 0.f;
            for (int rep = 0; rep < 4 && rs == TOPK_OK; ++rep) {
                if (cudaEventRecord(e0, st) != cudaSuccess) rs = TOPK_ECUDA;
                if (rs == TOPK_OK) rs = run_batched_dt(ctx, dtype, b, nt, st);
                if (rs == TOPK_OK && cudaEventRecord(e1, st) != cudaSuccess) rs = TOPK_ECUDA;
                if (rs == TOPK_OK && cudaEventSynchronize(e1) != cudaSuccess) rs = TOPK_ECUDA;
                float t = 0.f;
                if (rs == TOPK_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rs = TOPK_ECUDA;
                if (rs == TOPK_OK && rep > 0) ms = rep == 1 ? t : std::min(ms, t);
            }
            if (rs == TOPK_OK) rs = topk_status_sync(ctx, stream);
            if (rs != TOPK_OK) break;
            if (ms < best_ms) {
                best_ms = ms;
                choice = p;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs != TOPK_OK) return rs;
    ctx->tuned[{(int)dtype, log2_floor(rows)}] = choice;
    if (best) *best = choice;
    // leave the outputs as the chosen setting computes them
    int nt = 1024;
    const BatchArgs b = batch_args(ctx, d_keys, d_row_off, d_row_k, rows, dtype, d_out_keys, d_out_idx, d_out_off,
                                   d_kth_keys, d_kth_idx, choice, nt);
    ctx->last_kind = LAST_BATCHED;
    rs = run_batched_dt(ctx, dtype, b, nt, st);
    return rs == TOPK_OK ? topk_status_sync(ctx, stream) : rs;
}

extern "C" topk_status topk_tuning_save(topk_ctx* ctx, const char* path) {
    if (!ctx || !path) return TOPK_EINVAL;
    FILE* f = std::fopen(path, "w");
    if (!f) return TOPK_ECUDA;
    bool ok = std::fprintf(f, "topk-tuning 2\n") > 0;
    for (const auto& e : ctx->tuned)
        ok = ok && std::fprintf(f, "%s\t%d\t%d\t%u\t%u\t%u\t%u\n", ctx->device_name.c_str(), e.first.first,
                                e.first.second, e.second.block_threads, e.second.sample_size,
                                e.second.finish_threshold, e.second.split_rows) > 0;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? TOPK_OK : TOPK_ECUDA;
}

extern "C" topk_status topk_tuning_load(topk_ctx* ctx, const char* path) {
    if (!ctx || !path) return TOPK_EINVAL;
    FILE* f = std::fopen(path, "r");
    if (!f) return TOPK_EINVAL;
    char line[512];
    topk_status rs = TOPK_OK;
    // version 1 files have no split column (split chosen automatically)
    int version = 0;
    if (!std::fgets(line, sizeof line, f) || std::sscanf(line, "topk-tuning %d", &version) != 1 ||
        (version != 1 && version != 2))
        rs = TOPK_EINVAL;
    std::map<std::pair<int, int>, topk_params> add;
    while (rs == TOPK_OK && std::fgets(line, sizeof line, f)) {
        char* tab = std::strchr(line, '\t');
        if (!tab) {
            rs = TOPK_EINVAL;
            break;
        }
        const std::string name(line, (size_t)(tab - line));
        int dt = 0, bucket = 0;
        unsigned th = 0, sample = 0, T = 0, split = 0;
        const int want = version == 2 ? 6 : 5;
        if (std::sscanf(tab + 1, "%d\t%d\t%u\t%u\t%u\t%u", &dt, &bucket, &th, &sample, &T, &split) != want ||
            dt < 0 || dt > 4 || (th != 256 && th != 512 && th != 1024)) {
            rs = TOPK_EINVAL;
            break;
        }
        if (name != ctx->device_name) continue;
        topk_params p{};
        p.block_threads = th;
        p.sample_size = sample;
        p.finish_threshold = T;
        p.split_rows = split;
        add[{dt, bucket}] = p;
    }
    std::fclose(f);
    if (rs == TOPK_OK)
        for (const auto& e : add) ctx->tuned[e.first] = e.second;
    return rs;
}
