// batched.cu — topk_select_batched: many independent selections (rows of
// uneven length, each with its own k) in one persistent launch.
//
// The paper has no batched form; each row is the selection of Section 2
// (Algorithm "select") run by one thread block: sample, pivots, a block-wide
// partitioning pass into the block's candidate buffer, the branch, and the
// exact finish among at most T candidates (select_block.cuh).  Rows are
// handed out longest first from a device work queue, so the blocks that
// finish early take the short rows at the end.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>

#include "internal.h"
#include "select_block.cuh"

namespace topk {

constexpr u64 BATCH_CAP = 1ull << 16; // candidate pairs per buffer per block
constexpr u32 BATCH_SAMPLE = 2048;    // draws per level (rows are short)

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
};

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

template <int DT, int NT>
static topk_status launch_batched(topk_ctx* ctx, const BatchArgs& b, cudaStream_t st) {
    constexpr int KW = Key<DT>::KW;
    topk_status rs;
    const int per_sm = batched_blocks_per_sm<DT, NT>(ctx->device, rs);
    if (rs != TOPK_OK) return rs;
    cudaError_t e = launch_dep(k_batch_order, 1, 1024, 0, st, b);
    if (e == cudaSuccess) e = launch_dep(k_batched<DT, NT>, ctx->sms * per_sm, NT, sizeof(BatchSmem<KW, NT>), st, b);
    if (e != cudaSuccess) return cuda_status(e);
    count_launch(ctx, 2);
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

// Scratch regions of one batched launch over `rows` rows with `grid` blocks.
struct BatchCarve {
    size_t order, queue, states, cand;
};
template <int DT> static Carve batch_carve(u32 rows, int grid, BatchCarve& bc) {
    typedef typename Key<DT>::key_t key_t;
    Carve cv;
    bc.order = cv.take(4ull * rows);
    bc.queue = cv.take(256);
    bc.states = cv.take(sizeof(SelState) * (size_t)grid);
    bc.cand = cv.take((size_t)grid * 2 * BATCH_CAP * (sizeof(key_t) + 4));
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
    BatchCarve bc;
    const Carve cv = batch_carve<DT>(b.rows, grid, bc);
    const size_t o_order = bc.order, o_queue = bc.queue, o_states = bc.states, o_cand = bc.cand;
    rs = ensure_scratch(ctx, cv.off);
    if (rs != TOPK_OK) return rs;
    char* base = static_cast<char*>(ctx->scratch.base);
    b.order = reinterpret_cast<u32*>(base + o_order);
    b.queue = reinterpret_cast<u32*>(base + o_queue);
    b.states = reinterpret_cast<SelState*>(base + o_states);
    b.cand = base + o_cand;
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
    return ensure_scratch(ctx, batch_carve<DT>(rows, grid, bc).off);
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
    if (p.block_threads == 0 && p.sample_size == 0 && p.finish_threshold == 0) {
        auto it = ctx->tuned.find({(int)dtype, log2_floor(rows)});
        if (it != ctx->tuned.end()) {
            p.block_threads = it->second.block_threads;
            p.sample_size = it->second.sample_size;
            p.finish_threshold = it->second.finish_threshold;
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
        for (u32 sample : {1024u, 2048u, 4096u}) {
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
    bool ok = std::fprintf(f, "topk-tuning 1\n") > 0;
    for (const auto& e : ctx->tuned)
        ok = ok && std::fprintf(f, "%s\t%d\t%d\t%u\t%u\t%u\n", ctx->device_name.c_str(), e.first.first,
                                e.first.second, e.second.block_threads, e.second.sample_size,
                                e.second.finish_threshold) > 0;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? TOPK_OK : TOPK_ECUDA;
}

extern "C" topk_status topk_tuning_load(topk_ctx* ctx, const char* path) {
    if (!ctx || !path) return TOPK_EINVAL;
    FILE* f = std::fopen(path, "r");
    if (!f) return TOPK_EINVAL;
    char line[512];
    topk_status rs = TOPK_OK;
    if (!std::fgets(line, sizeof line, f) || std::strncmp(line, "topk-tuning 1", 13) != 0) rs = TOPK_EINVAL;
    std::map<std::pair<int, int>, topk_params> add;
    while (rs == TOPK_OK && std::fgets(line, sizeof line, f)) {
        char* tab = std::strchr(line, '\t');
        if (!tab) {
            rs = TOPK_EINVAL;
            break;
        }
        const std::string name(line, (size_t)(tab - line));
        int dt = 0, bucket = 0;
        unsigned th = 0, sample = 0, T = 0;
        if (std::sscanf(tab + 1, "%d\t%d\t%u\t%u\t%u", &dt, &bucket, &th, &sample, &T) != 5 || dt < 0 || dt > 4 ||
            (th != 256 && th != 512 && th != 1024)) {
            rs = TOPK_EINVAL;
            break;
        }
        if (name != ctx->device_name) continue;
        topk_params p{};
        p.block_threads = th;
        p.sample_size = sample;
        p.finish_threshold = T;
        add[{dt, bucket}] = p;
    }
    std::fclose(f);
    if (rs == TOPK_OK)
        for (const auto& e : add) ctx->tuned[e.first] = e.second;
    return rs;
}
