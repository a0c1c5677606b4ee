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

#include "internal.h"
#include "select_block.cuh"

namespace topk {

constexpr u64 BATCH_CAP = 1ull << 16; // candidate pairs per buffer per block
constexpr u32 BATCH_SAMPLE = 2048;    // draws per level (rows are short)

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

template <int DT> __global__ void __launch_bounds__(BLK_NT) k_batched(BatchArgs b) {
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    constexpr int KW = K::KW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<BlockSmem<KW>*>(smem_raw);
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

template <int DT>
static topk_status run_batched(topk_ctx* ctx, BatchArgs b, cudaStream_t st) {
    typedef typename Key<DT>::key_t key_t;
    constexpr int KW = Key<DT>::KW;
    const int grid = ctx->sms; // one 1024-thread block per SM (shared memory)
    Carve cv;
    const size_t o_order = cv.take(4ull * b.rows);
    const size_t o_queue = cv.take(256);
    const size_t o_states = cv.take(sizeof(SelState) * (size_t)grid);
    const size_t o_cand = cv.take((size_t)grid * 2 * BATCH_CAP * (sizeof(key_t) + 4));
    topk_status rs = ensure_scratch(ctx, cv.off);
    if (rs != TOPK_OK) return rs;
    char* base = static_cast<char*>(ctx->scratch.base);
    b.order = reinterpret_cast<u32*>(base + o_order);
    b.queue = reinterpret_cast<u32*>(base + o_queue);
    b.states = reinterpret_cast<SelState*>(base + o_states);
    b.cand = base + o_cand;
    static std::atomic<uint64_t> attr_mask{0};
    const uint64_t bit = 1ull << (ctx->device & 63);
    if (!(attr_mask.load() & bit)) {
        if (cudaFuncSetAttribute(k_batched<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(BlockSmem<KW>)) != cudaSuccess)
            return TOPK_ECUDA;
        attr_mask.fetch_or(bit);
    }
    k_batch_order<<<1, 1024, 0, st>>>(b);
    k_batched<DT><<<grid, BLK_NT, sizeof(BlockSmem<KW>), st>>>(b);
    count_launch(ctx, 2);
    return cuda_status(cudaGetLastError());
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
    b.sample = BATCH_SAMPLE;
    b.finish_T = dtype == TOPK_U64 ? Lim<64>::ELEMS : Lim<32>::ELEMS;
    b.z = 4.0f;
    b.flags = 0;
    b.err = ctx->d_err;
    ctx->last_kind = LAST_BATCHED;
    switch (dtype) {
    case TOPK_U32: return run_batched<DT_U32>(ctx, b, st);
    case TOPK_I32: return run_batched<DT_I32>(ctx, b, st);
    case TOPK_F32: return run_batched<DT_F32>(ctx, b, st);
    case TOPK_BF16: return run_batched<DT_BF16>(ctx, b, st);
    case TOPK_U64: return run_batched<DT_U64>(ctx, b, st);
    default: return TOPK_EINVAL;
    }
}

} // namespace topk

using namespace topk;

extern "C" topk_status topk_select_batched(topk_ctx* ctx, const void* d_keys, const uint64_t* d_row_off,
                                           const uint32_t* d_row_k, uint32_t rows, topk_dtype dtype,
                                           void* d_out_keys, uint32_t* d_out_idx, const uint64_t* d_out_off,
                                           void* d_kth_keys, uint32_t* d_kth_idx, const topk_params* params,
                                           void* stream) {
    if (!ctx || !d_keys || !d_row_off || !d_row_k || !d_out_keys || !d_out_idx || !d_out_off || !d_kth_keys ||
        !d_kth_idx || rows == 0)
        return TOPK_EINVAL;
    const int w = dtype_bytes(dtype);
    if (w == 0) return TOPK_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_keys) % (uintptr_t)w || reinterpret_cast<uintptr_t>(d_out_keys) % (uintptr_t)w)
        return TOPK_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return TOPK_ECUDA;
    topk_params p{};
    if (params) p = *params;
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
    const u32 elems = w == 8 ? Lim<64>::ELEMS : Lim<32>::ELEMS;
    b.sample = p.sample_size ? std::min<u32>(std::max<u32>(p.sample_size, 64), elems) : BATCH_SAMPLE;
    b.finish_T = p.finish_threshold ? std::min<u32>(std::max<u32>(p.finish_threshold, 64), elems) : elems;
    b.z = p.delta_factor > 0.f ? p.delta_factor : 4.0f;
    b.flags = p.flags;
    b.err = ctx->d_err;
    ctx->last_kind = LAST_BATCHED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (dtype) {
    case TOPK_U32: return run_batched<DT_U32>(ctx, b, st);
    case TOPK_I32: return run_batched<DT_I32>(ctx, b, st);
    case TOPK_F32: return run_batched<DT_F32>(ctx, b, st);
    case TOPK_BF16: return run_batched<DT_BF16>(ctx, b, st);
    case TOPK_U64: return run_batched<DT_U64>(ctx, b, st);
    default: return TOPK_EINVAL;
    }
}
