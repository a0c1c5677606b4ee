// select.cu — the C entry points of the selection of the k smallest of n
// unsorted keys (topk_select, topk_select_kth, topk_select_noalloc,
// topk_ctx_reserve, topk_last_stats).  The kernels and their host-side
// sequencing are in select_impl.cuh, instantiated per key type in
// select_<type>.cu.
#include "select_impl.cuh"

namespace topk {

TOPK_SELECT_TEMPLATES(extern, DT_U32)
TOPK_SELECT_TEMPLATES(extern, DT_I32)
TOPK_SELECT_TEMPLATES(extern, DT_F32)
TOPK_SELECT_TEMPLATES(extern, DT_BF16)
TOPK_SELECT_TEMPLATES(extern, DT_U64)

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64] = {};

// Device address of the array on the current device `dev` (set-up on first use).
static topk_status noalloc_base(int dev, int sms, char** out) {
    if (dev < 0 || dev >= 64) return TOPK_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        // the buffers must hold what the context path would allocate at the size limit
        if (candidate_capacity(NOALLOC_MAX_N, NOALLOC_MAX_N / 2, make_tuning<32>(nullptr, sms)) > NOALLOC_CAP ||
            candidate_capacity(NOALLOC_MAX_N, NOALLOC_MAX_N / 2, make_tuning<64>(nullptr, sms)) > NOALLOC_CAP)
            return TOPK_EINTERNAL;
        topk_status rs = noalloc_prepare_dt<DT_U32>(sms);
        if (rs == TOPK_OK) rs = noalloc_prepare_dt<DT_I32>(sms);
        if (rs == TOPK_OK) rs = noalloc_prepare_dt<DT_F32>(sms);
        if (rs == TOPK_OK) rs = noalloc_prepare_dt<DT_BF16>(sms);
        if (rs == TOPK_OK) rs = noalloc_prepare_dt<DT_U64>(sms);
        if (rs != TOPK_OK) return rs;
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

// Whether `p` is device (or managed) memory of device `dev`.
static bool on_device(const void* p, int dev) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
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
    if (params && (params->flags & TOPK_FLAG_LARGEST)) {
        switch (dtype) {
        case TOPK_U32: return run_select<DT_DESC + DT_U32>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
        case TOPK_I32: return run_select<DT_DESC + DT_I32>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
        case TOPK_F32: return run_select<DT_DESC + DT_F32>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
        case TOPK_BF16: return run_select<DT_DESC + DT_BF16>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
        case TOPK_U64: return run_select<DT_DESC + DT_U64>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
        default: return TOPK_EINVAL;
        }
    }
    switch (dtype) {
    case TOPK_U32: return run_select<DT_U32>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
    case TOPK_I32: return run_select<DT_I32>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
    case TOPK_F32: return run_select<DT_F32>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
    case TOPK_BF16: return run_select<DT_BF16>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
    case TOPK_U64: return run_select<DT_U64>(ctx, d_keys, n, k, d_out_keys, d_out_idx, d_kth_key, d_kth_idx, params, st);
    default: return TOPK_EINVAL;
    }
}

topk_status topk_select_kth(topk_ctx* ctx, const void* d_keys, uint64_t n, uint64_t k, topk_dtype dtype,
                            void* d_kth_key, uint32_t* d_kth_idx, const topk_params* params, void* stream) {
    if (!ctx || !d_keys || !d_kth_key || !d_kth_idx) return TOPK_EINVAL;
    const int w = dtype_bytes(dtype);
    if (w == 0) return TOPK_EINVAL;
    if (k < 1 || k > n || n > 0xFFFFFFFFull) return TOPK_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return TOPK_ECUDA;
    // the selected set goes to context-owned memory
    const size_t key_bytes = ((size_t)k * w + 255) & ~(size_t)255;
    const size_t need = key_bytes + (size_t)k * 4;
    Scratch& s = ctx->aux;
    if (s.bytes < need) {
        if (s.base) {
            if (cudaDeviceSynchronize() != cudaSuccess) return TOPK_ECUDA;
            cudaFree(s.base);
            s.base = nullptr;
            s.bytes = 0;
        }
        if (cudaMalloc(&s.base, need) != cudaSuccess) {
            cudaGetLastError();
            s.base = nullptr;
            return TOPK_ENOMEM;
        }
        s.bytes = need;
    }
    char* base = static_cast<char*>(s.base);
    return topk_select(ctx, d_keys, n, k, dtype, base, reinterpret_cast<uint32_t*>(base + key_bytes), d_kth_key,
                       d_kth_idx, params, stream);
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
    // every buffer must live on the current device, whose array and stream the call uses
    if (!on_device(d_keys, dev) || !on_device(d_out_keys, dev) || !on_device(d_out_idx, dev) ||
        !on_device(d_kth_key, dev) || !on_device(d_kth_idx, dev) || (d_status && !on_device(d_status, dev)))
        return TOPK_EINVAL;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TOPK_ECUDA;
    char* base = nullptr;
    topk_status rs = noalloc_base(dev, sms, &base);
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
    // the regions of run_select with the worst first bracket over k (k = n/2)
    // and the default tuning
    SelectCarve sc;
    if (w == 8) {
        const Tuning tu = make_tuning<64>(nullptr, ctx->sms);
        return ensure_scratch(ctx, select_carve<64>(candidate_capacity(n, std::max<u64>(2, n / 2), tu), ctx->sms, sc).off);
    }
    const Tuning tu = make_tuning<32>(nullptr, ctx->sms);
    return ensure_scratch(ctx, select_carve<32>(candidate_capacity(n, std::max<u64>(2, n / 2), tu), ctx->sms, sc).off);
}

topk_status topk_last_stats(topk_ctx* ctx, topk_stats* out) {
    if (!ctx || !out) return TOPK_EINVAL;
    *out = topk_stats{};
    if (ctx->last_kind == LAST_RUNS) return runs_last_stats(ctx, out);
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
