// ctx.cu — context lifetime, scratch memory, latched device status,
// statistics and the Philox diagnostic of libtopk.
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace topk {

topk_status cuda_status(cudaError_t e) { return e == cudaSuccess ? TOPK_OK : TOPK_ECUDA; }

int dtype_bytes(topk_dtype dt) {
    switch (dt) {
    case TOPK_U32:
    case TOPK_I32:
    case TOPK_F32: return 4;
    case TOPK_BF16: return 2;
    case TOPK_U64: return 8;
    default: return 0;
    }
}

topk_status ensure_scratch(topk_ctx* ctx, size_t bytes) {
    if (ctx->scratch.bytes >= bytes) return TOPK_OK;
    if (ctx->scratch.base) {
        // work of earlier calls may still read the old block
        if (cudaDeviceSynchronize() != cudaSuccess) return TOPK_ECUDA;
        cudaFree(ctx->scratch.base);
        ctx->scratch.base = nullptr;
        ctx->scratch.bytes = 0;
    }
    size_t want = bytes + bytes / 4; // headroom against repeated growth
    void* p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return TOPK_ENOMEM;
        }
        want = bytes;
    }
    ctx->scratch.base = p;
    ctx->scratch.bytes = want;
    return TOPK_OK;
}

static void drain_events(topk_ctx* ctx) {
    for (int i = 0; i < ctx->ev_used; ++i) {
        float ms = 0.f;
        if (cudaEventSynchronize(ctx->ev[i][1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, ctx->ev[i][0], ctx->ev[i][1]) == cudaSuccess) {
            ctx->pass_ms += ms;
            ctx->passes += 1;
        }
    }
    ctx->ev_used = 0;
}

void profile_pass_begin(topk_ctx* ctx, cudaStream_t st) {
    if (!ctx->profile) return;
    if (ctx->ev_used == topk_ctx::MAX_EVENTS) drain_events(ctx);
    cudaEvent_t* e = ctx->ev[ctx->ev_used];
    if (!e[0]) {
        cudaEventCreate(&e[0]);
        cudaEventCreate(&e[1]);
    }
    cudaEventRecord(e[0], st);
}

void profile_pass_end(topk_ctx* ctx, cudaStream_t st) {
    if (!ctx->profile) return;
    cudaEventRecord(ctx->ev[ctx->ev_used][1], st);
    ctx->ev_used++;
}

__global__ void k_philox(u32 c0, u32 c1, u32 c2, u32 c3, u32 k0, u32 k1, u32* out, u32 count) {
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const Philox4 r = philox4x32_10(c0 + i, c1, c2, c3, k0, k1);
    out[4 * i + 0] = r.v[0];
    out[4 * i + 1] = r.v[1];
    out[4 * i + 2] = r.v[2];
    out[4 * i + 3] = r.v[3];
}

// A pipeline wait that nothing completes (an mbarrier expecting one arrival
// that never comes), bounded by limit_ns: the same bounded wait every bulk
// copy pipeline uses, so this exercises its expiry path, which latches
// TOPK_ETIMEOUT and returns without a fault.
__global__ void k_wait_expire(u64 limit_ns, u32* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool done = mbar_wait_bounded(&bar, 0, limit_ns);
    if (!done && threadIdx.x == 0) atomicCAS(err, 0u, (u32)TOPK_ETIMEOUT);
}

} // namespace topk

using namespace topk;

extern "C" {

topk_status topk_ctx_create(topk_ctx** out, int device) {
    if (!out) return TOPK_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return TOPK_ECUDA;
    }
    if (device < 0 || device >= count) return TOPK_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return TOPK_ECUDA;
    topk_ctx* c = new topk_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) c->device_name = prop.name;
    }
    // error word, block-done counters (64 slots) and the state: one
    // allocation, zeroed once; every kernel that uses a counter leaves it at
    // zero
    void* p = nullptr;
    const size_t bytes = 256 + 64 * sizeof(u32) + 4096;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return TOPK_ENOMEM;
    }
    cudaMemset(p, 0, bytes);
    c->d_err = static_cast<u32*>(p);
    c->d_counter = reinterpret_cast<u32*>(static_cast<char*>(p) + 256);
    c->d_state = static_cast<char*>(p) + 256 + 64 * sizeof(u32);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(p);
        delete c;
        return TOPK_ECUDA;
    }
    *out = c;
    return TOPK_OK;
}

topk_status topk_ctx_profile(topk_ctx* ctx, int enable) {
    if (!ctx) return TOPK_EINVAL;
    ctx->profile = enable != 0;
    return TOPK_OK;
}

topk_status topk_ctx_profile_read(topk_ctx* ctx, double* pass_ms, uint64_t* passes, uint64_t* launches,
                                  int reset) {
    if (!ctx) return TOPK_EINVAL;
    cudaSetDevice(ctx->device);
    drain_events(ctx);
    if (pass_ms) *pass_ms = ctx->pass_ms;
    if (passes) *passes = ctx->passes;
    if (launches) *launches = ctx->launches;
    if (reset) {
        ctx->pass_ms = 0.0;
        ctx->passes = 0;
        ctx->launches = 0;
    }
    return TOPK_OK;
}

void topk_ctx_destroy(topk_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (int i = 0; i < topk_ctx::MAX_EVENTS; ++i)
        for (int j = 0; j < 2; ++j)
            if (ctx->ev[i][j]) cudaEventDestroy(ctx->ev[i][j]);
    if (ctx->scratch.base) cudaFree(ctx->scratch.base);
    if (ctx->freq.base) cudaFree(ctx->freq.base);
    if (ctx->aux.base) cudaFree(ctx->aux.base);
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
}

topk_status topk_status_sync(topk_ctx* ctx, void* stream) {
    if (!ctx) return TOPK_EINVAL;
    cudaSetDevice(ctx->device);
    // the error word is read on the caller's stream (a plain cudaMemcpy would
    // go through the legacy default stream and wait for unrelated work)
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    u32 err = 0;
    if (cudaMemcpyAsync(&err, ctx->d_err, sizeof(u32), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return TOPK_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return TOPK_ECUDA;
    if (err != 0) {
        if (cudaMemsetAsync(ctx->d_err, 0, sizeof(u32), st) != cudaSuccess) return TOPK_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return TOPK_ECUDA;
    }
    return static_cast<topk_status>(err);
}

const char* topk_status_string(topk_status s) {
    switch (s) {
    case TOPK_OK: return "ok";
    case TOPK_EINVAL: return "invalid argument";
    case TOPK_ENOMEM: return "out of device memory";
    case TOPK_ECUDA: return "CUDA runtime error";
    case TOPK_ETIMEOUT: return "device wait timed out";
    case TOPK_EBUDGET: return "request exceeds memory budget";
    case TOPK_EBUSY: return "server busy";
    case TOPK_EINTERNAL: return "selection did not converge";
    default: return "unknown status";
    }
}

topk_status topk_debug_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                              uint32_t k1, uint32_t* d_out, uint32_t count) {
    if (!d_out || count == 0) return TOPK_EINVAL;
    k_philox<<<(count + 255) / 256, 256>>>(c0, c1, c2, c3, k0, k1, d_out, count);
    if (cudaGetLastError() != cudaSuccess) return TOPK_ECUDA;
    return cuda_status(cudaDeviceSynchronize());
}

topk_status topk_debug_wait_timeout(topk_ctx* ctx, uint32_t limit_us, void* stream) {
    if (!ctx || limit_us == 0 || limit_us > 1000000) return TOPK_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return TOPK_ECUDA;
    k_wait_expire<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>((u64)limit_us * 1000ull, ctx->d_err);
    return cuda_status(cudaGetLastError());
}

} // extern "C"
