// internal.h — host-side context of libtopk (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <utility>
#include <cuda_runtime.h>

#include "../../include/topk.h"

namespace topk {

// One device allocation carved into regions per call; grown on demand.
struct Scratch {
    void* base = nullptr;
    size_t bytes = 0;
};

// Per-call region layout of the scratch block (byte offsets, 256-aligned).
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t at = off;
        off += (bytes + 255) & ~(size_t)255;
        return at;
    }
};

enum LastKind { LAST_NONE = 0, LAST_SELECT = 1, LAST_RUNS = 2, LAST_BATCHED = 3 };

} // namespace topk

struct topk_ctx {
    int device = 0;
    int sms = 0;
    topk::Scratch scratch;
    topk::Scratch freq;            // top-k most frequent objects: hash table and candidates
    topk::Scratch aux;             // outputs that a call forms but does not return (topk_select_kth)
    uint32_t* d_err = nullptr;     // first device error (latched), own allocation
    uint32_t* d_counter = nullptr; // last-block-done counters (zero between calls)
    void* d_state = nullptr;       // selection state (SelState or RunsState)
    int last_kind = topk::LAST_NONE;
    std::string device_name;
    // autotuned batched settings by (dtype, floor(log2(rows)))
    std::map<std::pair<int, int>, topk_params> tuned;
    topk_stats host_stats{};
    // measurement hooks
    bool profile = false;
    uint64_t launches = 0;
    uint64_t passes = 0;
    double pass_ms = 0.0;
    static constexpr int MAX_EVENTS = 256;
    cudaEvent_t ev[MAX_EVENTS][2] = {};
    int ev_used = 0;
};

namespace topk {

// Grows the context scratch to at least `bytes` (synchronising the device
// when an old block has to be released).
topk_status ensure_scratch(topk_ctx* ctx, size_t bytes);

// Measurement hooks: count a launch; bracket the first-level pass.
inline void count_launch(topk_ctx* ctx, uint64_t n = 1) {
    if (ctx->profile) ctx->launches += n;
}
void profile_pass_begin(topk_ctx* ctx, cudaStream_t st);
void profile_pass_end(topk_ctx* ctx, cudaStream_t st);

// Records a CUDA error; returns TOPK_ECUDA when `e` is not cudaSuccess.
topk_status cuda_status(cudaError_t e);

int dtype_bytes(topk_dtype dt);

// Kernel launch with programmatic stream serialization: the kernel's blocks
// may become resident before the previous kernel on the stream has ended;
// every kernel launched this way waits for its predecessor's grid on the
// device (grid_dep_wait in common.cuh) before touching its results.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Counters of the last sorted-runs call on the context (rounds).
topk_status runs_last_stats(topk_ctx* ctx, topk_stats* out);

// Batched selection with rows given by device pointer arrays (serving).
topk_status batched_by_pointers(topk_ctx* ctx, topk_dtype dtype, uint32_t rows, const void* ptrs,
                                cudaStream_t st);
constexpr uint64_t BATCH_ROW_MAX = 1ull << 18; // longest row the batched kernel takes
// Grows the context's scratch for a batched launch of up to `rows` rows.
topk_status batched_reserve(topk_ctx* ctx, topk_dtype dtype, uint32_t rows);

} // namespace topk
