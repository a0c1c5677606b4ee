// internal.h — host-side context of libtopk (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
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
    uint32_t* d_err = nullptr;     // first device error (latched), own allocation
    uint32_t* d_counter = nullptr; // last-block-done counters (zero between calls)
    void* d_state = nullptr;       // selection state (SelState or RunsState)
    int last_kind = topk::LAST_NONE;
    topk_stats host_stats{};
};

namespace topk {

// Grows the context scratch to at least `bytes` (synchronising the device
// when an old block has to be released).
topk_status ensure_scratch(topk_ctx* ctx, size_t bytes);

// Records a CUDA error; returns TOPK_ECUDA when `e` is not cudaSuccess.
topk_status cuda_status(cudaError_t e);

int dtype_bytes(topk_dtype dt);

} // namespace topk
