// frequent.cu — top-k most frequent objects on one GPU (Section 7):
// Algorithm PAC (Section 7.1: Bernoulli sample, count the sampled objects
// with hashing, select the k most frequently sampled) and Algorithm EC
// (Section 7.2: select the k* most frequently sampled, count those exactly
// over the whole input, select the k most frequent of them).
//
// One GPU is one PE: the paper's distributed hash table is a single
// open-addressing table in HBM, fed by block-local tables in shared memory
// (the local aggregation of Section 7.1's running-time lemma); the selections are
// topk_select calls on the table itself.  A table slot is one 64-bit word
// (0xFFFFFFFF - count) << 32 | object, so the table orders by count, larger
// first, equal counts by the smaller object, and an empty slot
// (all ones, count 0) sorts after every occupied one.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace topk {

constexpr u64 FQ_EMPTY = ~0ull;
constexpr u32 FQ_STREAM = 0x53414d50u; // counter word 2 of the sampling stream
constexpr int FQ_NT = 512;              // threads of the counting kernels
constexpr int FQ_QUADS = 4;             // 4-object groups per thread per tile
constexpr int FQ_LOCAL_LOG = 12;        // block-local table: 4096 slots (32 KB)
constexpr int FQ_LOCAL = 1 << FQ_LOCAL_LOG;
constexpr int FQ_LOCAL_PROBES = 4;
constexpr u32 FQ_EXACT_MAX = 4096;      // largest k* of the exact recount
constexpr u64 FQ_DEFAULT_DISTINCT = 1ull << 22;

// Finalizer of MurmurHash3 (public domain, A. Appleby): an avalanche mix of
// the object so that the table position behaves like a random function.
__host__ __device__ __forceinline__ u32 fq_mix(u32 x) {
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    x *= 0xc2b2ae35u;
    x ^= x >> 16;
    return x;
}

__device__ __forceinline__ u64 fq_word(u32 obj, u32 count) { return ((u64)(0xFFFFFFFFu - count) << 32) | obj; }

// Adds `c` occurrences of `obj` to the HBM table (linear probing from the
// hash's low bits).  False when neither the object nor a free slot turns up
// within FQ_TABLE_PROBES slots: the table holds more distinct objects than
// it was sized for (at the load it is sized for, at most one half, a probe
// sequence that long does not occur), so a call that overfills it ends in
// bounded time with TOPK_ENOMEM.
constexpr u32 FQ_TABLE_PROBES = 4096;

__device__ bool fq_table_add(u64* table, u32 mask, u32 obj, u32 c) {
    u32 h = fq_mix(obj) & mask;
    const u32 limit = mask < FQ_TABLE_PROBES ? mask + 1 : FQ_TABLE_PROBES;
    for (u32 probe = 0; probe < limit; ++probe) {
        u64* s = table + h;
        u64 w = __ldcg(s);
        if (w == FQ_EMPTY) {
            const u64 prev = atomicCAS(reinterpret_cast<unsigned long long*>(s), FQ_EMPTY, fq_word(obj, c));
            if (prev == FQ_EMPTY) return true;
            w = prev;
        }
        if ((u32)w == obj) {
            atomicAdd(reinterpret_cast<unsigned long long*>(s), (unsigned long long)(0ull - ((u64)c << 32)));
            return true;
        }
        h = (h + 1) & mask;
    }
    return false;
}

// Block-local table and per-warp queues of the counting kernel.  Objects
// claim slots of the local table until it is full and keep them (no flush
// before the end): the frequent objects, which appear early and often, are
// then counted in shared memory, and an object that finds neither itself
// nor a free slot within FQ_LOCAL_PROBES goes straight to the HBM table.
// The queue packs a warp's sampled objects so that every lane inserts one
// (at a sampling rate well below 1 most lanes of a quad sample nothing).
constexpr int FQ_QCAP = FQ_QUADS * 4 * 32;

struct FqLocal {
    u64 slot[FQ_LOCAL];
    u32 queue[FQ_NT / 32][FQ_QCAP];
    u32 warp_sum[FQ_NT / 32];
};

// One occurrence into the block-local table (probing from the hash's high
// bits, independent of the HBM table's position); false when neither the
// object nor a free slot is found within FQ_LOCAL_PROBES slots.
__device__ __forceinline__ bool fq_local_add(FqLocal& L, u32 obj) {
    u32 h = fq_mix(obj) >> (32 - FQ_LOCAL_LOG);
#pragma unroll 1
    for (int p = 0; p < FQ_LOCAL_PROBES; ++p) {
        u64 w = *reinterpret_cast<volatile u64*>(&L.slot[h]);
        if (w == FQ_EMPTY) {
            const u64 prev =
                atomicCAS(reinterpret_cast<unsigned long long*>(&L.slot[h]), FQ_EMPTY, fq_word(obj, 1));
            if (prev == FQ_EMPTY) return true;
            w = prev;
        }
        if ((u32)w == obj) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&L.slot[h]), (unsigned long long)(0ull - (1ull << 32)));
            return true;
        }
        h = (h + 1) & (FQ_LOCAL - 1);
    }
    return false;
}

struct FreqArgs {
    const u32* obj;
    u64 n;
    u32 thr;              // sampled iff Philox word < thr (unused when every object is)
    u32 seed_lo, seed_hi;
    u64* table;
    u32 mask;             // table slots - 1
    u64* sampled;         // sample size (zeroed before)
    u32* err;
};

// Moves every entry of the block-local table into the HBM table.  Each
// thread takes FQ_LOCAL / FQ_NT slots, four at a time, and reads their home
// positions in the HBM table at once; an object found at its home position
// costs one atomic add, the rest probe.
__device__ __forceinline__ void fq_flush(FqLocal& L, const FreqArgs& a) {
    constexpr int G = 4;
#pragma unroll 1
    for (u32 base = threadIdx.x; base < FQ_LOCAL; base += G * FQ_NT) {
        u64 mine[G], seen[G];
        u32 pos[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            mine[j] = L.slot[base + j * FQ_NT];
            pos[j] = fq_mix((u32)mine[j]) & a.mask;
        }
#pragma unroll
        for (int j = 0; j < G; ++j) seen[j] = mine[j] != FQ_EMPTY ? __ldcg(a.table + pos[j]) : FQ_EMPTY;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (mine[j] == FQ_EMPTY) continue;
            const u32 obj = (u32)mine[j], c = 0xFFFFFFFFu - (u32)(mine[j] >> 32);
            if (seen[j] != FQ_EMPTY && (u32)seen[j] == obj) {
                atomicAdd(reinterpret_cast<unsigned long long*>(a.table + pos[j]),
                          (unsigned long long)(0ull - ((u64)c << 32)));
            } else if (!fq_table_add(a.table, a.mask, obj, c)) {
                atomicCAS(a.err, 0u, (u32)TOPK_ENOMEM);
            }
        }
    }
}

__device__ __forceinline__ void fq_insert(FqLocal& L, const FreqArgs& a, u32 obj) {
    if (!fq_local_add(L, obj) && !fq_table_add(a.table, a.mask, obj, 1)) atomicCAS(a.err, 0u, (u32)TOPK_ENOMEM);
}

// Loads the FQ_QUADS quads of one tile (all loads in flight at once);
// FULL: the tile lies inside the objects and they are 16-byte aligned.
template <bool FULL, bool VEC>
__device__ __forceinline__ void fq_load_tile(const u32* obj, u64 n, u64 q0, uint4 (&x)[FQ_QUADS]) {
#pragma unroll
    for (int j = 0; j < FQ_QUADS; ++j) {
        const u64 q = q0 + (u64)j * FQ_NT;
        const u64 i0 = q * 4;
        if (FULL || (VEC && i0 + 4 <= n)) {
            x[j] = ld_stream(reinterpret_cast<const uint4*>(obj) + q);
        } else {
            x[j].x = i0 + 0 < n ? __ldcs(obj + i0 + 0) : 0u;
            x[j].y = i0 + 1 < n ? __ldcs(obj + i0 + 1) : 0u;
            x[j].z = i0 + 2 < n ? __ldcs(obj + i0 + 2) : 0u;
            x[j].w = i0 + 3 < n ? __ldcs(obj + i0 + 3) : 0u;
        }
    }
}

__device__ __forceinline__ u32 u4at(const uint4& v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }

// One tile: sample decisions for the thread's FQ_QUADS * 4 objects (bit
// 4j + e = object e of quad j); every sampled object is inserted, through
// the warp's queue unless every object is sampled.  Returns the number of
// objects this thread sampled.
template <bool ALL, bool FULL, bool VEC>
__device__ __forceinline__ u32 fq_tile(FqLocal& L, const FreqArgs& a, u64 q0, u32* queue, u32 lane) {
    uint4 x[FQ_QUADS];
    fq_load_tile<FULL, VEC>(a.obj, a.n, q0, x);
    u32 take = 0;
#pragma unroll
    for (int j = 0; j < FQ_QUADS; ++j) {
        const u64 q = q0 + (u64)j * FQ_NT;
        u32 t4 = 0xF;
        if (!ALL) {
            const Philox4 r = philox4x32_10((u32)q, (u32)(q >> 32), FQ_STREAM, 0u, a.seed_lo, a.seed_hi);
            t4 = (r.v[0] < a.thr ? 1u : 0u) | (r.v[1] < a.thr ? 2u : 0u) | (r.v[2] < a.thr ? 4u : 0u) |
                 (r.v[3] < a.thr ? 8u : 0u);
        }
        if (!FULL) {
            const u64 i0 = q * 4;
            t4 = i0 >= a.n ? 0u : i0 + 4 > a.n ? t4 & ((1u << (u32)(a.n - i0)) - 1u) : t4;
        }
        take |= t4 << (4 * j);
    }
    const u32 c = __popc(take);
    if (ALL) {
#pragma unroll
        for (int j = 0; j < FQ_QUADS; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (FULL || ((take >> (4 * j + e)) & 1u)) fq_insert(L, a, u4at(x[j], e));
        return c;
    }
    u32 incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (u32)o) incl += y;
    }
    const u32 total = __shfl_sync(0xffffffffu, incl, 31);
    u32 at = incl - c;
#pragma unroll
    for (int j = 0; j < FQ_QUADS; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if ((take >> (4 * j + e)) & 1u) queue[at++] = u4at(x[j], e);
    __syncwarp();
    for (u32 i = lane; i < total; i += 32) fq_insert(L, a, queue[i]);
    __syncwarp();
    return c;
}

// Sampling and counting (Section 7.1) in one pass: every block walks tiles
// of FQ_NT * FQ_QUADS * 4 objects; object i is sampled iff word i % 4 of
// Philox4x32-10 at counter (i / 4, FQ_STREAM) and the seed's key is below
// the threshold.  No block barrier until the final flush of the local
// table into the HBM table.
template <bool ALL, bool VEC>
__global__ void __launch_bounds__(FQ_NT, 3) k_freq_count(FreqArgs a) {
    extern __shared__ __align__(16) unsigned char fq_dyn[];
    FqLocal& L = *reinterpret_cast<FqLocal*>(fq_dyn);
    for (u32 s = threadIdx.x; s < FQ_LOCAL; s += FQ_NT) L.slot[s] = FQ_EMPTY;
    grid_dep_wait(); // the table was cleared by the previous operation
    __syncthreads();
    const u32 lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32* queue = L.queue[warp];
    const u64 quads = (a.n + 3) / 4;
    const u64 tile_quads = (u64)FQ_NT * FQ_QUADS;
    const u64 tiles = (quads + tile_quads - 1) / tile_quads;
    const u64 full_tiles = VEC ? (a.n / 4) / tile_quads : 0;
    u32 sampled = 0;
    for (u64 t = blockIdx.x; t < tiles; t += gridDim.x) {
        const u64 q0 = t * tile_quads + threadIdx.x;
        if (VEC && t < full_tiles) sampled += fq_tile<ALL, true, VEC>(L, a, q0, queue, lane);
        else sampled += fq_tile<ALL, false, VEC>(L, a, q0, queue, lane);
    }
    __syncthreads();
    fq_flush(L, a);
    // sample size: warp sums, then one atomic per block
    u32 w = sampled;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) L.warp_sum[warp] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 s = 0;
        for (int i = 0; i < FQ_NT / 32; ++i) s += L.warp_sum[i];
        atomicAdd(reinterpret_cast<unsigned long long*>(a.sampled), (unsigned long long)s);
    }
}

// Exact recount of the k* candidates (Section 7.2) over the whole input:
// the candidates sit in a shared-memory hash table of words
// (candidate number << 32 | object); every block counts its part and adds its counts to exact[] at
// the end.  The candidates are the most frequent objects, so many threads
// hit the same few counters: MODE 0 (k* <= FQ_PT_MAX) gives every thread
// its own counters (plain increments), MODE 1 (k* <= FQ_PW_MAX) every warp
// (shared-memory atomics within the warp only), MODE 2 one set per block.
constexpr u32 FQ_PT_MAX = 32;
constexpr int FQ_XQUADS = 4; // 4-object groups per thread per iteration (loads in flight)
constexpr u32 FQ_PW_MAX = 1024;

struct ExactArgs {
    const u32* obj;
    u64 n;
    const u64* cand; // k* table words: object in the low half
    u32 kstar;
    u32 log_slots;
    u32* exact;      // kstar counts (zeroed before)
};

__host__ __device__ inline size_t fq_exact_counters(int mode, u32 kstar) {
    return mode == 0 ? (size_t)kstar * FQ_NT : mode == 1 ? (size_t)kstar * (FQ_NT / 32) : (size_t)kstar;
}

// Position of an object in the recount's candidate table: one
// multiplication (the table holds at most a few thousand candidates and is
// at least four times larger, so a cheap hash keeps probes short).
__device__ __forceinline__ u32 fq_cand_pos(u32 v, u32 log_slots) { return (v * 0x2545F491u) >> (32 - log_slots); }

// Counts one object: a table word is (candidate number << 32) | object, an
// empty slot has a negative candidate number.
template <int MODE>
__device__ __forceinline__ void fq_recount_one(const u64* slot, u32 log_slots, u32* my, u32 v) {
    const u32 mask = (1u << log_slots) - 1;
    u32 h = fq_cand_pos(v, log_slots);
    u64 w = slot[h];
    int c = (int)(w >> 32);
    if (c >= 0 && (u32)w != v) {
        do {
            h = (h + 1) & mask;
            w = slot[h];
            c = (int)(w >> 32);
        } while (c >= 0 && (u32)w != v);
    }
    if (c >= 0) {
        if (MODE == 0) my[(u32)c * FQ_NT] += 1;
        else atomicAdd(&my[c], 1u);
    }
}

template <int MODE, bool VEC>
__global__ void __launch_bounds__(FQ_NT, 3) k_freq_exact(ExactArgs a) {
    extern __shared__ __align__(16) unsigned char fq_smem[];
    const u32 slots = 1u << a.log_slots;
    u64* slot = reinterpret_cast<u64*>(fq_smem);
    u32* cnt = reinterpret_cast<u32*>(slot + slots);
    const u32 ncnt = (u32)fq_exact_counters(MODE, a.kstar);
    for (u32 s = threadIdx.x; s < slots; s += FQ_NT) slot[s] = ~0ull;
    for (u32 c = threadIdx.x; c < ncnt; c += FQ_NT) cnt[c] = 0;
    grid_dep_wait(); // the candidates come from the previous selection
    __syncthreads();
    for (u32 c = threadIdx.x; c < a.kstar; c += FQ_NT) {
        const u32 o = (u32)a.cand[c];
        const u64 word = ((u64)c << 32) | o;
        u32 h = fq_cand_pos(o, a.log_slots);
        while (atomicCAS(reinterpret_cast<unsigned long long*>(&slot[h]), ~0ull, word) != ~0ull)
            h = (h + 1) & (slots - 1);
    }
    __syncthreads();
    // this thread's (MODE 0) or warp's (MODE 1) counters
    u32* my = MODE == 0 ? cnt + threadIdx.x : MODE == 1 ? cnt + (threadIdx.x >> 5) * a.kstar : cnt;
    const u64 quads = (a.n + 3) / 4;
    const u64 tile_quads = (u64)FQ_NT * FQ_XQUADS;
    const u64 full_tiles = VEC ? (a.n / 4) / tile_quads : 0;
    for (u64 t = blockIdx.x; t * tile_quads < quads; t += gridDim.x) {
        const u64 q0 = t * tile_quads + threadIdx.x;
        uint4 x[FQ_XQUADS];
        if (VEC && t < full_tiles) {
#pragma unroll
            for (int j = 0; j < FQ_XQUADS; ++j) x[j] = ld_stream(reinterpret_cast<const uint4*>(a.obj) + q0 + j * FQ_NT);
#pragma unroll
            for (int j = 0; j < FQ_XQUADS; ++j) {
                fq_recount_one<MODE>(slot, a.log_slots, my, x[j].x);
                fq_recount_one<MODE>(slot, a.log_slots, my, x[j].y);
                fq_recount_one<MODE>(slot, a.log_slots, my, x[j].z);
                fq_recount_one<MODE>(slot, a.log_slots, my, x[j].w);
            }
        } else {
            for (int j = 0; j < FQ_XQUADS; ++j) {
                const u64 i0 = (q0 + (u64)j * FQ_NT) * 4;
                for (int e = 0; e < 4; ++e)
                    if (i0 + e < a.n) fq_recount_one<MODE>(slot, a.log_slots, my, __ldcs(a.obj + i0 + e));
            }
        }
    }
    __syncthreads();
    if (MODE == 2) {
        for (u32 c = threadIdx.x; c < a.kstar; c += FQ_NT)
            if (cnt[c]) atomicAdd(&a.exact[c], cnt[c]);
        return;
    }
    // sum the private counters of each candidate: one warp per candidate
    const u32 lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u32 copies = MODE == 0 ? FQ_NT : FQ_NT / 32;
    for (u32 c = warp; c < a.kstar; c += FQ_NT / 32) {
        u32 sum = 0;
        for (u32 t = lane; t < copies; t += 32) sum += MODE == 0 ? cnt[c * FQ_NT + t] : cnt[t * a.kstar + c];
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0 && sum) atomicAdd(&a.exact[c], sum);
    }
}

// Table words of the candidates with their exact counts.
__global__ void k_freq_compose(const u64* cand, const u32* exact, u32 kstar, u64* out) {
    grid_dep_wait();
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kstar) out[i] = fq_word((u32)cand[i], exact[i]);
}

// Selected table words -> objects and counts; a selected empty slot means
// fewer than `need` distinct objects were sampled.
// Also writes the sample size: the sampler's cursor, or n when every
// object was taken.
__global__ void k_freq_decode(const u64* sel, const u64* kth, u32 k, u32* out_obj, u64* out_cnt, u32* err,
                              const u64* cursor, u64 all_n, u64* sample_size) {
    grid_dep_wait();
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && *kth == FQ_EMPTY) atomicCAS(err, 0u, (u32)TOPK_EINVAL);
    if (i == 0 && sample_size) *sample_size = cursor ? *cursor : all_n;
    if (i < k && out_obj) {
        const u64 w = sel[i];
        out_obj[i] = (u32)w;
        out_cnt[i] = 0xFFFFFFFFu - (u32)(w >> 32);
    }
}

__global__ void k_freq_check(const u64* kth, u32* err) {
    grid_dep_wait();
    if (threadIdx.x == 0 && *kth == FQ_EMPTY) atomicCAS(err, 0u, (u32)TOPK_EINVAL);
}

static topk_status plan(uint64_t n, const topk_freq_params* fp, double* rho_out, uint32_t* kstar_out) {
    if (!fp || n == 0 || fp->k == 0) return TOPK_EINVAL;
    if (fp->algorithm != TOPK_FREQ_PAC && fp->algorithm != TOPK_FREQ_EC) return TOPK_EINVAL;
    const bool ec = fp->algorithm == TOPK_FREQ_EC;
    const double k = fp->k;
    const double nn = (double)n;
    uint32_t kstar = fp->k;
    if (ec) {
        if (fp->kstar) {
            kstar = fp->kstar;
        } else {
            if (!(fp->epsilon > 0.0) || !(fp->delta > 0.0 && fp->delta < 1.0)) return TOPK_EINVAL;
            const double p = fp->pes ? fp->pes : 1;
            // k* = max(k, sqrt(2 log2(p) / p * ln(n / delta)) / eps)
            const double opt = std::ceil(std::sqrt(2.0 * std::log2(p) / p * std::log(nn / fp->delta)) / fp->epsilon);
            kstar = opt > k ? (opt >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)opt) : fp->k;
        }
        if (kstar < fp->k) return TOPK_EINVAL;
    }
    double rho = fp->rho;
    if (rho == 0.0) {
        if (!(fp->epsilon > 0.0) || !(fp->delta > 0.0 && fp->delta < 1.0)) return TOPK_EINVAL;
        const double e2 = fp->epsilon * fp->epsilon;
        double rho_n;
        if (!ec) {
            // expected sample size of equation sampleSize
            const double first = 3.0 / k * std::log(4.0 * nn / fp->delta);
            const double second = 2.0 * std::log(2.0 * k / fp->delta);
            rho_n = 4.0 / e2 * std::max(first, second);
        } else {
            rho_n = 2.0 / (e2 * (double)kstar) * std::log(nn / fp->delta); // Lemma "topkec"
        }
        rho = rho_n >= nn ? 1.0 : rho_n / nn;
    }
    if (!(rho > 0.0) || rho > 1.0) return TOPK_EINVAL;
    if (rho_out) *rho_out = rho;
    if (kstar_out) *kstar_out = kstar;
    return TOPK_OK;
}

static u32 ceil_log2(u64 x) {
    u32 l = 0;
    while ((1ull << l) < x) ++l;
    return l;
}

// Candidate table of the recount: at most one slot in eight used up to
// 2048 candidates (short probes for the many objects that are not
// candidates), 16384 slots above.
static u32 fq_exact_log_slots(u32 kstar) { return std::min<u32>(14, std::max<u32>(8, ceil_log2(8ull * kstar))); }

static topk_status ensure_freq(topk_ctx* ctx, size_t bytes) {
    Scratch& s = ctx->freq;
    if (s.bytes >= bytes) return TOPK_OK;
    if (s.base) {
        if (cudaDeviceSynchronize() != cudaSuccess) return TOPK_ECUDA;
        cudaFree(s.base);
        s.base = nullptr;
        s.bytes = 0;
    }
    if (cudaMalloc(&s.base, bytes) != cudaSuccess) {
        cudaGetLastError();
        s.base = nullptr;
        return TOPK_ENOMEM;
    }
    s.bytes = bytes;
    return TOPK_OK;
}

} // namespace topk

using namespace topk;

extern "C" {

topk_status topk_frequent_plan(uint64_t n, const topk_freq_params* fp, double* rho, uint32_t* kstar) {
    return plan(n, fp, rho, kstar);
}

topk_status topk_frequent(topk_ctx* ctx, const void* d_objects, uint64_t n, topk_dtype dtype,
                          const topk_freq_params* fp, uint32_t* d_out_obj, uint64_t* d_out_count,
                          uint64_t* d_sample_size, void* stream) {
    if (!ctx || !d_objects || !fp || !d_out_obj || !d_out_count) return TOPK_EINVAL;
    if (dtype != TOPK_U32 || n == 0 || n > 0xFFFFFFFEull) return TOPK_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_objects) % 4) return TOPK_EINVAL;
    double rho = 0.0;
    uint32_t kstar = 0;
    topk_status rs = plan(n, fp, &rho, &kstar);
    if (rs != TOPK_OK) return rs;
    const bool ec = fp->algorithm == TOPK_FREQ_EC;
    if (ec && kstar > FQ_EXACT_MAX) return TOPK_EINVAL;
    // distinct sampled objects are at most the sample size: bound it far
    // above its mean (a larger sample has negligible probability and would
    // only be reported as TOPK_ENOMEM) and by n
    const double mean = rho * (double)n;
    const u64 sample_bound = std::min<u64>(n, (u64)std::ceil(mean + 8.0 * std::sqrt(mean) + 1024.0));
    const u64 distinct =
        std::min<u64>(fp->max_distinct ? fp->max_distinct : FQ_DEFAULT_DISTINCT, sample_bound);
    const u32 log_cap = std::max<u32>(12, ceil_log2(2 * std::max<u64>(distinct, (u64)kstar)));
    if (log_cap > 31) return TOPK_EINVAL;
    const u64 cap = 1ull << log_cap;
    const u32 need = ec ? kstar : fp->k;
    if (need > cap) return TOPK_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return TOPK_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    const u64 thr = rho >= 1.0 ? (1ull << 32) : (u64)std::floor(std::ldexp(rho, 32));
    const bool all = thr >= (1ull << 32);

    Carve cv;
    const size_t o_table = cv.take(8 * cap);
    const size_t o_sel = cv.take(8ull * need), o_idx = cv.take(4ull * need), o_kth = cv.take(16);
    const size_t o_exact = cv.take(4ull * kstar), o_comp = cv.take(8ull * kstar);
    const size_t o_sel2 = cv.take(8ull * fp->k), o_idx2 = cv.take(4ull * fp->k), o_kth2 = cv.take(16);
    const size_t o_cursor = cv.take(8);
    rs = ensure_freq(ctx, cv.off);
    if (rs != TOPK_OK) return rs;
    char* base = static_cast<char*>(ctx->freq.base);
    u64* table = reinterpret_cast<u64*>(base + o_table);
    u64* sel = reinterpret_cast<u64*>(base + o_sel);
    u32* sel_idx = reinterpret_cast<u32*>(base + o_idx);
    u64* kth = reinterpret_cast<u64*>(base + o_kth);
    u32* kth_idx = reinterpret_cast<u32*>(base + o_kth + 8);
    u64* cursor = reinterpret_cast<u64*>(base + o_cursor); // sample size

    static std::atomic<uint64_t> count_attr{0};
    const uint64_t dbit = 1ull << (ctx->device & 63);
    if (!(count_attr.load() & dbit)) {
        for (auto kf : {k_freq_count<true, true>, k_freq_count<true, false>, k_freq_count<false, true>,
                        k_freq_count<false, false>})
            if (cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FqLocal)) !=
                cudaSuccess)
                return TOPK_ECUDA;
        count_attr.fetch_or(dbit);
    }

    // 1. sample and count (Section 7.1)
    cudaError_t e = cudaMemsetAsync(table, 0xFF, 8 * cap, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, 8, st);
    if (e != cudaSuccess) return cuda_status(e);
    const bool vec = reinterpret_cast<uintptr_t>(d_objects) % 16 == 0;
    FreqArgs a{};
    a.obj = static_cast<const u32*>(d_objects);
    a.n = n;
    a.thr = all ? 0u : (u32)thr;
    a.seed_lo = (u32)fp->seed;
    a.seed_hi = (u32)(fp->seed >> 32);
    a.table = table;
    a.mask = (u32)(cap - 1);
    a.sampled = cursor;
    a.err = ctx->d_err;
    auto kern = all ? (vec ? k_freq_count<true, true> : k_freq_count<true, false>)
                    : (vec ? k_freq_count<false, true> : k_freq_count<false, false>);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FQ_NT, sizeof(FqLocal));
    const u64 tile_objs = (u64)FQ_NT * FQ_QUADS * 4;
    const u64 tiles = (n + tile_objs - 1) / tile_objs;
    const int grid = (int)std::max<u64>(1, std::min<u64>(tiles, (u64)ctx->sms * std::max(per_sm, 1)));
    e = launch_dep(kern, grid, FQ_NT, sizeof(FqLocal), st, a);
    if (e != cudaSuccess) return cuda_status(e);
    count_launch(ctx);

    // 2. the `need` most frequently sampled objects: the smallest table words
    rs = topk_select(ctx, table, cap, need, TOPK_U64, sel, sel_idx, kth, kth_idx, nullptr, stream);
    if (rs != TOPK_OK) return rs;
    if (!ec) {
        e = launch_dep(k_freq_decode, (int)((fp->k + 255) / 256), 256, 0, st, (const u64*)sel, (const u64*)kth,
                       fp->k, d_out_obj, d_out_count, ctx->d_err, (const u64*)cursor,
                       (u64)n, d_sample_size);
        count_launch(ctx);
        return cuda_status(e);
    }
    // 3. EC: exact recount of the k* candidates (Section 7.2)
    e = launch_dep(k_freq_check, 1, 32, 0, st, (const u64*)kth, ctx->d_err);
    u32* exact = reinterpret_cast<u32*>(base + o_exact);
    if (e == cudaSuccess) e = cudaMemsetAsync(exact, 0, 4ull * kstar, st);
    if (e != cudaSuccess) return cuda_status(e);
    ExactArgs x{};
    x.obj = static_cast<const u32*>(d_objects);
    x.n = n;
    x.cand = sel;
    x.kstar = kstar;
    x.log_slots = fq_exact_log_slots(kstar);
    x.exact = exact;
    const int mode = kstar <= FQ_PT_MAX ? 0 : kstar <= FQ_PW_MAX ? 1 : 2;
    const size_t smem = (size_t)(1u << x.log_slots) * 8 + 4 * fq_exact_counters(mode, kstar);
    void (*exact_kernels[3][2])(ExactArgs) = {{k_freq_exact<0, false>, k_freq_exact<0, true>},
                                              {k_freq_exact<1, false>, k_freq_exact<1, true>},
                                              {k_freq_exact<2, false>, k_freq_exact<2, true>}};
    auto ek = exact_kernels[mode][vec ? 1 : 0];
    static std::atomic<uint64_t> attr_mask{0};
    const uint64_t bit = 1ull << (ctx->device & 63);
    if (!(attr_mask.load() & bit)) {
        for (int m = 0; m < 3; ++m) {
            const u32 kmax = m == 0 ? FQ_PT_MAX : m == 1 ? FQ_PW_MAX : FQ_EXACT_MAX;
            const int max_smem = (int)((1u << fq_exact_log_slots(kmax)) * 8 + 4 * fq_exact_counters(m, kmax));
            for (int v = 0; v < 2; ++v)
                if (cudaFuncSetAttribute(exact_kernels[m][v], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         max_smem) != cudaSuccess)
                    return TOPK_ECUDA;
        }
        attr_mask.fetch_or(bit);
    }
    int per_sm_x = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_x, ek, FQ_NT, smem);
    const u64 quad_blocks = ((n + 3) / 4 + (u64)FQ_NT * FQ_XQUADS - 1) / ((u64)FQ_NT * FQ_XQUADS);
    const int grid_x = (int)std::max<u64>(1, std::min<u64>(quad_blocks, (u64)ctx->sms * std::max(per_sm_x, 1)));
    e = launch_dep(ek, grid_x, FQ_NT, smem, st, x);
    u64* comp = reinterpret_cast<u64*>(base + o_comp);
    if (e == cudaSuccess)
        e = launch_dep(k_freq_compose, (int)((kstar + 255) / 256), 256, 0, st, (const u64*)sel, (const u32*)exact,
                       kstar, comp);
    if (e != cudaSuccess) return cuda_status(e);
    count_launch(ctx, 3);
    // 4. the k most frequent candidates by exact count
    u64* sel2 = reinterpret_cast<u64*>(base + o_sel2);
    u32* idx2 = reinterpret_cast<u32*>(base + o_idx2);
    u64* kth2 = reinterpret_cast<u64*>(base + o_kth2);
    u32* kth2_idx = reinterpret_cast<u32*>(base + o_kth2 + 8);
    rs = topk_select(ctx, comp, kstar, fp->k, TOPK_U64, sel2, idx2, kth2, kth2_idx, nullptr, stream);
    if (rs != TOPK_OK) return rs;
    e = launch_dep(k_freq_decode, (int)((fp->k + 255) / 256), 256, 0, st, (const u64*)sel2, (const u64*)kth2, fp->k,
                   d_out_obj, d_out_count, ctx->d_err, (const u64*)cursor, (u64)n,
                   d_sample_size);
    count_launch(ctx);
    return cuda_status(e);
}

} // extern "C"
