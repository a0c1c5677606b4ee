// frequent.cu — top-k most frequent objects on one GPU (Section 7):
// Algorithm PAC (Section 7.1: Bernoulli sample, count the sampled objects
// with hashing, select the k most frequently sampled) and Algorithm EC
// (Section 7.2: select the k* most frequently sampled, count those exactly
// over the whole input, select the k most frequent of them).
//
// One GPU is one PE: the paper's distributed hash table is a single
// open-addressing table in HBM, fed by block-local tables in shared memory
// (the local aggregation of Lemma "topkapproxtime"); the selections are
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
constexpr int FQ_LOCAL_LOG = 12;        // block-local table: 4096 slots
constexpr int FQ_LOCAL = 1 << FQ_LOCAL_LOG;
constexpr int FQ_LOCAL_PROBES = 16;
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
// hash's low bits).  False when the table has no free slot left.
__device__ bool fq_table_add(u64* table, u32 mask, u32 obj, u32 c) {
    u32 h = fq_mix(obj) & mask;
    for (u32 probe = 0; probe <= mask; ++probe) {
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

struct FqLocal {
    u64 slot[FQ_LOCAL];
    u32 fill;      // slots claimed since the last flush
    u32 flush;     // flush decision of this tile
    u32 warp_sum[FQ_NT / 32];
};

// One occurrence into the block-local table (probing from the hash's high
// bits, independent of the HBM table's position); false after
// FQ_LOCAL_PROBES occupied slots.
__device__ __forceinline__ bool fq_local_add(FqLocal& L, u32 obj) {
    u32 h = fq_mix(obj) >> (32 - FQ_LOCAL_LOG);
#pragma unroll 1
    for (int p = 0; p < FQ_LOCAL_PROBES; ++p) {
        u64 w = *reinterpret_cast<volatile u64*>(&L.slot[h]);
        if (w == FQ_EMPTY) {
            const u64 prev =
                atomicCAS(reinterpret_cast<unsigned long long*>(&L.slot[h]), FQ_EMPTY, fq_word(obj, 1));
            if (prev == FQ_EMPTY) {
                atomicAdd(&L.fill, 1u);
                return true;
            }
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
    u64 thr;       // sampled iff Philox word < thr (2^32: every object)
    u32 seed_lo, seed_hi;
    u64* table;
    u32 mask;      // table slots - 1
    u64* sample_size;
    u32* err;
};

__device__ __forceinline__ void fq_flush(FqLocal& L, const FreqArgs& a) {
    for (u32 s = threadIdx.x; s < FQ_LOCAL; s += FQ_NT) {
        const u64 w = L.slot[s];
        if (w != FQ_EMPTY) {
            if (!fq_table_add(a.table, a.mask, (u32)w, 0xFFFFFFFFu - (u32)(w >> 32)))
                atomicCAS(a.err, 0u, (u32)TOPK_ENOMEM);
            L.slot[s] = FQ_EMPTY;
        }
    }
}

// Sampling and counting (Section 7.1): every block walks tiles of
// FQ_NT * FQ_QUADS * 4 objects; object i is sampled iff word i % 4 of
// Philox4x32-10 at counter (i / 4, FQ_STREAM) is below the threshold.
// Sampled objects go to the block-local table, which is flushed into the
// HBM table whenever it is more than half full, and at the end.
template <bool ALL, bool VEC>
__global__ void __launch_bounds__(FQ_NT) k_freq_count(FreqArgs a) {
    __shared__ FqLocal L;
    for (u32 s = threadIdx.x; s < FQ_LOCAL; s += FQ_NT) L.slot[s] = FQ_EMPTY;
    if (threadIdx.x == 0) L.fill = 0;
    grid_dep_wait(); // the table was cleared by the previous operation
    __syncthreads();
    const u64 quads = (a.n + 3) / 4;
    const u64 tile_quads = (u64)FQ_NT * FQ_QUADS;
    const u64 tiles = (quads + tile_quads - 1) / tile_quads;
    u64 sampled = 0;
    for (u64 t = blockIdx.x; t < tiles; t += gridDim.x) {
#pragma unroll
        for (int j = 0; j < FQ_QUADS; ++j) {
            const u64 q = t * tile_quads + (u64)j * FQ_NT + threadIdx.x;
            if (q >= quads) break;
            const u64 i0 = q * 4;
            u32 v[4];
            if (VEC && i0 + 4 <= a.n) {
                const uint4 x = ld_stream(reinterpret_cast<const uint4*>(a.obj) + q);
                v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = i0 + e < a.n ? __ldcs(a.obj + i0 + e) : 0u;
            }
            u32 take = 0;
            if (ALL) {
                take = 0xF;
            } else {
                const Philox4 r = philox4x32_10((u32)q, (u32)(q >> 32), FQ_STREAM, 0u, a.seed_lo, a.seed_hi);
#pragma unroll
                for (int e = 0; e < 4; ++e) take |= ((u64)r.v[e] < a.thr ? 1u : 0u) << e;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (!((take >> e) & 1u) || i0 + e >= a.n) continue;
                ++sampled;
                if (!fq_local_add(L, v[e]) && !fq_table_add(a.table, a.mask, v[e], 1))
                    atomicCAS(a.err, 0u, (u32)TOPK_ENOMEM);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) L.flush = L.fill > FQ_LOCAL / 2 ? 1u : 0u;
        __syncthreads();
        if (L.flush) {
            fq_flush(L, a);
            if (threadIdx.x == 0) L.fill = 0;
            __syncthreads();
        }
    }
    fq_flush(L, a);
    // sample size: warp sums, then one atomic per block
    u64 w = sampled;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) L.warp_sum[threadIdx.x >> 5] = (u32)w;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 s = 0;
        for (int i = 0; i < FQ_NT / 32; ++i) s += L.warp_sum[i];
        if (a.sample_size) atomicAdd(reinterpret_cast<unsigned long long*>(a.sample_size), (unsigned long long)s);
    }
}

// Exact recount of the k* candidates (Section 7.2) over the whole input:
// the candidates sit in a shared-memory hash table (object, candidate
// number); every block counts its tiles in shared memory and adds its
// counts to exact[] at the end.
struct ExactArgs {
    const u32* obj;
    u64 n;
    const u64* cand; // k* table words: object in the low half
    u32 kstar;
    u32 log_slots;
    u32* exact;      // kstar counts (zeroed before)
};

template <bool VEC>
__global__ void __launch_bounds__(FQ_NT) k_freq_exact(ExactArgs a) {
    extern __shared__ __align__(16) unsigned char fq_smem[];
    const u32 slots = 1u << a.log_slots;
    u32* key = reinterpret_cast<u32*>(fq_smem);
    int* id = reinterpret_cast<int*>(key + slots);
    u32* cnt = reinterpret_cast<u32*>(id + slots);
    for (u32 s = threadIdx.x; s < slots; s += FQ_NT) id[s] = -1;
    for (u32 c = threadIdx.x; c < a.kstar; c += FQ_NT) cnt[c] = 0;
    grid_dep_wait(); // the candidates come from the previous selection
    __syncthreads();
    for (u32 c = threadIdx.x; c < a.kstar; c += FQ_NT) {
        const u32 o = (u32)a.cand[c];
        u32 h = fq_mix(o) >> (32 - a.log_slots);
        while (atomicCAS(&id[h], -1, (int)c) != -1) h = (h + 1) & (slots - 1);
        key[h] = o;
    }
    __syncthreads();
    const u64 quads = (a.n + 3) / 4;
    for (u64 q = (u64)blockIdx.x * FQ_NT + threadIdx.x; q < quads; q += (u64)gridDim.x * FQ_NT) {
        const u64 i0 = q * 4;
        u32 v[4];
        if (VEC && i0 + 4 <= a.n) {
            const uint4 x = ld_stream(reinterpret_cast<const uint4*>(a.obj) + q);
            v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = i0 + e < a.n ? __ldcs(a.obj + i0 + e) : 0u;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (i0 + e >= a.n) break;
            u32 h = fq_mix(v[e]) >> (32 - a.log_slots);
            int c;
            while ((c = id[h]) >= 0 && key[h] != v[e]) h = (h + 1) & (slots - 1);
            if (c >= 0) atomicAdd(&cnt[c], 1u);
        }
    }
    __syncthreads();
    for (u32 c = threadIdx.x; c < a.kstar; c += FQ_NT)
        if (cnt[c]) atomicAdd(&a.exact[c], cnt[c]);
}

// Table words of the candidates with their exact counts.
__global__ void k_freq_compose(const u64* cand, const u32* exact, u32 kstar, u64* out) {
    grid_dep_wait();
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kstar) out[i] = fq_word((u32)cand[i], exact[i]);
}

// Selected table words -> objects and counts; a selected empty slot means
// fewer than `need` distinct objects were sampled.
__global__ void k_freq_decode(const u64* sel, const u64* kth, u32 k, u32* out_obj, u64* out_cnt, u32* err) {
    grid_dep_wait();
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && *kth == FQ_EMPTY) atomicCAS(err, 0u, (u32)TOPK_EINVAL);
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
    const u64 distinct = fp->max_distinct ? fp->max_distinct : FQ_DEFAULT_DISTINCT;
    const u32 log_cap = std::max<u32>(12, ceil_log2(2 * std::max<u64>(distinct, (u64)kstar)));
    if (log_cap > 31) return TOPK_EINVAL;
    const u64 cap = 1ull << log_cap;
    const u32 need = ec ? kstar : fp->k;
    if (need > cap) return TOPK_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return TOPK_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    Carve cv;
    const size_t o_table = cv.take(8 * cap);
    const size_t o_sel = cv.take(8ull * need), o_idx = cv.take(4ull * need), o_kth = cv.take(16);
    const size_t o_exact = cv.take(4ull * kstar), o_comp = cv.take(8ull * kstar);
    const size_t o_sel2 = cv.take(8ull * fp->k), o_idx2 = cv.take(4ull * fp->k), o_kth2 = cv.take(16);
    rs = ensure_freq(ctx, cv.off);
    if (rs != TOPK_OK) return rs;
    char* base = static_cast<char*>(ctx->freq.base);
    u64* table = reinterpret_cast<u64*>(base + o_table);
    u64* sel = reinterpret_cast<u64*>(base + o_sel);
    u32* sel_idx = reinterpret_cast<u32*>(base + o_idx);
    u64* kth = reinterpret_cast<u64*>(base + o_kth);
    u32* kth_idx = reinterpret_cast<u32*>(base + o_kth + 8);

    // 1. sample and count (Section 7.1)
    cudaError_t e = cudaMemsetAsync(table, 0xFF, 8 * cap, st);
    if (e == cudaSuccess && d_sample_size) e = cudaMemsetAsync(d_sample_size, 0, 8, st);
    if (e != cudaSuccess) return cuda_status(e);
    FreqArgs a{};
    a.obj = static_cast<const u32*>(d_objects);
    a.n = n;
    a.thr = rho >= 1.0 ? (1ull << 32) : (u64)std::floor(std::ldexp(rho, 32));
    a.seed_lo = (u32)fp->seed;
    a.seed_hi = (u32)(fp->seed >> 32);
    a.table = table;
    a.mask = (u32)(cap - 1);
    a.sample_size = d_sample_size;
    a.err = ctx->d_err;
    const bool all = a.thr >= (1ull << 32);
    const bool vec = reinterpret_cast<uintptr_t>(d_objects) % 16 == 0;
    auto kern = all ? (vec ? k_freq_count<true, true> : k_freq_count<true, false>)
                    : (vec ? k_freq_count<false, true> : k_freq_count<false, false>);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FQ_NT, 0);
    const u64 tiles = ((n + 3) / 4 + (u64)FQ_NT * FQ_QUADS - 1) / ((u64)FQ_NT * FQ_QUADS);
    const int grid = (int)std::max<u64>(1, std::min<u64>(tiles, (u64)ctx->sms * std::max(per_sm, 1)));
    e = launch_dep(kern, grid, FQ_NT, 0, st, a);
    if (e != cudaSuccess) return cuda_status(e);
    count_launch(ctx);

    // 2. the `need` most frequently sampled objects: the smallest table words
    rs = topk_select(ctx, table, cap, need, TOPK_U64, sel, sel_idx, kth, kth_idx, nullptr, stream);
    if (rs != TOPK_OK) return rs;
    if (!ec) {
        e = launch_dep(k_freq_decode, (int)((fp->k + 255) / 256), 256, 0, st, (const u64*)sel, (const u64*)kth,
                       fp->k, d_out_obj, d_out_count, ctx->d_err);
        count_launch(ctx);
        return cuda_status(e);
    }
    // 3. EC: exact recount of the k* candidates (Section 7.2)
    e = launch_dep(k_freq_check, 1, 32, 0, st, (const u64*)kth, ctx->d_err);
    u32* exact = reinterpret_cast<u32*>(base + o_exact);
    if (e == cudaSuccess) e = cudaMemsetAsync(exact, 0, 4ull * kstar, st);
    if (e != cudaSuccess) return cuda_status(e);
    ExactArgs x{};
    x.obj = a.obj;
    x.n = n;
    x.cand = sel;
    x.kstar = kstar;
    x.log_slots = std::max<u32>(6, ceil_log2(2ull * kstar));
    x.exact = exact;
    const size_t smem = (size_t)(1u << x.log_slots) * 8 + 4ull * kstar;
    auto ek = vec ? k_freq_exact<true> : k_freq_exact<false>;
    static std::atomic<uint64_t> attr_mask{0};
    const uint64_t bit = 1ull << (ctx->device & 63);
    if (!(attr_mask.load() & bit)) {
        const int max_smem = (int)((1u << ceil_log2(2ull * FQ_EXACT_MAX)) * 8 + 4ull * FQ_EXACT_MAX);
        if (cudaFuncSetAttribute(k_freq_exact<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_freq_exact<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem) !=
                cudaSuccess)
            return TOPK_ECUDA;
        attr_mask.fetch_or(bit);
    }
    int per_sm_x = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_x, ek, FQ_NT, smem);
    const u64 quad_blocks = ((n + 3) / 4 + FQ_NT - 1) / FQ_NT;
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
                   d_out_obj, d_out_count, ctx->d_err);
    count_launch(ctx);
    return cuda_status(e);
}

} // extern "C"
