// common.cuh — device building blocks shared by every selection kernel.
//
// Key order (paper, Section 2): every object's value v is made unique by
// pairing it with the object itself; here the object is its position, so the
// order is on the pair (key', idx), where key' is an order-preserving
// unsigned image of the key:
//   u32 -> itself; i32 -> x ^ 0x80000000; u64 -> itself;
//   f32 / bf16 -> sign-magnitude to unsigned: negative patterns are
//   complemented, non-negative ones get the sign bit set, which realises IEEE
//   754 totalOrder on the bit patterns.
// The pair is packed into one unsigned integer, the "composite":
//   32-bit keys: (key' << 32) | idx   in a uint64
//   64-bit keys: (key' << 32) | idx   in an unsigned __int128 (96 bits used)
// so every comparison of the method is one integer comparison.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace topk {

typedef uint32_t u32;
typedef uint64_t u64;
typedef unsigned __int128 u128;

enum : int { DT_U32 = 0, DT_I32 = 1, DT_F32 = 2, DT_BF16 = 3, DT_U64 = 4 };
// DT_DESC + DT: the same key type ordered the other way (selection of the k
// largest); ties are still broken by the smaller position.
constexpr int DT_DESC = 8;

// ---------------------------------------------------------------- key maps

template <int DT> struct Key;

template <> struct Key<DT_U32> {
    typedef u32 raw_t;
    typedef u32 key_t;
    static constexpr int KW = 32;
    __host__ __device__ static key_t fwd(raw_t x) { return x; }
    __host__ __device__ static raw_t inv(key_t k) { return k; }
};
template <> struct Key<DT_I32> {
    typedef u32 raw_t;
    typedef u32 key_t;
    static constexpr int KW = 32;
    __host__ __device__ static key_t fwd(raw_t x) { return x ^ 0x80000000u; }
    __host__ __device__ static raw_t inv(key_t k) { return k ^ 0x80000000u; }
};
template <> struct Key<DT_F32> {
    typedef u32 raw_t;
    typedef u32 key_t;
    static constexpr int KW = 32;
    // negative: all bits flipped; non-negative: sign bit set
    __host__ __device__ static key_t fwd(raw_t x) {
        return x ^ ((u32)((int32_t)x >> 31) | 0x80000000u);
    }
    __host__ __device__ static raw_t inv(key_t k) {
        return k ^ ((u32)((int32_t)~k >> 31) | 0x80000000u);
    }
};
template <> struct Key<DT_BF16> {
    typedef uint16_t raw_t;
    typedef u32 key_t; // 16-bit image, zero-extended
    static constexpr int KW = 32;
    __host__ __device__ static key_t fwd(raw_t x) {
        u32 v = x;
        return v ^ ((v & 0x8000u) ? 0xFFFFu : 0x8000u);
    }
    __host__ __device__ static raw_t inv(key_t k) {
        return (raw_t)(k ^ ((k & 0x8000u) ? 0x8000u : 0xFFFFu));
    }
};
template <> struct Key<DT_U64> {
    typedef u64 raw_t;
    typedef u64 key_t;
    static constexpr int KW = 64;
    __host__ __device__ static key_t fwd(raw_t x) { return x; }
    __host__ __device__ static raw_t inv(key_t k) { return k; }
};

// Descending order: the ascending key image complemented within its width
// (16 bits for bf16), so the k smallest images are the k largest keys.
template <int DT> struct Key {
    static_assert(DT >= DT_DESC && DT < DT_DESC + 5, "descending key codes only");
    typedef Key<DT - DT_DESC> A;
    typedef typename A::raw_t raw_t;
    typedef typename A::key_t key_t;
    static constexpr int KW = A::KW;
    static constexpr key_t FLIP = (DT - DT_DESC == DT_BF16) ? (key_t)0xFFFFu : (key_t)~(key_t)0;
    __host__ __device__ static key_t fwd(raw_t x) { return A::fwd(x) ^ FLIP; }
    __host__ __device__ static raw_t inv(key_t k) { return A::inv(k ^ FLIP); }
};

// ------------------------------------------------------------- composites

template <int KW> struct Comp;

template <> struct Comp<32> {
    typedef u64 t;
    typedef u32 key_t;
    static constexpr int DIGITS = 8; // 8-bit digits, most significant first
    __host__ __device__ static t make(u32 key, u32 idx) { return ((u64)key << 32) | idx; }
    __host__ __device__ static u32 key(t c) { return (u32)(c >> 32); }
    __host__ __device__ static u32 idx(t c) { return (u32)c; }
    __host__ __device__ static t max_value() { return ~(u64)0; }
    __host__ __device__ static t from128(u128 v) { return (u64)v; }
    __device__ static u32 digit(t c, int d) { return (u32)(c >> (56 - 8 * d)) & 0xFFu; }
};

template <> struct Comp<64> {
    typedef u128 t;
    typedef u64 key_t;
    static constexpr int DIGITS = 12;
    __host__ __device__ static t make(u64 key, u32 idx) { return ((u128)key << 32) | idx; }
    __host__ __device__ static u64 key(t c) { return (u64)(c >> 32); }
    __host__ __device__ static u32 idx(t c) { return (u32)c; }
    __host__ __device__ static t max_value() { return ((u128)1 << 96) - 1; }
    __host__ __device__ static t from128(u128 v) { return v; }
    __device__ static u32 digit(t c, int d) { return (u32)(c >> (88 - 8 * d)) & 0xFFu; }
};

// -------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon, Moraes, Dror and Shaw ("Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64
// multiplications whose halves are xored with the other counter words and the
// round key; the key is bumped by the two Weyl constants between rounds.
struct Philox4 {
    u32 v[4];
};

__host__ __device__ inline Philox4 philox4x32_10(u32 c0, u32 c1, u32 c2, u32 c3, u32 k0, u32 k1) {
    const u32 M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const u32 W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        u64 p0 = (u64)M0 * c0;
        u64 p1 = (u64)M1 * c2;
        u32 hi0 = (u32)(p0 >> 32), lo0 = (u32)p0;
        u32 hi1 = (u32)(p1 >> 32), lo1 = (u32)p1;
        u32 n0 = hi1 ^ c1 ^ k0;
        u32 n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    Philox4 out;
    out.v[0] = c0;
    out.v[1] = c1;
    out.v[2] = c2;
    out.v[3] = c3;
    return out;
}

// ------------------------------------------------------------ call state
// One selection in progress.  The window [lo, hi] (composites, inclusive)
// holds the m_win elements of the current source that are still undecided;
// the element sought has rank k_rem (1-based) inside the window; out_base
// outputs are already committed.  A pass splits the window into
//   a = [lo, pl)   (all selected),  b = [pl, pr]  (candidates),  c = (pr, hi]
// exactly as Algorithm "select" partitions s into a, b, c (Section 2).

enum : u32 { PH_RUN = 0, PH_FINISH = 1, PH_DONE = 2, PH_ERROR = 3 };
enum : u32 { SRC_INPUT = 0, SRC_CAND0 = 1, SRC_CAND1 = 2 };
enum : u32 { ST_OK = 0, ST_EINVAL = 1, ST_ETIMEOUT = 4, ST_EINTERNAL = 7 };

struct alignas(16) SelState {
    u128 lo, hi;          // window
    u128 pl, pr;          // pivots of the pending pass
    u64 m_src;            // elements in the current source array
    u64 m_win;            // elements of the source inside the window
    u64 k_rem;            // rank sought inside the window, >= 1
    u64 out_base;         // outputs committed so far
    u64 cnt_a, cnt_b;     // pass counters (accumulated by atomics)
    u64 cap_b;            // capacity of each candidate buffer
    u64 first_cand;       // statistics
    u32 level, phase, src, dst;
    u32 pending;          // a pass ran whose counters are not yet consumed
    u32 status;           // first device error, ST_*
    u32 levels_grid, levels_block, failures, overflows;
    u32 sample_kept;
    u32 dense;            // the armed pass expects many a-elements
};

// Number of significant bits of v (0 for 0).
__device__ __forceinline__ int bit_length_fast(u64 v) { return v ? 64 - __clzll((long long)v) : 0; }
__device__ __forceinline__ int bit_length_fast(u128 v) {
    const u64 hi = (u64)(v >> 64);
    return hi ? 128 - __clzll((long long)hi) : bit_length_fast((u64)v);
}

// Arguments common to every kernel of one topk_select call.
struct SelArgs {
    const void* keys;         // input (raw keys)
    u64 n, k;
    void* out_keys;           // k raw keys
    u32* out_idx;             // k positions
    void* kth_key;
    u32* kth_idx;
    void* cand_key[2];        // candidate buffers: key' (u32 or u64)
    u32* cand_idx[2];
    SelState* st;
    u64 cap_b;
    u64 seed;
    u32 parts;                // sampling partitions
    u32 sample;               // draws per level
    u32 finish_T;             // single-block finish threshold
    u32 grid_G;               // grid levels run while m_src > G
    float z;                  // pivot margin factor
    u32 flags;
    u32 aligned;              // input is 16-byte aligned
    u32* err;                 // context's latched error word
    // grid-level sampling (k_sample / k_pivots) and the end-of-pass branch
    void* samp;               // sample composites, capacity samp_cap
    u32* samp_count;          // number drawn into samp (zero between levels)
    u32* pass_done;           // block-done counter of the pass (zero between passes)
    u32 samp_cap;
    int first_dense;          // first level's pass mode chosen by the host (0/1), or -1
};


// Largest composite of a key type's domain (the first window's upper end):
// every composite of that type is at or below it, and the window histogram
// spreads over the key bits actually used (16 for bf16).
template <int DT> __host__ __device__ inline u128 key_domain_max() {
    constexpr int B = DT % DT_DESC;
    return B == DT_U64 ? (((u128)~(u64)0) << 32) | 0xFFFFFFFFu
                       : (((u128)(B == DT_BF16 ? 0xFFFFu : 0xFFFFFFFFu)) << 32) | 0xFFFFFFFFu;
}


// ------------------------------------------------- dependent launches
// The kernels of one call are launched with programmatic stream
// serialization: a kernel's blocks may become resident while the previous
// kernel is still finishing, and wait here, before their first access to
// anything the previous kernels wrote, until that grid has completed and its
// memory is visible.  Each kernel lets its successor start launching at once
// (its grids are single waves, so the successor's early blocks never keep
// one of its own blocks from being scheduled).  Without the launch attribute
// both instructions do nothing.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------- warp helpers

__device__ __forceinline__ u32 lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ u32 lanemask_lt() { return (1u << lane_id()) - 1u; }

// Streaming 16-byte load (cache-streaming policy: the input is read once per
// level, so it should not displace the candidate buffers from L2).
__device__ __forceinline__ uint4 ld_stream(const uint4* p) { return __ldcs(p); }

// ------------------------------------------- mbarrier and bulk copies
// Shared-memory barriers with transaction counts and the bulk (TMA) copy
// engine, for streaming kernels whose loads must not wait on the compute.

__device__ __forceinline__ u32 smem_addr(const void* p) {
    return (u32)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Makes barrier initialisation visible to the bulk-copy (async) proxy.
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, u32 bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, u32 parity) {
    u32 ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// As mbar_try_wait, but the thread may stay suspended in the instruction for
// up to `hint_ns` nanoseconds while the phase is incomplete (it resumes as soon
// as the phase completes), so a long wait costs few issued instructions.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, u32 parity, u32 hint_ns) {
    u32 ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
                 : "memory");
    return ok != 0;
}
// Waits for phase `parity` of `bar` to complete, for at most ~`limit_ns`
// nanoseconds of wall time; returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, u32 parity, u64 limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    u64 t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (true) {
        if (mbar_try_wait_hint(bar, parity, 100000u)) return true;
        u64 t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) return false;
    }
}
// Global -> shared bulk copy; completion counted on `bar` as transaction
// bytes.  dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, u32 bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ u32 u4get(const uint4& v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

} // namespace topk
