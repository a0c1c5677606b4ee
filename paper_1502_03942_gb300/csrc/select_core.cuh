// select_core.cuh — the steps of sample-based selection as block-level device
// functions, shared by the single-selection kernels (select_impl.cuh) and the
// batched kernels (batched.cu).
//
// One recursion level of Algorithm "select" (paper, Section 2) is
//   pickPivots : draw a sample of the undecided elements, take the sample
//                elements of ranks k|S|/n -/+ Delta as pivots l <= r
//                ("Distributed FR-Selection", Section 2);
//   partition  : split the elements into a (< l), b (l..r), c (> r);
//   reduction  : n_a, n_b summed over all partitions;
//   branch     : recurse into a, b or c.
// Here a pass writes a straight into the output (when the bracket holds rank
// k they are all selected) and b into a candidate buffer, so one read of the
// input classifies and compacts.  The reduction is the sum of per-block
// atomics.  The branch is `decide`, run by one thread before the next level.
#pragma once

#include "common.cuh"

namespace topk {

// ------------------------------------------------------------------ sources
// A source yields (key', idx) for positions 0..m-1.

template <int DT> struct InputSrc {
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    static constexpr int KW = K::KW;
    static constexpr int EPV = 16 / (int)sizeof(raw_t); // elements per 16-byte vector
    static constexpr int NV = 16 / EPV;                 // vectors per 16-element slot set
    static constexpr bool IMPLICIT_IDX = true;          // position = element index
    // Tiles are laid on the 16-byte-aligned address at or below the first
    // key: `keys` is that address, `head` the number of keys before the
    // first one.  Tile coordinates e map to positions e - head; the slots
    // with e < head or e >= head + m are masked out.  Those extra reads stay
    // inside 16-byte segments that also hold valid keys.
    const raw_t* keys;
    u64 m;
    u32 head;

    __host__ __device__ static InputSrc make(const void* p, u64 m) {
        InputSrc s;
        const uintptr_t a = reinterpret_cast<uintptr_t>(p);
        s.head = (u32)((a & 15u) / sizeof(raw_t));
        s.keys = reinterpret_cast<const raw_t*>(a & ~(uintptr_t)15u);
        s.m = m;
        return s;
    }
    __device__ __forceinline__ u64 extent() const { return m + head; } // in tile coordinates

    __device__ __forceinline__ void at(u64 i, key_t& k, u32& x) const {
        k = K::fwd(keys[head + i]);
        x = (u32)i;
    }
    // position of slot s of this thread in the tile starting at `base`
    template <int NT> __device__ __forceinline__ u32 idx_of(u64 base, int s) const {
        return (u32)(base + (u64)((s / EPV) * NT + threadIdx.x) * EPV + (s % EPV) - head);
    }

    // Keys of the NV 16-byte vectors of one thread, in slot order.
    __device__ __forceinline__ static void unpack(const uint4 (&v)[NV], key_t (&kk)[16]) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
#pragma unroll
            for (int i = 0; i < EPV; ++i) {
                raw_t r;
                if (sizeof(raw_t) == 4) {
                    r = (raw_t)u4get(v[j], i);
                } else if (sizeof(raw_t) == 2) {
                    u32 w = u4get(v[j], i >> 1);
                    r = (raw_t)((i & 1) ? (w >> 16) : (w & 0xFFFFu));
                } else {
                    r = (raw_t)(((u64)u4get(v[j], 2 * i + 1) << 32) | u4get(v[j], 2 * i));
                }
                kk[j * EPV + i] = K::fwd(r);
            }
        }
    }

    // Raw key words of the NV 16-byte vectors, in slot order.
    __device__ __forceinline__ static void unpack_raw(const uint4 (&v)[NV], raw_t (&rr)[16]) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
#pragma unroll
            for (int i = 0; i < EPV; ++i) {
                if (sizeof(raw_t) == 4) {
                    rr[j * EPV + i] = (raw_t)u4get(v[j], i);
                } else if (sizeof(raw_t) == 2) {
                    const u32 w = u4get(v[j], i >> 1);
                    rr[j * EPV + i] = (raw_t)((i & 1) ? (w >> 16) : (w & 0xFFFFu));
                } else {
                    rr[j * EPV + i] = (raw_t)(((u64)u4get(v[j], 2 * i + 1) << 32) | u4get(v[j], 2 * i));
                }
            }
        }
    }

    // 16 elements per thread from a tile staged in shared memory.
    template <int NT>
    __device__ __forceinline__ static void load16_smem(const uint4* stage, key_t (&kk)[16]) {
        uint4 v[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = stage[j * NT + threadIdx.x];
        unpack(v, kk);
    }

    // The keys alone (positions from idx_of); bit s of the result = valid.
    template <int NT> __device__ __forceinline__ u32 load16_keys(u64 base, key_t (&kk)[16]) const {
        const u32 tid = threadIdx.x;
        const u64 ext = extent();
        if (base + (u64)NT * 16 <= ext) {
            const uint4* p = reinterpret_cast<const uint4*>(keys) + base / EPV;
            uint4 v[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) v[j] = ld_stream(p + j * NT + tid);
            unpack(v, kk);
            u32 valid = 0xFFFFu;
            if (base < head) { // the first tile: slots before the first key
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (base + (u64)((q / EPV) * NT + tid) * EPV + (q % EPV) < head) valid &= ~(1u << q);
            }
            return valid;
        }
        u32 valid = 0;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
#pragma unroll
            for (int i = 0; i < EPV; ++i) {
                const u64 e = base + (u64)(j * NT + tid) * EPV + i;
                const int q = j * EPV + i;
                if (e >= head && e < ext) {
                    kk[q] = K::fwd(keys[e]);
                    valid |= 1u << q;
                } else {
                    kk[q] = 0;
                }
            }
        }
        return valid;
    }

    // 16 elements per thread of the tile at tile coordinate `base`: slot
    // s = j*EPV + i is tile element base + (j*NT + tid)*EPV + i.  Bit s of the
    // returned mask = valid; ii receives positions.
    template <int NT>
    __device__ __forceinline__ u32 load16(u64 base, key_t (&kk)[16], u32 (&ii)[16]) const {
        const u32 tid = threadIdx.x;
        const u64 ext = extent();
        if (base + (u64)NT * 16 <= ext) {
            const uint4* p = reinterpret_cast<const uint4*>(keys) + base / EPV;
            uint4 v[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) v[j] = ld_stream(p + j * NT + tid);
            unpack(v, kk);
            u32 valid = 0xFFFFu;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const u64 e = base + (u64)((q / EPV) * NT + tid) * EPV + (q % EPV);
                ii[q] = (u32)(e - head);
                if (e < head) valid &= ~(1u << q);
            }
            return valid;
        }
        u32 valid = 0;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
#pragma unroll
            for (int i = 0; i < EPV; ++i) {
                const u64 e = base + (u64)(j * NT + tid) * EPV + i;
                const int q = j * EPV + i;
                if (e >= head && e < ext) {
                    kk[q] = K::fwd(keys[e]);
                    valid |= 1u << q;
                } else {
                    kk[q] = 0;
                }
                ii[q] = (u32)(e - head);
            }
        }
        return valid;
    }
};

template <int KW> struct CandSrc;

template <> struct CandSrc<32> {
    typedef u32 key_t;
    static constexpr int KW = 32;
    static constexpr bool IMPLICIT_IDX = false;
    const u32* ck;
    const u32* ci;
    u64 m;
    __device__ __forceinline__ u64 extent() const { return m; }
    __device__ __forceinline__ void at(u64 i, key_t& k, u32& x) const {
        k = __ldcg(ck + i);
        x = __ldcg(ci + i);
    }
    template <int NT>
    __device__ __forceinline__ u32 load16(u64 base, key_t (&kk)[16], u32 (&ii)[16]) const {
        const u32 tid = threadIdx.x;
        if (base + (u64)NT * 16 <= m) {
            const uint4* pk = reinterpret_cast<const uint4*>(ck) + base / 4;
            const uint4* pi = reinterpret_cast<const uint4*>(ci) + base / 4;
            uint4 vk[4], vi[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                vk[j] = __ldcg(pk + j * NT + tid);
                vi[j] = __ldcg(pi + j * NT + tid);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    kk[j * 4 + i] = u4get(vk[j], i);
                    ii[j * 4 + i] = u4get(vi[j], i);
                }
            return 0xFFFFu;
        }
        u32 valid = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const u64 e = base + (u64)(j * NT + tid) * 4 + i;
                const int s = j * 4 + i;
                if (e < m) {
                    kk[s] = __ldcg(ck + e);
                    ii[s] = __ldcg(ci + e);
                    valid |= 1u << s;
                } else {
                    kk[s] = 0;
                    ii[s] = 0;
                }
            }
        return valid;
    }
};

template <> struct CandSrc<64> {
    typedef u64 key_t;
    static constexpr int KW = 64;
    static constexpr bool IMPLICIT_IDX = false;
    const u64* ck;
    const u32* ci;
    u64 m;
    __device__ __forceinline__ u64 extent() const { return m; }
    __device__ __forceinline__ void at(u64 i, key_t& k, u32& x) const {
        k = __ldcg(reinterpret_cast<const unsigned long long*>(ck) + i);
        x = __ldcg(ci + i);
    }
    template <int NT>
    __device__ __forceinline__ u32 load16(u64 base, key_t (&kk)[16], u32 (&ii)[16]) const {
        const u32 tid = threadIdx.x;
        if (base + (u64)NT * 16 <= m) {
            const uint4* pk = reinterpret_cast<const uint4*>(ck) + base / 2;
            const uint2* pi = reinterpret_cast<const uint2*>(ci) + base / 2;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                uint4 vk = __ldcg(pk + j * NT + tid);
                uint2 vi = __ldcg(pi + j * NT + tid);
                kk[2 * j] = ((u64)vk.y << 32) | vk.x;
                kk[2 * j + 1] = ((u64)vk.w << 32) | vk.z;
                ii[2 * j] = vi.x;
                ii[2 * j + 1] = vi.y;
            }
            return 0xFFFFu;
        }
        u32 valid = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const u64 e = base + (u64)(j * NT + tid) * 2 + i;
                const int s = j * 2 + i;
                if (e < m) {
                    at(e, kk[s], ii[s]);
                    valid |= 1u << s;
                } else {
                    kk[s] = 0;
                    ii[s] = 0;
                }
            }
        return valid;
    }
};

// --------------------------------------------------------- output targets
// Where a pass writes its a elements (selected: raw keys + positions) and its
// b elements (candidates: key' + positions).

template <int DT> struct Sink {
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    raw_t* out_keys;
    u32* out_idx;
    u64 out_base; // first free output slot
    u64 cap_a;    // slots available to this pass (k_rem)
    key_t* ck;
    u32* ci;
    u64 cap_b;
    u64* cnt_a; // global counters (atomics)
    u64* cnt_b;

    __device__ __forceinline__ void put_a(u64 pos, key_t k, u32 x) const {
        if (pos < cap_a) {
            out_keys[out_base + pos] = K::inv(k);
            out_idx[out_base + pos] = x;
        }
    }
    // a-element given by its raw key bits
    __device__ __forceinline__ void put_a_raw(u64 pos, raw_t r, u32 x) const {
        if (pos < cap_a) {
            out_keys[out_base + pos] = r;
            out_idx[out_base + pos] = x;
        }
    }
    // n staged a-elements (raw keys) to output positions pos..pos+n-1 (all
    // lanes of a warp call; coalesced)
    template <class QK>
    __device__ __forceinline__ void copy_a(u64 pos, const QK* sk, const u32* si, u32 n) const {
        if (pos + n <= cap_a) {
            raw_t* ok = out_keys + out_base + pos;
            u32* oi = out_idx + out_base + pos;
            for (u32 e = lane_id(); e < n; e += 32) {
                ok[e] = (raw_t)sk[e];
                oi[e] = si[e];
            }
        } else {
            for (u32 e = lane_id(); e < n; e += 32) put_a_raw(pos + e, (raw_t)sk[e], si[e]);
        }
    }
    template <class QK>
    __device__ __forceinline__ void copy_b(u64 pos, const QK* sk, const u32* si, u32 n) const {
        if (pos + n <= cap_b) {
            key_t* bk = ck + pos;
            u32* bi = ci + pos;
            for (u32 e = lane_id(); e < n; e += 32) {
                bk[e] = (key_t)sk[e];
                bi[e] = si[e];
            }
        } else {
            for (u32 e = lane_id(); e < n; e += 32) put_b(pos + e, (key_t)sk[e], si[e]);
        }
    }
    __device__ __forceinline__ void put_b(u64 pos, key_t k, u32 x) const {
        if (pos < cap_b) {
            ck[pos] = k;
            ci[pos] = x;
        }
    }
};

// ---------------------------------------------- bounds on raw key bits
// Whether image(x) <= T (or >= T) for the order-preserving image of a key
// type, decided by one integer comparison of the raw bits x against a bound
// derived from T once, instead of transforming every key.  For the IEEE
// types the image of a non-negative pattern is x + 2^(w-1) and that of a
// negative one ~x (w = 32 for f32, 16 for bf16), so
//   image(x) <= T, T >= 2^(w-1):  x <= T - 2^(w-1)  (x as a signed w-bit integer)
//   image(x) <= T, T <  2^(w-1):  x >= ~T           (unsigned)
//   image(x) >= T, T >= 2^(w-1):  x >= T - 2^(w-1)  (signed)
//   image(x) >= T, T <  2^(w-1):  x <= ~T           (unsigned)
// i32's image is x ^ 2^31, a signed comparison; u32 and u64 are their own
// images.  The descending codes (image = ascending image ^ FLIP) turn
// image <= T into ascending image >= T ^ FLIP.
enum : u32 { RB_LE_S = 0, RB_LE_U = 1, RB_GE_S = 2, RB_GE_U = 3 };

template <int DT> struct RawBound {
    typedef Key<DT> K;
    typedef typename K::raw_t raw_t;
    typedef typename K::key_t key_t;
    typedef key_t cmp_t; // u32 for 32- and 16-bit keys, u64 for u64
    static constexpr int B = DT % DT_DESC;
    u32 mode;
    cmp_t v;

    __device__ static RawBound make(u32 m, cmp_t v) { RawBound r; r.mode = m; r.v = v; return r; }
    __device__ static RawBound asc_le(key_t T) {
        if (B == DT_U32 || B == DT_U64) return make(RB_LE_U, T);
        if (B == DT_I32) return make(RB_LE_S, (cmp_t)(T ^ 0x80000000u));
        constexpr key_t H = B == DT_BF16 ? 0x8000u : 0x80000000u;
        constexpr key_t M = B == DT_BF16 ? 0xFFFFu : 0xFFFFFFFFu;
        return T >= H ? make(RB_LE_S, (cmp_t)(T - H)) : make(RB_GE_U, (cmp_t)(~T & M));
    }
    __device__ static RawBound asc_ge(key_t T) {
        if (B == DT_U32 || B == DT_U64) return make(RB_GE_U, T);
        if (B == DT_I32) return make(RB_GE_S, (cmp_t)(T ^ 0x80000000u));
        constexpr key_t H = B == DT_BF16 ? 0x8000u : 0x80000000u;
        constexpr key_t M = B == DT_BF16 ? 0xFFFFu : 0xFFFFFFFFu;
        return T >= H ? make(RB_GE_S, (cmp_t)(T - H)) : make(RB_LE_U, (cmp_t)(~T & M));
    }
    // the bound for image(x) <= T
    __device__ static RawBound le(key_t T) {
        if constexpr (DT >= DT_DESC) return asc_ge((key_t)(T ^ K::FLIP));
        else return asc_le(T);
    }
    // signed value of a raw pattern (sign-extended from its own width)
    __device__ static int sval(raw_t x) {
        if constexpr (sizeof(raw_t) == 2) return (int)(int16_t)x;
        else return (int)(u32)x;
    }
    template <u32 MODE> __device__ static bool test(raw_t x, cmp_t v) {
        if constexpr (sizeof(raw_t) == 8) {
            return MODE == RB_LE_U ? (u64)x <= (u64)v : (u64)x >= (u64)v;
        } else {
            if constexpr (MODE == RB_LE_S) return sval(x) <= (int)(u32)v;
            else if constexpr (MODE == RB_LE_U) return (u32)x <= (u32)v;
            else if constexpr (MODE == RB_GE_S) return sval(x) >= (int)(u32)v;
            else return (u32)x >= (u32)v;
        }
    }
};

// Masks of a tile's 16 slots whose pair is below pl (ma) and at most pr (le),
// for a tile whose positions all lie on one side of each pivot's position:
// ties with a pivot's key are then decided for the whole tile, and each
// slot costs two comparisons of raw bits.  `any_a` / `any_l` false: no slot
// qualifies.
template <int DT, u32 MA, u32 MB>
__device__ __forceinline__ void tile_masks_raw(const typename Key<DT>::raw_t (&rr)[16], typename RawBound<DT>::cmp_t va,
                                               typename RawBound<DT>::cmp_t vb, bool any_a, bool any_l, u32& ma,
                                               u32& le) {
    typedef RawBound<DT> R;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        ma |= (u32)(any_a && R::template test<MA>(rr[q], va)) << q;
        le |= (u32)(any_l && R::template test<MB>(rr[q], vb)) << q;
    }
}

// The bounds of the tiles that contain neither pivot's position, computed
// once per pass: pair < pl  <=>  image <= a_le and pair <= pr  <=>
// image <= b_le, where a tile wholly before the pivot's position takes the
// pivot's key itself as the bound and one wholly after it the next smaller
// key (no element qualifies when there is none).
template <int DT> struct TileBounds {
    typedef Comp<Key<DT>::KW> C;
    typedef typename Key<DT>::key_t key_t;
    RawBound<DT> ba_before, ba_after, bb_before, bb_after;
    bool any_a_after, any_l_after;
    u32 plx, prx;
    __device__ static TileBounds make(typename C::t pl, typename C::t pr) {
        TileBounds t;
        const key_t plk = (key_t)C::key(pl), prk = (key_t)C::key(pr);
        t.plx = C::idx(pl);
        t.prx = C::idx(pr);
        t.ba_before = RawBound<DT>::le(plk);
        t.bb_before = RawBound<DT>::le(prk);
        t.ba_after = RawBound<DT>::le((key_t)(plk - 1));
        t.bb_after = RawBound<DT>::le((key_t)(prk - 1));
        t.any_a_after = plk != 0;
        t.any_l_after = prk != 0;
        return t;
    }
    // The bounds of tile [tb, te]; false when it contains a pivot's position
    // (then compare pairs).
    __device__ __forceinline__ bool get(u32 tb, u32 te, RawBound<DT>& ba, RawBound<DT>& bb, bool& any_a,
                                        bool& any_l) const {
        if ((plx >= tb && plx <= te) || (prx >= tb && prx <= te)) return false;
        const bool sa = te < plx;  // wholly before pl's position: ties with pl's key are in a
        const bool sl = te <= prx; // wholly at or before pr's position: ties with pr's key are <= pr
        ba.mode = sa ? ba_before.mode : ba_after.mode;
        ba.v = sa ? ba_before.v : ba_after.v;
        bb.mode = sl ? bb_before.mode : bb_after.mode;
        bb.v = sl ? bb_before.v : bb_after.v;
        any_a = sa || any_a_after;
        any_l = sl || any_l_after;
        return true;
    }
};

// The two comparison kinds RawBound<DT>::le can produce: M0 for a bound in
// the non-negative half of an IEEE type (and the only kind of the integer
// types), M1 for a bound in the negative half.
template <int DT> struct RawModes {
    static constexpr int B = DT % DT_DESC;
    static constexpr bool DESC = DT >= DT_DESC;
    static constexpr bool IEEE = B == DT_F32 || B == DT_BF16;
    static constexpr u32 M0 = (B == DT_U32 || B == DT_U64) ? (DESC ? RB_GE_U : RB_LE_U) : (DESC ? RB_GE_S : RB_LE_S);
    static constexpr u32 M1 = IEEE ? (DESC ? RB_LE_U : RB_GE_U) : M0;
};

// The mask of a tile's slots whose pair is at most pr, from the raw bits.
template <int DT, u32 MB>
__device__ __forceinline__ u32 tile_le_raw(const typename Key<DT>::raw_t (&rr)[16], typename RawBound<DT>::cmp_t vb) {
    u32 le = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) le |= (u32)RawBound<DT>::template test<MB>(rr[q], vb) << q;
    return le;
}
template <int DT>
__device__ __forceinline__ u32 tile_le_dispatch(const typename Key<DT>::raw_t (&rr)[16], const RawBound<DT>& bb,
                                                bool any_l) {
    typedef RawModes<DT> M;
    if (!any_l) return 0;
    if (!M::IEEE || bb.mode == M::M0) return tile_le_raw<DT, M::M0>(rr, bb.v);
    return tile_le_raw<DT, M::M1>(rr, bb.v);
}

// tile_masks_raw with the comparison kinds of (ba, bb), chosen at run time
// among the combinations the key type can produce.
template <int DT>
__device__ __forceinline__ void tile_masks_dispatch(const typename Key<DT>::raw_t (&rr)[16], const RawBound<DT>& ba,
                                                    const RawBound<DT>& bb, bool any_a, bool any_l, u32& ma, u32& le) {
    typedef RawModes<DT> M;
    if constexpr (!M::IEEE) {
        tile_masks_raw<DT, M::M0, M::M0>(rr, ba.v, bb.v, any_a, any_l, ma, le);
    } else {
        if (ba.mode == M::M0 && bb.mode == M::M0) tile_masks_raw<DT, M::M0, M::M0>(rr, ba.v, bb.v, any_a, any_l, ma, le);
        else if (ba.mode == M::M1 && bb.mode == M::M1) tile_masks_raw<DT, M::M1, M::M1>(rr, ba.v, bb.v, any_a, any_l, ma, le);
        else if (ba.mode == M::M1) tile_masks_raw<DT, M::M1, M::M0>(rr, ba.v, bb.v, any_a, any_l, ma, le);
        else tile_masks_raw<DT, M::M0, M::M1>(rr, ba.v, bb.v, any_a, any_l, ma, le);
    }
}

// ------------------------------------------------------------ the pass
// Streams the source in tiles of NT*16 elements, classifies every element
// against (lo, pl, pr) and compacts a and b.  A tile with neither costs one
// barrier; otherwise per-warp counts are scanned, one atomic per class and
// tile reserves output room, and every warp writes its elements slot by slot
// as contiguous runs (ballot + popc).

template <int NT> struct PassSmem {
    u32 wa[NT / 32], wb[NT / 32];
    u64 ba[NT / 32], bb[NT / 32];
};

// Barrier among all threads of the block.
struct SyncBlock {
    __device__ static int any(int p) { return __syncthreads_or(p); }
    __device__ static void sync() { __syncthreads(); }
};

// Barrier among the first N threads only (named barrier ID), for kernels with
// a producer warp that does not take part in the tile processing.
template <int ID, int N> struct SyncNamed {
    __device__ static int any(int p) {
        int r;
        asm volatile("{\n\t.reg .pred a, b;\n\tsetp.ne.s32 a, %1, 0;\n\t"
                     "bar.red.or.pred b, %2, %3, a;\n\tselp.s32 %0, 1, 0, b;\n\t}"
                     : "=r"(r)
                     : "r"(p), "n"(ID), "n"(N)
                     : "memory");
        return r;
    }
    __device__ static void sync() { asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(N) : "memory"); }
};

// Classification and compaction of one tile whose 16 elements per thread are
// in registers; pos(s) gives the position of slot s.
//
// Fast path (window starting at the smallest pair, lo = 0): a key below the
// key of pl is in a; a key inside [key(pl), key(pr)] may be in a, b or c and
// is classified exactly on the full (key, position) pair; any other key is in
// c.  So most elements cost one subtraction and one comparison.  EXACT
// classifies every element on the pair (used when lo > 0, a narrowed window).
template <int NT, bool HAS_A, bool EXACT, class Sync, int DT, class CT, class KeyT, class PosF>
__device__ __forceinline__ void classify_emit(const KeyT (&kk)[16], PosF pos, u32 valid, CT lo, CT pl, CT pr,
                                              const Sink<DT>& sink, PassSmem<NT>& sm) {
    typedef Comp<Key<DT>::KW> C;
    const u32 warp = threadIdx.x >> 5, lane = lane_id();
    u32 ma = 0, mb = 0;
    if (EXACT) {
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            const CT c = C::make(kk[s], pos(s));
            const bool ge_pl = c >= pl;
            mb |= (u32)(ge_pl && c <= pr) << s;
            if (HAS_A) ma |= (u32)(!ge_pl && c >= lo) << s;
        }
        ma &= valid;
        mb &= valid;
        if (!Sync::any((int)(ma | mb))) return;
    } else {
        const KeyT plk = (KeyT)C::key(pl), span = (KeyT)C::key(pr) - plk;
        u32 hit = 0;
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            hit |= (u32)((KeyT)(kk[s] - plk) <= span) << s;
            if (HAS_A) ma |= (u32)(kk[s] < plk) << s;
        }
        hit &= valid;
        ma &= valid;
        if (!Sync::any((int)(ma | hit))) return;
        if (hit) { // keys equal to a pivot's key: decide on the position
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                if (!((hit >> s) & 1u)) continue;
                const CT c = C::make(kk[s], pos(s));
                if (c < pl) ma |= 1u << s;
                else if (c <= pr) mb |= 1u << s;
            }
        }
    }

    const u32 wa = __reduce_add_sync(0xffffffffu, (u32)__popc(ma));
    const u32 wb = __reduce_add_sync(0xffffffffu, (u32)__popc(mb));
    if (lane == 0) {
        sm.wa[warp] = wa;
        sm.wb[warp] = wb;
    }
    Sync::sync();
    if (threadIdx.x == 0) {
        u64 ta = 0, tb = 0;
        for (int w = 0; w < NT / 32; ++w) {
            sm.ba[w] = ta;
            sm.bb[w] = tb;
            ta += sm.wa[w];
            tb += sm.wb[w];
        }
        const u64 ga = ta ? atomicAdd((unsigned long long*)sink.cnt_a, (unsigned long long)ta) : 0;
        const u64 gb = tb ? atomicAdd((unsigned long long*)sink.cnt_b, (unsigned long long)tb) : 0;
        for (int w = 0; w < NT / 32; ++w) {
            sm.ba[w] += ga;
            sm.bb[w] += gb;
        }
    }
    Sync::sync();
    u64 ra = sm.ba[warp], rb = sm.bb[warp];
    const u32 below = lanemask_lt();
    typedef typename Key<DT>::raw_t raw_t;
    if (HAS_A && __any_sync(0xffffffffu, ma)) {
        if (ra + wa <= sink.cap_a) { // the warp's run fits: no per-element bound
            raw_t* okp = sink.out_keys + sink.out_base + ra;
            u32* oip = sink.out_idx + sink.out_base + ra;
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const bool bit = (ma >> s) & 1u;
                const u32 bal = __ballot_sync(0xffffffffu, bit);
                const u32 r = (u32)__popc(bal & below);
                const raw_t key = Key<DT>::inv(kk[s]);
                const u32 x = pos(s);
                if (bit) {
                    okp[r] = key;
                    oip[r] = x;
                }
                const u32 c = (u32)__popc(bal);
                okp += c;
                oip += c;
            }
        } else {
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const u32 bal = __ballot_sync(0xffffffffu, (ma >> s) & 1u);
                if ((ma >> s) & 1u) sink.put_a(ra + __popc(bal & below), kk[s], pos(s));
                ra += __popc(bal);
            }
        }
    }
    if (__any_sync(0xffffffffu, mb)) {
        if (rb + wb <= sink.cap_b) {
            auto* bkp = sink.ck + rb;
            u32* bip = sink.ci + rb;
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const bool bit = (mb >> s) & 1u;
                const u32 bal = __ballot_sync(0xffffffffu, bit);
                const u32 r = (u32)__popc(bal & below);
                const u32 x = pos(s);
                if (bit) {
                    bkp[r] = kk[s];
                    bip[r] = x;
                }
                const u32 c = (u32)__popc(bal);
                bkp += c;
                bip += c;
            }
        } else {
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const u32 bal = __ballot_sync(0xffffffffu, (mb >> s) & 1u);
                if ((mb >> s) & 1u) sink.put_b(rb + __popc(bal & below), kk[s], pos(s));
                rb += __popc(bal);
            }
        }
    }
}

// ------------------------------------------------- sparse compaction
// When a and b are a small fraction of the source (every k except around
// n/2), a warp needs no block barrier: one pair comparison per element finds
// the few elements that can be in a or b (pair <= pr); those are appended to
// the warp's own shared-memory queue, which is classified exactly and written
// to the output / candidate buffer with one atomic per class per full queue.
//
// The queue is double-buffered so that a warp never waits for its atomics:
// when the active queue is full, its classes are counted and the two
// reservations issued, and the warp goes on filling the other buffer; the
// full one is written out at the next flush (or at the end of the pass), by
// which time the reservations have long arrived.  A warp that stopped on
// every flush would hold its block's shared-memory stage, and with it the
// whole block, for the atomics' round trip.

template <int KW> struct WarpQ {
    static constexpr int QCAP = KW == 32 ? 256 : 192; // fits the 48 KiB static limit at 8 warps
    typename Comp<KW>::key_t k[2][QCAP];
    u32 i[2][QCAP];
};

// ---- per-lane warp queues.  Lane L's j-th entry sits at index j * 32 + L
// of a buffer, so a lane appends its own hits with no cross-lane step (no
// scan) and without bank conflicts; the lanes' counts differ, so flushing and
// writing go over rows j < the warp's largest count.  Two buffers: a full one
// is counted and its reservations issued, and it is written at the next
// flush, so no warp waits for its atomics.
template <int KW> struct LQ {
    static constexpr u32 PER_LANE = WarpQ<KW>::QCAP / 32; // entries of one lane per buffer
    static constexpr u32 CH = PER_LANE >= 8 ? 8 : 4;      // slots per chunk on the slow path
    static_assert(PER_LANE >= CH, "a chunk of hits always fits an emptied lane");
};
struct LQState {
    u32 cnt;   // this lane's entries in the active buffer
    u32 cq;    // active buffer (warp-uniform)
    u32 pcnt;  // this lane's entries in the other buffer still to be written
    u32 pmax;  // largest pcnt of the warp (0: nothing pending)
    u64 ra, rb; // lane 0: reservations of the pending entries
    __device__ static LQState make() { return LQState{0u, 0u, 0u, 0u, 0ull, 0ull}; }
};

template <int DT>
__device__ __forceinline__ void lq_write(const typename Comp<Key<DT>::KW>::key_t* qk, const u32* qi, u32 cnt, u32 mx,
                                         u64 ra, u64 rb, const Sink<DT>& sink, typename Comp<Key<DT>::KW>::t lo,
                                         typename Comp<Key<DT>::KW>::t pl, typename Comp<Key<DT>::KW>::t pr) {
    typedef Comp<Key<DT>::KW> C;
    typedef typename C::t ct;
    u64 ba = __shfl_sync(0xffffffffu, (unsigned long long)ra, 0);
    u64 bb = __shfl_sync(0xffffffffu, (unsigned long long)rb, 0);
    const u32 below = lanemask_lt(), lane = lane_id();
    for (u32 j = 0; j < mx; ++j) {
        bool isa = false, isb = false;
        typename C::key_t kv = 0;
        u32 iv = 0;
        if (j < cnt) {
            kv = qk[j * 32 + lane];
            iv = qi[j * 32 + lane];
            const ct c = C::make(kv, iv);
            isa = c >= lo && c < pl;
            isb = c >= pl && c <= pr;
        }
        const u32 bala = __ballot_sync(0xffffffffu, isa), balb = __ballot_sync(0xffffffffu, isb);
        if (isa) sink.put_a(ba + __popc(bala & below), kv, iv);
        if (isb) sink.put_b(bb + __popc(balb & below), kv, iv);
        ba += __popc(bala);
        bb += __popc(balb);
    }
}

template <int DT>
__device__ __forceinline__ void lq_flush(WarpQ<Key<DT>::KW>& q, LQState& qs, const Sink<DT>& sink,
                                         typename Comp<Key<DT>::KW>::t lo, typename Comp<Key<DT>::KW>::t pl,
                                         typename Comp<Key<DT>::KW>::t pr) {
    typedef Comp<Key<DT>::KW> C;
    typedef typename C::t ct;
    __syncwarp();
    if (qs.pmax) lq_write<DT>(q.k[qs.cq ^ 1u], q.i[qs.cq ^ 1u], qs.pcnt, qs.pmax, qs.ra, qs.rb, sink, lo, pl, pr);
    const u32 lane = lane_id();
    const u32 mx = __reduce_max_sync(0xffffffffu, qs.cnt);
    u32 ca = 0, cb = 0;
    for (u32 j = 0; j < qs.cnt; ++j) {
        const ct c = C::make(q.k[qs.cq][j * 32 + lane], q.i[qs.cq][j * 32 + lane]);
        ca += (u32)(c >= lo && c < pl);
        cb += (u32)(c >= pl && c <= pr);
    }
    ca = __reduce_add_sync(0xffffffffu, ca);
    cb = __reduce_add_sync(0xffffffffu, cb);
    u64 ra = 0, rb = 0;
    if (lane == 0) {
        if (ca) ra = atomicAdd((unsigned long long*)sink.cnt_a, (unsigned long long)ca);
        if (cb) rb = atomicAdd((unsigned long long*)sink.cnt_b, (unsigned long long)cb);
    }
    qs.ra = ra;
    qs.rb = rb;
    qs.pcnt = qs.cnt;
    qs.pmax = mx;
    qs.cq ^= 1u;
    qs.cnt = 0;
    __syncwarp();
}

template <int DT>
__device__ __forceinline__ void lq_drain(WarpQ<Key<DT>::KW>& q, LQState& qs, const Sink<DT>& sink,
                                         typename Comp<Key<DT>::KW>::t lo, typename Comp<Key<DT>::KW>::t pl,
                                         typename Comp<Key<DT>::KW>::t pr) {
    if (__any_sync(0xffffffffu, qs.cnt)) lq_flush<DT>(q, qs, sink, lo, pl, pr);
    if (qs.pmax) lq_write<DT>(q.k[qs.cq ^ 1u], q.i[qs.cq ^ 1u], qs.pcnt, qs.pmax, qs.ra, qs.rb, sink, lo, pl, pr);
    qs.pmax = 0;
    __syncwarp();
}

// Each lane appends its own hits (bit q of `hit`: slot q; key_at(q) and
// pos(q) for a lane-dependent q) to its part of the active buffer; a flush
// first when some lane's part would overflow.  All 32 lanes call.
template <int DT, class PosF, class KeyAt>
__device__ __forceinline__ void lq_append(u32 hit, PosF pos, KeyAt key_at, typename Comp<Key<DT>::KW>::t lo,
                                          typename Comp<Key<DT>::KW>::t pl, typename Comp<Key<DT>::KW>::t pr,
                                          const Sink<DT>& sink, WarpQ<Key<DT>::KW>& q, LQState& qs) {
    constexpr u32 PER_LANE = LQ<Key<DT>::KW>::PER_LANE, CH = LQ<Key<DT>::KW>::CH;
    if (!__any_sync(0xffffffffu, hit)) return;
    const u32 lane = lane_id();
    if (__any_sync(0xffffffffu, qs.cnt + (u32)__popc(hit) > PER_LANE)) {
        // slow path: chunks of CH slots in turn (at most CH hits each, which
        // always fit a lane once its part is flushed)
#pragma unroll 1
        for (u32 h = 0; h < 16 / CH; ++h) {
            u32 m = (hit >> (CH * h)) & ((1u << CH) - 1u);
            if (__any_sync(0xffffffffu, qs.cnt + (u32)__popc(m) > PER_LANE)) lq_flush<DT>(q, qs, sink, lo, pl, pr);
            while (m) {
                const u32 sq = CH * h + (u32)(__ffs(m) - 1);
                m &= m - 1;
                q.k[qs.cq][qs.cnt * 32 + lane] = key_at(sq);
                q.i[qs.cq][qs.cnt * 32 + lane] = pos((int)sq);
                ++qs.cnt;
            }
        }
        return;
    }
    u32 m = hit;
    while (m) {
        const u32 sq = (u32)(__ffs(m) - 1);
        m &= m - 1;
        q.k[qs.cq][qs.cnt * 32 + lane] = key_at(sq);
        q.i[qs.cq][qs.cnt * 32 + lane] = pos((int)sq);
        ++qs.cnt;
    }
}
// r[q] for a lane-dependent q without dynamic register indexing (which would
// move r to local memory): a tree of selects.
template <class T> __device__ __forceinline__ T pick16(const T (&r)[16], u32 q) {
    T l1[8], l2[4], l3[2];
#pragma unroll
    for (int j = 0; j < 8; ++j) l1[j] = (q & 1u) ? r[2 * j + 1] : r[2 * j];
#pragma unroll
    for (int j = 0; j < 4; ++j) l2[j] = (q & 2u) ? l1[2 * j + 1] : l1[2 * j];
#pragma unroll
    for (int j = 0; j < 2; ++j) l3[j] = (q & 4u) ? l2[2 * j + 1] : l2[2 * j];
    return (q & 8u) ? l3[1] : l3[0];
}

// Register path in sparse mode.
template <int NT, int DT, class Src>
__device__ void pass_tiles_sparse(const Src& src, u64 tile0, u64 tile_step, typename Comp<Src::KW>::t lo,
                                  typename Comp<Src::KW>::t pl, typename Comp<Src::KW>::t pr, const Sink<DT>& sink,
                                  WarpQ<Key<DT>::KW>& q) {
    typedef typename Src::key_t key_t;
    constexpr u64 TILE = (u64)NT * 16;
    typedef Comp<Src::KW> C;
    const u64 ntiles = (src.extent() + TILE - 1) / TILE;
    LQState qs = LQState::make();
    for (u64 t = tile0; t < ntiles; t += tile_step) {
        key_t kk[16];
        u32 ii[16];
        const u64 tb = t * TILE;
        const u32 valid = src.template load16<NT>(tb, kk, ii);
        auto pos = [&](int s) -> u32 {
            if constexpr (Src::IMPLICIT_IDX) return src.template idx_of<NT>(tb, s);
            else return pick16(ii, (u32)s);
        };
        u32 hit = 0;
#pragma unroll
        for (int s = 0; s < 16; ++s) hit |= (u32)(C::make(kk[s], pos(s)) <= pr) << s;
        lq_append<DT>(hit & valid, pos, [&](u32 sq) { return pick16(kk, sq); }, lo, pl, pr, sink, q, qs);
    }
    lq_drain<DT>(q, qs, sink, lo, pl, pr);
}

// Register path: every thread loads its 16 elements of each tile itself.
template <int NT, bool HAS_A, bool EXACT, int DT, class Src>
__device__ void pass_tiles(const Src& src, u64 tile0, u64 tile_step,
                           typename Comp<Src::KW>::t lo, typename Comp<Src::KW>::t pl,
                           typename Comp<Src::KW>::t pr, const Sink<DT>& sink,
                           PassSmem<NT>& sm) {
    typedef typename Src::key_t key_t;
    constexpr u64 TILE = (u64)NT * 16;
    const u64 ntiles = (src.extent() + TILE - 1) / TILE;
    for (u64 t = tile0; t < ntiles; t += tile_step) {
        key_t kk[16];
        u32 ii[16];
        const u64 tb = t * TILE;
        const u32 valid = src.template load16<NT>(tb, kk, ii);
        auto pos = [&](int s) -> u32 {
            if constexpr (Src::IMPLICIT_IDX) return src.template idx_of<NT>(tb, s);
            else return ii[s];
        };
        classify_emit<NT, HAS_A, EXACT, SyncBlock>(kk, pos, valid, lo, pl, pr, sink, sm);
    }
}

// ------------------------------------------------------- radix selection
// Block-wide selection of the elements of given 0-based ranks among
// v[0..count) (duplicates counted), by most-significant-digit-first radix
// selection over 8-bit digits of the composite.  Used to read the pivots off
// the sample (the sample order statistics of ranks k|S|/n -/+ Delta) and the
// k-th element off the final candidates.  Equivalent to sorting and indexing.
//
// Per digit, every element that still matches a target's prefix is counted
// into that target's 256-bin histogram.  Lanes of a warp holding the same
// digit are grouped with eight ballots (one per digit bit), so each distinct
// digit costs one shared-memory atomic per warp even when all keys tie; warps
// without a matching element skip the grouping.  A target is resolved as
// soon as its bin holds a single element.

template <int KW, int NTGT> struct RadixSmem {
    typedef typename Comp<KW>::t ct;
    ct diff[32];
    u32 hist[NTGT][256];
    ct prefix[NTGT];
    ct mask[NTGT];
    u32 rank[NTGT];
    u32 done[NTGT];
    u32 unique[NTGT];
    ct result[NTGT];
};

// Lanes whose 8-bit `dig` equals this lane's (all 32 lanes call).
__device__ __forceinline__ u32 warp_same_digit(u32 dig) {
    u32 same = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const u32 bal = __ballot_sync(0xffffffffu, (dig >> b) & 1u);
        same &= ((dig >> b) & 1u) ? bal : ~bal;
    }
    return same;
}

template <int KW, int NTGT>
__device__ void block_select_ranks(const typename Comp<KW>::t* v, u32 count, const u32 (&rank)[NTGT],
                                   RadixSmem<KW, NTGT>& sm) {
    typedef Comp<KW> C;
    typedef typename C::t ct;
    const u32 tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    // Leading digits shared by every element need no pass: find the highest
    // bit in which any element differs from the first one.
    ct x = 0;
    if (count > 0) {
        const ct v0 = v[0];
        for (u32 i = tid; i < count; i += blockDim.x) x |= v[i] ^ v0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const u64 lo64 = __shfl_xor_sync(0xffffffffu, (unsigned long long)(u64)x, o);
        ct y = (ct)lo64;
        if constexpr (sizeof(ct) > 8) y |= (ct)__shfl_xor_sync(0xffffffffu, (unsigned long long)(u64)((u128)x >> 64), o) << 64;
        x |= y;
    }
    if (lane == 0) sm.diff[warp] = x;
    __syncthreads();
    ct diff = 0;
    for (u32 w = 0; w < (blockDim.x >> 5); ++w) diff |= sm.diff[w];
    constexpr int TOTAL = C::DIGITS * 8;
    int d0 = C::DIGITS; // all equal: every target is v[0]
    if (diff != 0) d0 = (TOTAL - bit_length_fast(diff)) / 8;
    ct top = 0; // mask of the shared leading digits
    if (d0 > 0) {
        const int keep = 8 * (C::DIGITS - (d0 < C::DIGITS ? d0 : C::DIGITS));
        if constexpr (TOTAL == 64) top = keep >= 64 ? (ct)0 : (ct)(~(u64)0 << keep);
        else top = (keep >= TOTAL) ? (ct)0 : (ct)(((ct)1 << TOTAL) - 1) & ~(ct)(((ct)1 << keep) - 1);
    }
    if (tid < NTGT) {
        sm.prefix[tid] = count > 0 ? (v[0] & top) : (ct)0;
        sm.mask[tid] = top;
        sm.rank[tid] = rank[tid];
        sm.done[tid] = d0 >= C::DIGITS;
        sm.unique[tid] = 0;
    }
    __syncthreads();
    for (int d = d0; d < C::DIGITS; ++d) {
        bool all_done = true;
#pragma unroll
        for (int t = 0; t < NTGT; ++t) all_done = all_done && sm.done[t];
        if (all_done) break; // uniform: every thread reads the same smem
        for (u32 i = tid; i < NTGT * 256; i += blockDim.x) (&sm.hist[0][0])[i] = 0;
        __syncthreads();
        ct pfx[NTGT], msk[NTGT];
        bool live[NTGT];
#pragma unroll
        for (int t = 0; t < NTGT; ++t) {
            pfx[t] = sm.prefix[t];
            msk[t] = sm.mask[t];
            live[t] = !sm.done[t];
        }
        for (u32 base = 0; base < count; base += blockDim.x) {
            const u32 i = base + tid;
            const bool ok = i < count;
            const ct c = ok ? v[i] : (ct)0;
            const u32 dig = C::digit(c, d);
            bool m[NTGT];
            bool anym = false;
#pragma unroll
            for (int t = 0; t < NTGT; ++t) {
                m[t] = ok && live[t] && ((c & msk[t]) == pfx[t]);
                anym = anym || m[t];
            }
            if (!__any_sync(0xffffffffu, anym)) continue;
            const u32 same = warp_same_digit(dig);
#pragma unroll
            for (int t = 0; t < NTGT; ++t) {
                const u32 grp = same & __ballot_sync(0xffffffffu, m[t]);
                if (m[t] && lane == (u32)(__ffs(grp) - 1)) atomicAdd(&sm.hist[t][dig], (u32)__popc(grp));
            }
        }
        __syncthreads();
        if (warp < (u32)NTGT && live[warp]) {
            const int t = warp;
            u32 h[8], s = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                h[j] = sm.hist[t][lane * 8 + j];
                s += h[j];
            }
            u32 incl = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (u32)o) incl += y;
            }
            const u32 excl = incl - s;
            const u32 r = sm.rank[t];
            if (r >= excl && r < incl) {
                // the bin of this lane's 8 holding rank r, and the count below it
                u32 acc = excl, hb = 0;
                int b = -1;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (b < 0) {
                        if (r < acc + h[j]) {
                            b = j;
                            hb = h[j];
                        } else {
                            acc += h[j];
                        }
                    }
                }
                const u32 bin = lane * 8 + b;
                const int shift = (C::DIGITS - 1 - d) * 8;
                sm.prefix[t] = pfx[t] | ((ct)bin << shift);
                sm.mask[t] = msk[t] | ((ct)0xFFu << shift);
                sm.rank[t] = r - acc;
                if (hb == 1) {
                    sm.unique[t] = 1;
                    sm.done[t] = 1;
                } else if (d == C::DIGITS - 1) {
                    sm.done[t] = 1;
                }
            }
        }
        __syncthreads();
    }
    // Targets fixed on every digit are the prefix itself; a target whose bin
    // held one element is that element.
    if (tid < NTGT) sm.result[tid] = sm.prefix[tid];
    __syncthreads();
#pragma unroll
    for (int t = 0; t < NTGT; ++t) {
        if (!sm.unique[t]) continue;
        const ct msk = sm.mask[t], pfx = sm.prefix[t];
        for (u32 i = tid; i < count; i += blockDim.x)
            if ((v[i] & msk) == pfx) sm.result[t] = v[i];
    }
    __syncthreads();
}

// A composite from lane `src` (all 32 lanes call).
template <class CT> __device__ __forceinline__ CT shfl_comp(CT x, u32 src) {
    CT y = (CT)__shfl_sync(0xffffffffu, (unsigned long long)(u64)x, src);
    if constexpr (sizeof(CT) > 8)
        y |= (CT)__shfl_sync(0xffffffffu, (unsigned long long)(u64)((u128)x >> 64), src) << 64;
    return y;
}

// Selection among at most 64 elements by counting (one warp, no shared
// memory): lane l holds v[l] and v[l + 32]; an element's place in the sorted
// order, ties by index, is the number of smaller elements plus the number of
// equal ones before it, and exactly one element has place `rank`.
template <int KW>
__device__ typename Comp<KW>::t warp_rank_small(const typename Comp<KW>::t* v, u32 count, u32 rank) {
    typedef typename Comp<KW>::t ct;
    const u32 lane = lane_id();
    const bool h0 = lane < count, h1 = lane + 32 < count;
    const ct e0 = h0 ? v[lane] : (ct)0, e1 = h1 ? v[lane + 32] : (ct)0;
    u32 p0 = 0, p1 = 0;
    const u32 n0 = count < 32 ? count : 32;
    for (u32 j = 0; j < n0; ++j) { // element j (index j < 32)
        const ct o = shfl_comp(e0, j);
        p0 += (u32)(o < e0 || (o == e0 && j < lane));
        p1 += (u32)(o <= e1); // index j < lane + 32
    }
    for (u32 j = 0; j + 32 < count; ++j) { // element 32 + j
        const ct o = shfl_comp(e1, j);
        p0 += (u32)(o < e0); // index 32 + j > lane
        p1 += (u32)(o < e1 || (o == e1 && j < lane));
    }
    const u32 m0 = __ballot_sync(0xffffffffu, h0 && p0 == rank);
    const u32 m1 = __ballot_sync(0xffffffffu, h1 && p1 == rank);
    return m0 ? shfl_comp(e0, (u32)__ffs(m0) - 1) : shfl_comp(e1, (u32)__ffs(m1) - 1);
}

// Warp-level version for small sets: one warp selects the element of 0-based
// rank `rank` among v[0..count) with its own 256-bin histogram in shared
// memory (no block barrier, so several warps can select concurrently); up to
// 64 elements by counting instead.
template <int KW>
__device__ typename Comp<KW>::t warp_select_rank(const typename Comp<KW>::t* v, u32 count, u32 rank, u32* hist) {
    typedef Comp<KW> C;
    typedef typename C::t ct;
    if (count <= 64) return warp_rank_small<KW>(v, count, rank);
    const u32 lane = lane_id();
    const ct v0 = v[0];
    ct x = 0;
    for (u32 i = lane; i < count; i += 32) x |= v[i] ^ v0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ct y = (ct)__shfl_xor_sync(0xffffffffu, (unsigned long long)(u64)x, o);
        if constexpr (sizeof(ct) > 8) y |= (ct)__shfl_xor_sync(0xffffffffu, (unsigned long long)(u64)((u128)x >> 64), o) << 64;
        x |= y;
    }
    if (x == 0) return v0; // all equal
    constexpr int TOTAL = C::DIGITS * 8;
    const int d0 = (TOTAL - bit_length_fast(x)) / 8;
    ct mask = 0;
    if (d0 > 0) {
        const int keep = 8 * (C::DIGITS - d0);
        mask = (TOTAL == 64) ? (ct)(~(u64)0 << keep) : (ct)((((ct)1 << TOTAL) - 1) & ~(((ct)1 << keep) - 1));
    }
    ct prefix = v0 & mask;
    u32 r = rank;
    for (int d = d0; d < C::DIGITS; ++d) {
#pragma unroll
        for (int j = 0; j < 8; ++j) hist[lane * 8 + j] = 0;
        __syncwarp();
        for (u32 i = lane; i < count; i += 32) {
            const ct c = v[i];
            if ((c & mask) == prefix) atomicAdd(&hist[C::digit(c, d)], 1u);
        }
        __syncwarp();
        u32 h[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            h[j] = hist[lane * 8 + j];
            sum += h[j];
        }
        u32 incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (u32)o) incl += y;
        }
        const u32 excl = incl - sum;
        u32 bin = 0, below = 0, hb = 0;
        const bool mine = r >= excl && r < incl;
        if (mine) {
            u32 acc = excl;
            int b = -1;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if (b < 0) {
                    if (r < acc + h[j]) {
                        b = j;
                        hb = h[j];
                    } else {
                        acc += h[j];
                    }
                }
            }
            bin = lane * 8 + b;
            below = acc;
        }
        const u32 src = __ffs(__ballot_sync(0xffffffffu, mine)) - 1;
        bin = __shfl_sync(0xffffffffu, bin, src);
        below = __shfl_sync(0xffffffffu, below, src);
        hb = __shfl_sync(0xffffffffu, hb, src);
        const int shift = (C::DIGITS - 1 - d) * 8;
        prefix |= (ct)bin << shift;
        mask |= (ct)0xFFu << shift;
        r -= below;
        __syncwarp();
        if (hb == 1) { // the single element with this prefix
            ct res = 0;
            bool found = false;
            for (u32 i = lane; i < count; i += 32) {
                const ct c = v[i];
                if ((c & mask) == prefix) {
                    res = c;
                    found = true;
                }
            }
            const u32 who = __ffs(__ballot_sync(0xffffffffu, found)) - 1;
            const u64 lo64 = __shfl_sync(0xffffffffu, (unsigned long long)(u64)res, who);
            ct out = (ct)lo64;
            if constexpr (sizeof(ct) > 8) out |= (ct)__shfl_sync(0xffffffffu, (unsigned long long)(u64)((u128)res >> 64), who) << 64;
            return out;
        }
    }
    return prefix;
}

// ------------------------------------------------ selection by histogram
// Block-wide selection of the element of 0-based rank `rank` among
// v[0..count) (duplicates counted), all of which lie in the window [lo, hi]:
// a histogram of 2^HS_BITS equal bins over the window (one pass, one shared
// atomic per element), a prefix over the bins to find the bin holding the
// rank, then either the bin's elements gathered and ranked by one warp
// (warp_select_rank) or, for a larger bin, the window narrowed to that bin
// and the step repeated.  A bin of width 1 holds copies of one composite, so
// at most ceil(96 / HS_BITS) steps are taken.  Equivalent to sorting and
// indexing; for sets that are spread over their window (samples, candidate
// sets) it costs about two passes over them.
constexpr u32 HS_BITS = 11;
constexpr u32 HS_BINS = 1u << HS_BITS;
constexpr u32 HS_GATHER = 512;

template <int KW> struct HistSelSmem {
    typedef typename Comp<KW>::t ct;
    u32 hist[HS_BINS];
    ct gath[HS_GATHER];
    u32 whist[2][256];
    u32 wsum[32];
    ct wlo, whi, result, res2[2];
    u32 rank, bin, below, cnt, ng;
    u32 bin2[2], below2[2], cnt2[2], ng2[2];
};

template <int KW, int NT>
__device__ typename Comp<KW>::t block_select_hist(const typename Comp<KW>::t* v, u32 count, typename Comp<KW>::t lo,
                                                   typename Comp<KW>::t hi, u32 rank, HistSelSmem<KW>& hs) {
    typedef typename Comp<KW>::t ct;
    static_assert(HS_BINS % NT == 0 && NT <= 1024, "bins per thread");
    constexpr u32 PER = HS_BINS / NT; // consecutive bins per thread in the prefix
    const u32 tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    if (tid == 0) {
        hs.wlo = lo;
        hs.whi = hi;
        hs.rank = rank;
    }
    __syncthreads();
    for (int step = 0; step < 12; ++step) {
        const ct wlo = hs.wlo, whi = hs.whi;
        const int bl = bit_length_fast((ct)(whi - wlo));
        const u32 sh = bl > (int)HS_BITS ? (u32)(bl - HS_BITS) : 0u;
        auto bin_of = [&](ct c) -> u32 {
            const ct d = (ct)(c - wlo) >> sh;
            return d < (ct)HS_BINS ? (u32)d : HS_BINS - 1;
        };
        for (u32 i = tid; i < HS_BINS; i += NT) hs.hist[i] = 0;
        __syncthreads();
        for (u32 i = tid; i < count; i += NT) {
            const ct c = v[i];
            if (c >= wlo && c <= whi) atomicAdd(&hs.hist[bin_of(c)], 1u);
        }
        __syncthreads();
        // the bin holding the rank: per-thread sums of PER bins, block scan
        u32 h[PER], t = 0;
#pragma unroll
        for (u32 q = 0; q < PER; ++q) {
            h[q] = hs.hist[tid * PER + q];
            t += h[q];
        }
        u32 incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (u32)o) incl += y;
        }
        if (lane == 31) hs.wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const u32 x = lane < NT / 32 ? hs.wsum[lane] : 0u;
            u32 wi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u32 y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= (u32)o) wi += y;
            }
            if (lane < NT / 32) hs.wsum[lane] = wi - x;
        }
        __syncthreads();
        const u32 r = hs.rank;
        u32 run = hs.wsum[warp] + incl - t;
#pragma unroll
        for (u32 q = 0; q < PER; ++q) {
            if (h[q] && r >= run && r < run + h[q]) {
                hs.bin = tid * PER + q;
                hs.below = run;
                hs.cnt = h[q];
            }
            run += h[q];
        }
        if (tid == 0) hs.ng = 0;
        __syncthreads();
        const u32 b = hs.bin, cnt = hs.cnt, rr = r - hs.below;
        if (cnt <= HS_GATHER) {
            // the bin's elements (few: each takes its own slot), then one
            // warp ranks them
            for (u32 i = tid; i < count; i += NT) {
                const ct c = v[i];
                if (c >= wlo && c <= whi && bin_of(c) == b) {
                    const u32 slot = atomicAdd(&hs.ng, 1u);
                    if (slot < HS_GATHER) hs.gath[slot] = c;
                }
            }
            __syncthreads();
            if (warp == 0) {
                const ct res = warp_select_rank<KW>(hs.gath, cnt, rr, hs.whist[0]);
                if (lane == 0) hs.result = res;
            }
            __syncthreads();
            return hs.result;
        }
        // a large bin: narrow the window to it and repeat
        if (tid == 0) {
            const ct nlo = (ct)(wlo + ((ct)b << sh));
            const ct top = (ct)(nlo + (((ct)1 << sh) - 1)); // wraps past the largest composite
            hs.wlo = nlo;
            hs.whi = (b == HS_BINS - 1 || top > whi || top < nlo) ? whi : top;
            hs.rank = rr;
        }
        __syncthreads();
    }
    return hs.wlo; // not reached: each step narrows the window by 2^HS_BITS
}

// The elements of ranks r0 and r1 among v[0..count) (all in [lo, hi]) at
// once: one histogram pass finds both bins, one gather pass collects both,
// and two warps rank them concurrently.  A bin too large to gather is
// selected by block_select_hist on that bin's window alone.
template <int KW, int NT>
__device__ void block_select_two(const typename Comp<KW>::t* v, u32 count, typename Comp<KW>::t lo,
                                 typename Comp<KW>::t hi, u32 r0, u32 r1, HistSelSmem<KW>& hs,
                                 typename Comp<KW>::t& out0, typename Comp<KW>::t& out1) {
    typedef typename Comp<KW>::t ct;
    static_assert(HS_BINS % NT == 0 && NT <= 1024 && NT >= 64, "bins per thread");
    constexpr u32 PER = HS_BINS / NT;
    constexpr u32 HALF = HS_GATHER / 2;
    const u32 tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const int bl = bit_length_fast((ct)(hi - lo));
    const u32 sh = bl > (int)HS_BITS ? (u32)(bl - HS_BITS) : 0u;
    auto bin_of = [&](ct c) -> u32 {
        const ct d = (ct)(c - lo) >> sh;
        return d < (ct)HS_BINS ? (u32)d : HS_BINS - 1;
    };
    for (u32 i = tid; i < HS_BINS; i += NT) hs.hist[i] = 0;
    __syncthreads();
    for (u32 i = tid; i < count; i += NT) {
        const ct c = v[i];
        if (c >= lo && c <= hi) atomicAdd(&hs.hist[bin_of(c)], 1u);
    }
    __syncthreads();
    u32 h[PER], t = 0;
#pragma unroll
    for (u32 q = 0; q < PER; ++q) {
        h[q] = hs.hist[tid * PER + q];
        t += h[q];
    }
    u32 incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (u32)o) incl += y;
    }
    if (lane == 31) hs.wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const u32 x = lane < NT / 32 ? hs.wsum[lane] : 0u;
        u32 wi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= (u32)o) wi += y;
        }
        if (lane < NT / 32) hs.wsum[lane] = wi - x;
    }
    __syncthreads();
    u32 run = hs.wsum[warp] + incl - t;
#pragma unroll
    for (u32 q = 0; q < PER; ++q) {
        if (h[q] && r0 >= run && r0 < run + h[q]) {
            hs.bin2[0] = tid * PER + q;
            hs.below2[0] = run;
            hs.cnt2[0] = h[q];
        }
        if (h[q] && r1 >= run && r1 < run + h[q]) {
            hs.bin2[1] = tid * PER + q;
            hs.below2[1] = run;
            hs.cnt2[1] = h[q];
        }
        run += h[q];
    }
    if (tid == 0) hs.ng2[0] = hs.ng2[1] = 0;
    __syncthreads();
    const u32 b0 = hs.bin2[0], b1 = hs.bin2[1], c0 = hs.cnt2[0], c1 = hs.cnt2[1];
    const bool same = b0 == b1;
    if (same ? c0 <= HS_GATHER : (c0 <= HALF && c1 <= HALF)) {
        const u32 off1 = same ? 0u : HALF;
        const u32 cap0 = same ? HS_GATHER : HALF;
        // the two bins' elements (few: each takes its own slot)
        for (u32 i = tid; i < count; i += NT) {
            const ct c = v[i];
            if (c >= lo && c <= hi) {
                const u32 b = bin_of(c);
                if (b == b0) {
                    const u32 slot = atomicAdd(&hs.ng2[0], 1u);
                    if (slot < cap0) hs.gath[slot] = c;
                } else if (b == b1) {
                    const u32 slot = atomicAdd(&hs.ng2[1], 1u);
                    if (slot < HALF) hs.gath[off1 + slot] = c;
                }
            }
        }
        __syncthreads();
        if (warp < 2) {
            const ct res = warp == 0 ? warp_select_rank<KW>(hs.gath, c0, r0 - hs.below2[0], hs.whist[0])
                                     : warp_select_rank<KW>(hs.gath + off1, c1, r1 - hs.below2[1], hs.whist[1]);
            if (lane == 0) hs.res2[warp] = res;
        }
        __syncthreads();
        out0 = hs.res2[0];
        out1 = hs.res2[1];
        return;
    }
    // a large bin: select inside its own window
    const u32 bb[2] = {b0, b1}, rr[2] = {r0 - hs.below2[0], r1 - hs.below2[1]};
    ct res[2];
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
        const ct nlo = (ct)(lo + ((ct)bb[q] << sh));
        const ct top = (ct)(nlo + (((ct)1 << sh) - 1));
        const ct nhi = (bb[q] == HS_BINS - 1 || top > hi || top < nlo) ? hi : top;
        __syncthreads(); // every thread has read the bins above before hs is reused
        res[q] = block_select_hist<KW, NT>(v, count, nlo, nhi, rr[q], hs);
    }
    out0 = res[0];
    out1 = res[1];
}

// ------------------------------------------------------------- sampling
// Per-partition sampling (Section 2 "Bernoulli sampling"; Section 4.1: the
// sample is drawn from every PE in proportion to its share).  The source is
// cut into `parts` equal partitions; draw j belongs to partition j mod parts
// (so every partition gets the same share of draws, i.e. a share proportional
// to its size) and picks a position uniformly inside it.  The uniform
// numbers come from Philox4x32-10 keyed by the seed: the block of counter
// (j0, level, salt, const) gives draws j0..j0+3.  Draws that fall outside the
// window are discarded.  Returns the number kept (<= cap).

template <class Src>
__device__ u32 block_sample(const Src& src, typename Comp<Src::KW>::t lo, typename Comp<Src::KW>::t hi,
                            u32 draws, u32 parts, u64 seed, u32 level, u32 salt,
                            typename Comp<Src::KW>::t* samp, u32 cap, u32* kept_smem) {
    typedef Comp<Src::KW> C;
    typedef typename C::t ct;
    const u32 tid = threadIdx.x;
    if (tid == 0) *kept_smem = 0;
    __syncthreads();
    const u64 m = src.m;
    const u32 p = (u32)((u64)parts < m ? parts : m);
    // partition q covers [q*len + min(q, rem), ...) with len + (q < rem) elements
    const u64 len = m / p;
    const u32 rem = (u32)(m - len * p);
    constexpr int U = 8; // draws per thread per round: two Philox blocks
    for (u32 base = 0; base < draws; base += blockDim.x * U) {
        u64 pos[U];
        bool ok[U];
#pragma unroll
        for (int h = 0; h < U / 4; ++h) {
            // one Philox block gives the four draws j0..j0+3
            const u32 j0 = base + (h * blockDim.x + tid) * 4;
            const Philox4 r = philox4x32_10(j0, level, salt, 0x5A3E1Du, (u32)seed, (u32)(seed >> 32));
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const u32 j = j0 + q;
                const int u = h * 4 + q;
                ok[u] = j < draws;
                const u32 part = j % p; // draws dealt round-robin: equal share per partition
                const u64 plo = (u64)part * len + (part < rem ? part : rem);
                const u64 psz = len + (part < rem ? 1 : 0);
                pos[u] = plo + (((u64)r.v[q] * psz) >> 32);
            }
        }
        typename Src::key_t kk[U];
        u32 ii[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (ok[u]) src.at(pos[u], kk[u], ii[u]);
            else { kk[u] = 0; ii[u] = 0; }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const ct c = C::make(kk[u], ii[u]);
            const bool keep = ok[u] && c >= lo && c <= hi;
            const u32 bal = __ballot_sync(0xffffffffu, keep);
            u32 slot0 = 0;
            if (lane_id() == 0 && bal) slot0 = atomicAdd(kept_smem, (u32)__popc(bal));
            slot0 = __shfl_sync(0xffffffffu, slot0, 0);
            const u32 slot = slot0 + __popc(bal & lanemask_lt());
            if (keep && slot < cap) samp[slot] = c;
        }
    }
    __syncthreads();
    const u32 kept = *kept_smem;
    __syncthreads();
    return kept < cap ? kept : cap;
}

// --------------------------------------------------- branch of "select"
// Consumes the counters of the pass just run (Algorithm "select": if
// n_a >= k recurse into a; if n_a + n_b < k recurse into c with
// k - n_a - n_b; else into b with k - n_a).  a is never materialised apart
// from the output, so "recurse into a" narrows the window on the same source;
// "recurse into c" commits a only and narrows the window to [l, hi]; the
// common case continues on the candidate buffer b.  One thread.

__device__ inline void decide(SelState& s) {
    if (!s.pending) return;
    s.pending = 0;
    const u64 na = s.cnt_a, nb = s.cnt_b;
    if (s.level == 1) s.first_cand = nb;
    if (na >= s.k_rem) {          // l too high: answer in a = [lo, pl)
        s.hi = s.pl - 1;
        s.m_win = na;
        s.failures++;
        return;
    }
    s.out_base += na;             // all of a is selected
    s.k_rem -= na;
    s.m_win -= na;
    s.lo = s.pl;
    if (nb >= s.k_rem) {          // answer in b = [pl, pr]
        s.hi = s.pr;
        s.m_win = nb;
        if (nb <= s.cap_b) {
            s.src = s.dst;
            s.m_src = nb;
        } else {
            s.overflows++;
        }
    } else {
        s.failures++;             // r too low: window [pl, hi] on same source
    }
}

// Pivot ranks in a sample of `kept` elements of a window of m_win elements
// for rank k_rem: the sample count below the target is binomial with mean
// kept*k_rem/m_win; the margin is z standard deviations plus z^2/3 + 1, a
// Bernstein-type allowance that keeps the tails small when the mean is near
// 0 (the paper's Delta = p^(1/4 + delta) plays this role, Section 2).
__device__ inline void pivot_ranks(u32 kept, u64 m_win, u64 k_rem, float z, bool raw,
                                   long long& jl, long long& jr) {
    // single precision: the ranks only steer the bracket (any pivots give the
    // exact result), and double precision is slow on this part
    const float s = (float)kept, m = __ull2float_rn(m_win);
    const float mu_le = s * (__ull2float_rn(k_rem) / m);
    const float mu_lt = s * (__ull2float_rn(k_rem - 1) / m);
    float dle, dlt;
    if (raw) {
        dle = z;
        dlt = z;
    } else {
        const float vle = mu_le * (1.0f - mu_le / s), vlt = mu_lt * (1.0f - mu_lt / s);
        const float extra = z * z / 3.0f + 1.0f;
        dle = z * sqrtf(fmaxf(vle, 0.0f)) + extra;
        dlt = z * sqrtf(fmaxf(vlt, 0.0f)) + extra;
    }
    jl = (long long)floorf(mu_le - dle) - 1;
    jr = (long long)ceilf(mu_lt + dlt);
}

} // namespace topk
