// batched_common.cuh -- device helpers of the batched day kernels (batched.cu,
// batched_bwd.cu): per-lane vectors of SPL sets, the grouped row sums with their
// load pipeline, and the (Bp, SPL) schedules built.
#pragma once

#include <algorithm>

#include "gabm_internal.cuh"
#include "rowsum.cuh"

// Resident blocks per SM the batched day kernels are compiled for (register budget
// 65536 / (256 x blocks) per thread).
#ifndef GABM_BFWD_MINBLOCKS
#define GABM_BFWD_MINBLOCKS 3
#endif
#ifndef GABM_BBWD_MINBLOCKS
#define GABM_BBWD_MINBLOCKS 2
#endif

namespace gabm {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kUmin = 5.9604644775390625e-8f;   // 2^-24: the smallest uniform (u < p is then impossible)

// Adds w * x (x finite).  Invalid entries carry w = 0: s + 0 * x = s exactly for the
// plain sum (s is never -0); the compensated sum skips them explicitly.
template <bool KAHAN>
__device__ __forceinline__ void acc_add(float &s, float &c, float w, float x, bool take) {
    if (KAHAN) kahan_add_if(s, c, w * x, take);
    else s = __fmaf_rn(w, x, s);
}

// ---- per-lane vectors of SPL sets ----------------------------------------
// SPL int16 exposure days travel as SPL/2 32-bit words, SPL floats as one or two
// vector accesses; the predicated forms load nothing (zeros) when !ok.
template <int SPL>
__device__ __forceinline__ void ld_words(const uint32_t *p, bool ok, uint32_t (&w)[SPL / 2]) {
    const uint32_t pr = ok;
    if constexpr (SPL == 2) {
        w[0] = 0u;
        asm("{ .reg .pred q; setp.ne.u32 q, %2, 0; @q ld.global.u32 %0, [%1]; }" : "+r"(w[0]) : "l"(p), "r"(pr));
    } else if constexpr (SPL == 4) {
        w[0] = w[1] = 0u;
        asm("{ .reg .pred q; setp.ne.u32 q, %3, 0; @q ld.global.v2.u32 {%0, %1}, [%2]; }"
                     : "+r"(w[0]), "+r"(w[1]) : "l"(p), "r"(pr));
    } else {
        w[0] = w[1] = w[2] = w[3] = 0u;
        asm("{ .reg .pred q; setp.ne.u32 q, %5, 0; @q ld.global.v4.u32 {%0, %1, %2, %3}, [%4]; }"
                     : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3]) : "l"(p), "r"(pr));
    }
}

template <int SPL>
__device__ __forceinline__ void ld_floats(const float *p, bool ok, float (&v)[SPL]) {
    const uint32_t pr = ok;
#pragma unroll
    for (int h = 0; h < SPL; ++h) v[h] = 0.f;
    if constexpr (SPL == 2) {
        asm("{ .reg .pred q; setp.ne.u32 q, %3, 0; @q ld.global.v2.f32 {%0, %1}, [%2]; }"
                     : "+f"(v[0]), "+f"(v[1]) : "l"(p), "r"(pr));
    } else {
#pragma unroll
        for (int h = 0; h < SPL; h += 4)
            asm("{ .reg .pred q; setp.ne.u32 q, %5, 0; @q ld.global.v4.f32 {%0, %1, %2, %3}, [%4]; }"
                         : "+f"(v[h]), "+f"(v[h + 1]), "+f"(v[h + 2]), "+f"(v[h + 3]) : "l"(p + h), "r"(pr));
    }
}

template <int SPL>
__device__ __forceinline__ void st_floats(float *p, const float (&v)[SPL]) {
    if constexpr (SPL == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
#pragma unroll
        for (int h = 0; h < SPL; h += 4)
            *reinterpret_cast<float4 *>(p + h) = make_float4(v[h], v[h + 1], v[h + 2], v[h + 3]);
    }
}

template <int SPL>
__device__ __forceinline__ void st_words(uint32_t *p, const uint32_t (&w)[SPL / 2]) {
    if constexpr (SPL == 2) *p = w[0];
    else if constexpr (SPL == 4) *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
    else *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ int half_of(uint32_t w, int h) { return (int16_t)(h ? (w >> 16) : (w & 0xffffu)); }

// Lane of the i-th (0-based) set bit of m; i < popc(m).
__device__ __forceinline__ int nth_set_bit(uint32_t m, int i) {
    uint32_t pos;
    asm("fns.b32 %0, %1, 0, %2;" : "=r"(pos) : "r"(m), "r"(i + 1));
    return (int)(pos & 31u);
}

// c[t - e] for 1 <= t - e < L, else 0, from a table c_s[0..kMaxL] with c_s[k] = 0 for k >= L:
// t - e is negative for susceptible agents (e = NEVER) and huge for padding (e = kPad), both
// of which clamp (as unsigned) to L, and c[0] = 0.
__device__ __forceinline__ float infect_lut(int e, const float *c_s, int t, unsigned L) {
    return c_s[min((unsigned)(t - e), L)];
}

// Row data of one pass (one row per group), loaded a pass ahead of use: the
// lane's exposure words of its row, the row's entry range and the first chunk
// of its entries (entry q for lane q of the group).
template <int SPL>
struct PassRow {
    uint32_t ew[SPL / 2];
    uint32_t p0, len;      // entries [p0, p0 + len)
    uint32_t j0;           // column and weight of entry q, when q < len
    float w0;
};

// Loads the pass row of tile row r (0..31) into pr; lane r holds the row bounds
// (rowptr of tile row r and r + 1) in rp_lo / rp_hi.  Called by all 32 lanes.
template <int SPL>
__device__ __forceinline__ void load_pass_row(const Csr &m, const uint32_t *ew_ptr, uint32_t rp_lo, uint32_t rp_hi,
                                              int r, int q, PassRow<SPL> &pr) {
    pr.p0 = __shfl_sync(kFull, rp_lo, r);
    pr.len = __shfl_sync(kFull, rp_hi, r) - pr.p0;
    ld_words<SPL>(ew_ptr, true, pr.ew);
    const bool v = (uint32_t)q < pr.len;
    pr.j0 = ld_cs_if(m.col + pr.p0 + q, v);
    pr.w0 = ld_cs_if(m.w + pr.p0 + q, v);
}

// V marked entries of the current chunk, taken from mm in entry order (lowest lane
// of the group first): their columns and weights broadcast from the lanes holding
// them, every lane's gathers issued before any of their values is used, then the
// sums.  Slots past the group's last marked entry carry weight 0 and load nothing.
template <int V, int LPR, int SPL, bool KAHAN, class Raw, class Ld, class Val>
__device__ __forceinline__ void gather_batch(unsigned &mm, uint32_t j, float w, Ld &ld, Val &val, float (&sum)[SPL],
                                             float (&comp)[SPL]) {
    uint32_t jv[V];
    float wv[V];
    bool ok[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
        ok[u] = mm != 0u;
        const int src = ok[u] ? __ffs(mm) - 1 : 0;
        mm &= mm - 1u;
        jv[u] = __shfl_sync(kFull, j, src, LPR);
        const float ws = __shfl_sync(kFull, w, src, LPR);
        wv[u] = ok[u] ? ws : 0.f;   // a zero weight leaves a plain sum unchanged
    }
    Raw rv[V];
#pragma unroll
    for (int u = 0; u < V; ++u) ld(jv[u], ok[u], rv[u]);
#pragma unroll
    for (int u = 0; u < V; ++u)
#pragma unroll
        for (int h = 0; h < SPL; ++h) acc_add<KAHAN>(sum[h], comp[h], wv[u], val(rv[u], h), ok[u]);
}

// For this lane's group row (entries [p0, p0 + len)), sum[h] = sum over the
// entries whose column is marked in `bits` of w * x_h(j), in entry order, where
// ld(j, ok, raw) gathers column j's values for this lane's sets (predicated by
// ok) and val(raw, h) is set h's value.  (j0, w0) is the row's entry q, loaded
// by the caller; each later chunk of LPR entries is in flight while the one
// before it is used.  A chunk's marked entries go in batches of U gathers in
// flight, and the rest (fewer than U, counted by the group with the most) in
// batches of U/2, U/4, ..., 1: where few neighbours are marked, as early in an
// epidemic, a batch no larger than needed is most of the saving.  Called by all
// 32 lanes.
template <int LPR, int SPL, bool KAHAN, class Raw, class Ld, class Val>
__device__ __forceinline__ void group_row_sums(const Csr &m, uint32_t p0, uint32_t len, uint32_t j0, float w0,
                                               const uint32_t *__restrict__ bits, int lane, Ld ld, Val val,
                                               float (&sum)[SPL]) {
    constexpr int U = (SPL == 8) ? 4 : 8;
    const int grp = lane / LPR, q = lane % LPR;
    const unsigned gmask = (LPR == 32) ? kFull : ((1u << LPR) - 1u);
    float comp[SPL];
#pragma unroll
    for (int h = 0; h < SPL; ++h) sum[h] = comp[h] = 0.f;
    const uint32_t kmax = __reduce_max_sync(kFull, len);
    uint32_t jn = j0;
    float wn = w0;
    for (uint32_t k0 = 0; k0 < kmax; k0 += LPR) {
        const uint32_t kk = k0 + (uint32_t)q;
        const bool valid = kk < len;
        const uint32_t j = jn;
        const float w = wn;
        const bool vn = kk + LPR < len;
        jn = ld_cs_if(m.col + p0 + kk + LPR, vn);
        wn = ld_cs_if(m.w + p0 + kk + LPR, vn);
        const bool mk = valid && marked(bits, j);
        unsigned mm = (__ballot_sync(kFull, mk) >> (grp * LPR)) & gmask;
        const int nmax = (int)__reduce_max_sync(kFull, (unsigned)__popc(mm));
        int i0 = 0;
        for (; i0 + U <= nmax; i0 += U) gather_batch<U, LPR, SPL, KAHAN, Raw>(mm, j, w, ld, val, sum, comp);
        const int rest = nmax - i0;   // < U, warp-uniform
        if constexpr (U >= 8)
            if (rest & 4) gather_batch<4, LPR, SPL, KAHAN, Raw>(mm, j, w, ld, val, sum, comp);
        if (rest & 2) gather_batch<2, LPR, SPL, KAHAN, Raw>(mm, j, w, ld, val, sum, comp);
        if (rest & 1) gather_batch<1, LPR, SPL, KAHAN, Raw>(mm, j, w, ld, val, sum, comp);
    }
}

// Whether any lane of each group voted, packed as one bit per group.
template <int LPR>
__device__ __forceinline__ uint32_t group_bits(unsigned ballot) {
    constexpr int RPW = 32 / LPR;
    const unsigned gmask = (LPR == 32) ? kFull : ((1u << LPR) - 1u);
    uint32_t part = 0u;
#pragma unroll
    for (int gi = 0; gi < RPW; ++gi) part |= (((ballot >> (gi * LPR)) & gmask) != 0u ? 1u : 0u) << gi;
    return part;
}

// Sum a per-lane value over the groups of the warp (lanes with the same q hold the same sets).
template <int LPR>
__device__ __forceinline__ int group_reduce(int v) {
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <int SPL>
struct EWords {
    uint32_t w[SPL / 2];
};
template <int SPL>
struct FVec {
    float v[SPL];
};

template <class K>
int blocks_of(K kernel) {
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, kBlock, 0);
    return blocks > 0 ? blocks : 1;
}

// The (Bp, SPL) pairs built: SPL in {2, 4, 8} with Bp / SPL lanes per row (1..32).
#define GABM_BATCH_CONFIGS(X) \
    X(2, 2)                   \
    X(4, 2) X(4, 4)           \
    X(8, 2) X(8, 4) X(8, 8)   \
    X(16, 2) X(16, 4) X(16, 8) \
    X(32, 2) X(32, 4) X(32, 8) \
    X(64, 2) X(64, 4) X(64, 8)

}  // namespace

}  // namespace gabm
