// rowsum.cuh -- per-lane partial sums over one CSR row, shared by the forward
// and backward day kernels so that a recomputed neighbour sum is bitwise the
// one the forward used (same vectors, same order, same fused multiply-adds).
#pragma once

#include "gabm_internal.cuh"

namespace gabm {

// Infectiousness of neighbour j on day t: c[t - e_j] for 1 <= t - e_j < L, else 0
// (susceptible and padding agents have t - e_j outside that range).
__device__ __forceinline__ float neighbour_infectiousness(const int16_t *e, uint32_t j, const float *c_s,
                                                          int t, int L) {
    const int k = t - (int)e[j];
    return ((unsigned)(k - 1) < (unsigned)(L - 1)) ? c_s[k] : 0.f;
}

// Lane gl of a GL-lane group sums w_ji * c[t - e_j] over the 4-edge vectors
// v = rs/4 + gl, rs/4 + gl + GL, ... of the row [rs, re).  Vector loads are
// 16-byte aligned; entries outside the row are masked.  Streaming loads
// (evict-first) keep the edge stream from displacing the gathered state in L2.
template <int GL>
__device__ __forceinline__ float lane_infectious_sum(const uint4 *__restrict__ col4,
                                                     const float4 *__restrict__ w4, const int16_t *e,
                                                     const float *c_s, uint32_t rs, uint32_t re, int gl,
                                                     int t, int L) {
    float part = 0.f;
    const uint32_t v1 = (re + 3u) >> 2;
    for (uint32_t v = (rs >> 2) + (uint32_t)gl; v < v1; v += GL) {
        const uint4 cc = __ldcs(col4 + v);
        const float4 ww = __ldcs(w4 + v);
        const uint32_t i0 = v << 2;
        if (i0 + 0u >= rs && i0 + 0u < re) part = __fmaf_rn(ww.x, neighbour_infectiousness(e, cc.x, c_s, t, L), part);
        if (i0 + 1u >= rs && i0 + 1u < re) part = __fmaf_rn(ww.y, neighbour_infectiousness(e, cc.y, c_s, t, L), part);
        if (i0 + 2u >= rs && i0 + 2u < re) part = __fmaf_rn(ww.z, neighbour_infectiousness(e, cc.z, c_s, t, L), part);
        if (i0 + 3u >= rs && i0 + 3u < re) part = __fmaf_rn(ww.w, neighbour_infectiousness(e, cc.w, c_s, t, L), part);
    }
    return part;
}

// Backward variant over the same vectors: the transpose gather sum w * r_next[j]
// (when want_gx) and, in the same pass, the recomputed infectiousness sum (when
// WITH_LAM and want_lam) with exactly the forward's operation sequence.
template <int GL, bool WITH_LAM>
__device__ __forceinline__ void lane_adjoint_sums(const uint4 *__restrict__ col4, const float4 *__restrict__ w4,
                                                  const int16_t *E, const float *r_next, const float *c_s,
                                                  uint32_t rs, uint32_t re, int gl, int t, int L,
                                                  bool want_gx, bool want_lam, float &gx, float &lam) {
    const uint32_t v1 = (re + 3u) >> 2;
    for (uint32_t v = (rs >> 2) + (uint32_t)gl; v < v1; v += GL) {
        const uint4 cc = __ldcs(col4 + v);
        const float4 ww = __ldcs(w4 + v);
        const uint32_t i0 = v << 2;
        const uint32_t jj[4] = {cc.x, cc.y, cc.z, cc.w};
        const float wv[4] = {ww.x, ww.y, ww.z, ww.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t idx = i0 + (uint32_t)q;
            if (idx >= rs && idx < re) {
                if (want_gx) gx = __fmaf_rn(wv[q], r_next[jj[q]], gx);
                if (WITH_LAM && want_lam) lam = __fmaf_rn(wv[q], neighbour_infectiousness(E, jj[q], c_s, t, L), lam);
            }
        }
    }
}

}  // namespace gabm
