// rowsum.cuh -- warp-cooperative row sums over a 32-row tile of a CSR matrix,
// shared by the forward and backward day kernels.
//
// The active rows of a warp tile are laid end to end as one stream of 16-byte
// edge vectors (4 columns / 4 weights each, aligned to the edge index, so a
// vector shared by two rows appears once per row with the other row's edges
// masked).  In chunks of kChunkVec vectors, every lane loads up to four vectors
// of that stream at once (coalesced, streaming loads), computes the per-edge
// contributions (which gather the neighbours' state), adds the four of a
// vector in order and stores that partial in shared memory.  Each lane then
// adds up its own row's vector partials in order with compensated (Kahan)
// summation.  The result depends only on the row's edges, not on which rows
// were active together, so a sum recomputed in the backward is bitwise the
// forward's, and long rows keep fp32 sums accurate to a few ulps.
#pragma once

#include "gabm_internal.cuh"

namespace gabm {

constexpr int kChunkVec = 128;   // edge vectors staged per warp and chunk
constexpr int kVecPerLane = kChunkVec / 32;

template <int NARR>
struct WarpStage {
    int pv[32];          // first stream vector of each active row (exclusive prefix)
    uint32_t vs[32];     // first 16-byte vector of each active row
    uint32_t rs[32];     // edge range of each active row
    uint32_t re[32];
    uint32_t fl[32];     // per-row flags handed to the contribution functor
    uint8_t rowid[kChunkVec];       // active-row index of each stream vector of the chunk
    float val[NARR][kChunkVec];     // per-vector partial sums of the chunk
};

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Infectiousness of a neighbour exposed on day e_j, seen on day t: c[t - e_j] for
// 1 <= t - e_j < L, else 0 (susceptible agents, padding rows, long-recovered agents).
__device__ __forceinline__ float infectiousness(int e_j, const float *c_s, int t, int L) {
    const int k = t - e_j;
    return ((unsigned)(k - 1) < (unsigned)(L - 1)) ? c_s[k] : 0.f;
}

__device__ __forceinline__ int next_tile(int *ctr, int lane) {
    int v = 0;
    if (lane == 0) v = atomicAdd(ctr, 1);
    return __shfl_sync(0xffffffffu, v, 0);
}

// For every lane with `act`, sum[a] = the sum over the row's edges p in [rs, re)
// of contribution a of edge p: the edges of each 16-byte vector are added in
// order into a vector partial, and the row's vector partials are added in order
// with compensated summation.  Both orders depend only on the row itself.
// contrib(flags, col, w, out) writes NARR values for one edge.  Called by all 32 lanes.
template <int NARR, class F>
__device__ __forceinline__ void warp_row_sums(WarpStage<NARR> &ws, const uint4 *__restrict__ col4,
                                              const float4 *__restrict__ w4, bool act, uint32_t rs,
                                              uint32_t re, uint32_t flags, int lane, F contrib,
                                              float (&sum)[NARR]) {
    float comp[NARR];
#pragma unroll
    for (int a = 0; a < NARR; ++a) { sum[a] = 0.f; comp[a] = 0.f; }
    const unsigned amask = __ballot_sync(0xffffffffu, act);
    if (amask == 0u) return;
    const uint32_t vs = rs >> 2;
    const int nv = (act && re > rs) ? (int)(((re + 3u) >> 2) - vs) : 0;
    int incl = nv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int pv = incl - nv;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int rank = __popc(amask & ((1u << lane) - 1u));
    if (act) {
        ws.pv[rank] = pv;
        ws.vs[rank] = vs;
        ws.rs[rank] = rs;
        ws.re[rank] = re;
        ws.fl[rank] = flags;
    }
    for (int c0 = 0; c0 < total; c0 += kChunkVec) {
        const int cn = min(kChunkVec, total - c0);
        const int f_lo = max(pv, c0), f_hi = min(pv + nv, c0 + cn);
        for (int f = f_lo; f < f_hi; ++f) ws.rowid[f - c0] = (uint8_t)rank;
        __syncwarp();
        uint4 cc[kVecPerLane];
        float4 ww[kVecPerLane];
        int jr[kVecPerLane];
        uint32_t vv[kVecPerLane];
#pragma unroll
        for (int u = 0; u < kVecPerLane; ++u) {
            const int k = lane + 32 * u;
            jr[u] = -1;
            if (k < cn) {
                const int j = ws.rowid[k];
                jr[u] = j;
                vv[u] = ws.vs[j] + (uint32_t)(c0 + k - ws.pv[j]);
                cc[u] = __ldcs(col4 + vv[u]);
                ww[u] = __ldcs(w4 + vv[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < kVecPerLane; ++u) {
            if (jr[u] >= 0) {
                const int k = lane + 32 * u;
                const uint32_t rsj = ws.rs[jr[u]], rej = ws.re[jr[u]], flj = ws.fl[jr[u]];
                const uint32_t p0 = vv[u] << 2;
                const uint32_t cq[4] = {cc[u].x, cc[u].y, cc[u].z, cc[u].w};
                const float wq[4] = {ww[u].x, ww[u].y, ww[u].z, ww[u].w};
                float part[NARR];
#pragma unroll
                for (int a = 0; a < NARR; ++a) part[a] = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t p = p0 + (uint32_t)q;
                    if (p >= rsj && p < rej) {
                        float out[NARR];
#pragma unroll
                        for (int a = 0; a < NARR; ++a) out[a] = 0.f;
                        contrib(flj, cq[q], wq[q], out);
#pragma unroll
                        for (int a = 0; a < NARR; ++a) part[a] = __fadd_rn(part[a], out[a]);
                    }
                }
#pragma unroll
                for (int a = 0; a < NARR; ++a) ws.val[a][k] = part[a];
            }
        }
        __syncwarp();
        for (int f = f_lo; f < f_hi; ++f) {
#pragma unroll
            for (int a = 0; a < NARR; ++a) kahan_add(sum[a], comp[a], ws.val[a][f - c0]);
        }
        __syncwarp();
    }
}

}  // namespace gabm
