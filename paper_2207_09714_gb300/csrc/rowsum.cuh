// rowsum.cuh -- device helpers shared by the forward and backward day kernels.
//
// Edge storage is SELL-32 (sliced ELLPACK, one slice per 32-row warp tile):
// slice s holds max_len(s) x 32 entries, column-major, so entry k of the row in
// lane l of the slice sits at slice_ptr[s] + 32 k + l.  A warp reads entry k of
// its 32 rows with one coalesced 128-byte load per array, and every lane sums
// its own row in entry order.  The sum of a row therefore depends only on the
// row (the same operation sequence wherever and whenever it is computed), so a
// sum recomputed in the backward is bitwise the forward's.  Rows are laid out
// so that a slice holds rows of similar length (little padding).
#pragma once

#include "gabm_internal.cuh"

namespace gabm {

constexpr int kUnroll = 8;   // entries per lane loaded ahead of use

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

// Whether row j is marked in a per-day bitmap of infectious rows (read-only during the launch).
__device__ __forceinline__ bool marked(const uint32_t *__restrict__ bits, uint32_t j) {
    return (__ldg(bits + (j >> 5)) >> (j & 31u)) & 1u;
}

__device__ __forceinline__ int next_tile(int *ctr, int lane) {
    int v = 0;
    if (lane == 0) v = atomicAdd(ctr, 1);
    return __shfl_sync(0xffffffffu, v, 0);
}

// Ask L2 to fetch one slice (entries [p0, p1) of both arrays) ahead of use.
// Slices start on 128-byte boundaries and hold multiples of 32 entries.
__device__ __forceinline__ void prefetch_slice(const Sell &m, uint32_t p0, uint32_t p1, int lane) {
    if (lane == 0 && p1 > p0) {
        const uint32_t bytes = (p1 - p0) * 4u;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(m.col + p0), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(m.w + p0), "r"(bytes) : "memory");
    }
}

// Row data of one tile, loaded one tile ahead of use.
struct TileRows {
    int tile;
    int e;            // exposure day of this lane's row
    uint32_t len;     // entries of this lane's row
    uint32_t p0, p1;  // the tile's slice bounds
    int g;            // graph of the tile
};

__device__ __forceinline__ void load_tile_rows(const Sell &m, const int16_t *e, const uint16_t *tile_graph,
                                               int ntiles, int tile, int lane, TileRows &tr) {
    tr.tile = tile;
    tr.e = kPad;
    tr.len = 0;
    tr.p0 = tr.p1 = 0;
    tr.g = 0;
    if (tile < ntiles) {
        const int row = tile * kTile + lane;
        tr.e = e[row];
        tr.len = m.row_len[row];
        tr.p0 = m.slice_ptr[tile];
        tr.p1 = m.slice_ptr[tile + 1];
        tr.g = tile_graph ? (int)tile_graph[tile] : 0;
    }
}

// For this lane's row (when act), sum[a] = the sum of contribution a over the
// row's entries in entry order, with compensated summation; f(j, w, out) writes
// the NARR contributions of the entry with column j and weight w, and want[a]
// says whether sum a is taken for this row.  Called by all 32 lanes.
template <int NARR, class F>
__device__ __forceinline__ void row_sums(const Sell &m, uint32_t p0, uint32_t len, bool act, int lane, F f,
                                         const bool (&want)[NARR], float (&sum)[NARR]) {
    float comp[NARR];
#pragma unroll
    for (int a = 0; a < NARR; ++a) { sum[a] = 0.f; comp[a] = 0.f; }
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, act ? len : 0u);
    for (uint32_t k0 = 0; k0 < kmax; k0 += kUnroll) {
        uint32_t jv[kUnroll];
        float wv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint32_t k = k0 + (uint32_t)u;
            const bool v = act && k < len;
            const uint32_t idx = p0 + k * 32u + (uint32_t)lane;
            jv[u] = v ? __ldcs(m.col + idx) : 0u;
            wv[u] = v ? __ldcs(m.w + idx) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint32_t k = k0 + (uint32_t)u;
            if (act && k < len) {
                float out[NARR];
                f(jv[u], wv[u], out);
#pragma unroll
                for (int a = 0; a < NARR; ++a)
                    if (want[a]) kahan_add(sum[a], comp[a], out[a]);
            }
        }
    }
}

}  // namespace gabm
