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

#include <type_traits>

#include "gabm_internal.cuh"

namespace gabm {

#ifndef GABM_UNROLL
#define GABM_UNROLL 8
#endif
#ifndef GABM_PIPE
#define GABM_PIPE 1
#endif
#ifndef GABM_PREFETCH
#define GABM_PREFETCH 0
#endif
#ifndef GABM_MINBLOCKS
#define GABM_MINBLOCKS 3
#endif
constexpr int kUnroll = GABM_UNROLL;   // entries per lane loaded ahead of use

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// kahan_add when `take`, else no change (selects instead of a branch).
__device__ __forceinline__ void kahan_add_if(float &s, float &c, float x, bool take) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    const float cn = __fsub_rn(__fsub_rn(t, s), y);
    s = take ? t : s;
    c = take ? cn : c;
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

// Hands tiles to a warp in runs claimed with one atomic each from the launch's
// counter.  All warps hammering one counter with a tile per atomic serialises
// on that address, so runs hold up to 16 tiles and shrink as the counter nears
// the end (guided scheduling keeps the tail short); the next run is claimed
// one run ahead so the atomic's latency is hidden.
struct TileDispenser {
    int *ctr;
    int ntiles, nwarps, lane;
    int next, end;     // current run [next, end)
    int pend;          // lane 0: first tile of the claimed next run
    int pend_len;      // its length (warp-uniform)

    __device__ __forceinline__ int run_len(int from) const {
        const int rem = ntiles - from;
        return max(1, min(16, rem / (4 * nwarps)));
    }
    __device__ __forceinline__ void init(int *c, int nt, int nw, int ln) {
        ctr = c;
        ntiles = nt;
        nwarps = nw;
        lane = ln;
        next = end = 0;
        pend_len = run_len(0);
        pend = (lane == 0) ? atomicAdd(ctr, pend_len) : 0;
    }
    // the next tile of this warp, or a value >= ntiles when the launch's tiles are gone
    __device__ __forceinline__ int get() {
        if (next >= end) {
            const int base = __shfl_sync(0xffffffffu, pend, 0);
            if (base >= ntiles) return ntiles;
            next = base;
            end = base + pend_len;
            pend_len = run_len(end);
            if (lane == 0) pend = atomicAdd(ctr, pend_len);
        }
        return next < ntiles ? next++ : ntiles;
    }
};

// Hands each block one contiguous range of tiles, claimed tile by tile by its
// warps through a shared-memory counter.  Rows are laid out breadth-first, so
// the neighbours of a range's rows mostly lie in and around the same range:
// the warps of a block gather from lines their own SM has just cached, where a
// launch-wide counter would spread consecutive tiles over all SMs.  (Measured
// on the 1M-agent typed graph: 10% shorter day kernels than the launch-wide
// dispenser; handing the last eighth of the tiles out launch-wide to balance
// the tail costs more locality than it gains.  The batched kernels, whose rows
// carry up to 64 sets each, keep the launch-wide dispenser: there the ranges'
// imbalance cost 7%.)  Called by every thread of the block (init holds a barrier).
struct BlockTiles {
    int *ctr;          // the block's counter (shared memory)
    int end, ntiles, lane, pend;
    __device__ __forceinline__ void init(int nt, int ln) {
        __shared__ int s_ctr;
        ntiles = nt;
        lane = ln;
        const int b0 = (int)(((long long)blockIdx.x * nt) / gridDim.x);
        end = (int)(((long long)(blockIdx.x + 1) * nt) / gridDim.x);
        if (threadIdx.x == 0) s_ctr = b0;
        __syncthreads();
        ctr = &s_ctr;
        pend = (lane == 0) ? atomicAdd(ctr, 1) : 0;
    }
    // the next tile of this warp, or ntiles when the block's range is done
    __device__ __forceinline__ int get() {
        const int tile = __shfl_sync(0xffffffffu, pend, 0);
        if (tile >= end) return ntiles;
        if (lane == 0) pend = atomicAdd(ctr, 1);
        return tile;
    }
};

// Ask L2 to fetch one slice (entries [p0, p1) of both arrays) ahead of use.
// Slices start on 128-byte boundaries and hold multiples of 32 entries.
__device__ __forceinline__ void prefetch_slice(const Sell &m, uint32_t p0, uint32_t p1, int lane) {
    if (GABM_PREFETCH == 0) return;
    if (lane == 0 && p1 > p0) {
        const uint32_t bytes = (p1 - p0) * 4u;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(m.col + p0), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(m.w + p0), "r"(bytes) : "memory");
    }
}

// Warp sums of v by bin (bins 0..15; lanes with nothing to add pass v = 0): a
// reduce-scatter over the lanes, each step keeping half of a lane's bins and receiving
// the same half from the partner lane, 16 shuffles for all 16 bins (a butterfly per bin
// would take 80).  On return lanes 2b and 2b + 1 hold bin b's sum.  The addition tree is
// fixed, so the sums do not depend on anything but the inputs.  Called by all 32 lanes.
__device__ __forceinline__ float warp_bin_sums16(float v, int bin, int lane) {
    float x[16];
#pragma unroll
    for (int b = 0; b < 16; ++b) x[b] = (bin == b) ? v : 0.f;
#pragma unroll
    for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = hi ? x[i] : x[i + h];
            const float keep = hi ? x[i + h] : x[i];
            x[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, o));
        }
    }
    return __fadd_rn(x[0], __shfl_xor_sync(0xffffffffu, x[0], 1));
}

// Row data of one tile, loaded one tile ahead of use.
struct TileRows {
    int tile;
    int e;            // exposure day of this lane's row
    uint32_t len;     // entries of this lane's row
    uint32_t p0, p1;  // the tile's slice bounds
    int g;            // graph of the tile
    bool flag;        // the row has an infectious in-neighbour today (true without flags)
};

__device__ __forceinline__ void load_tile_rows(const Sell &m, const int16_t *e, const uint16_t *tile_graph,
                                               int ntiles, int tile, int lane, TileRows &tr,
                                               const uint8_t *flags = nullptr) {
    tr.tile = tile;
    tr.e = kPad;
    tr.len = 0;
    tr.p0 = tr.p1 = 0;
    tr.g = 0;
    tr.flag = true;
    if (tile < ntiles) {
        const int row = tile * kTile + lane;
        tr.e = e[row];
        tr.len = m.row_len[row];
        tr.p0 = m.slice_ptr[tile];
        tr.p1 = m.slice_ptr[tile + 1];
        tr.g = tile_graph ? (int)tile_graph[tile] : 0;
        if (flags) tr.flag = flags[row] != 0;
    }
}

// Sets flags[j] = 1 for every out-neighbour j of the tile rows whose lane has `push`
// (one byte store each: every writer stores the same value, so the result does not
// depend on their order).  The warp takes those rows one at a time, its lanes splitting
// the row's entries (entry k of tile row r sits at slice_ptr[tile] + 32 k + r), so a
// row costs a load round trip per 32 entries.  Called by all 32 lanes.
__device__ __forceinline__ void push_flags(const Sell &m_out, int tile, int lane, bool push, uint8_t *flags) {
    unsigned rows = __ballot_sync(0xffffffffu, push);
    if (!rows) return;
    const uint32_t base = m_out.slice_ptr[tile];
    const uint32_t my_len = push ? m_out.row_len[tile * kTile + lane] : 0u;
    while (rows) {
        const int r = __ffs(rows) - 1;
        rows &= rows - 1u;
        const uint32_t len = __shfl_sync(0xffffffffu, my_len, r);
        for (uint32_t k = (uint32_t)lane; k < len; k += 32u) flags[__ldg(m_out.col + base + 32u * k + (uint32_t)r)] = 1;
    }
}

// Loads that are skipped (value left at `dflt`) when pred is false, written as
// predicated PTX so that a batch of them issues without branches.
__device__ __forceinline__ uint32_t ld_cs_if(const uint32_t *p, bool pred) {
    uint32_t v = 0u;
    asm("{ .reg .pred q; setp.ne.u32 q, %2, 0; @q ld.global.cs.u32 %0, [%1]; }" : "+r"(v) : "l"(p), "r"((uint32_t)pred));
    return v;
}
__device__ __forceinline__ float ld_cs_if(const float *p, bool pred) {
    float v = 0.f;
    asm("{ .reg .pred q; setp.ne.u32 q, %2, 0; @q ld.global.cs.f32 %0, [%1]; }" : "+f"(v) : "l"(p), "r"((uint32_t)pred));
    return v;
}
__device__ __forceinline__ float ld_if(const float *p, bool pred) {
    float v = 0.f;
    asm("{ .reg .pred q; setp.ne.u32 q, %2, 0; @q ld.global.f32 %0, [%1]; }" : "+f"(v) : "l"(p), "r"((uint32_t)pred));
    return v;
}
__device__ __forceinline__ uint32_t ld_if(const uint32_t *p, bool pred) {
    uint32_t v = 0u;
    asm("{ .reg .pred q; setp.ne.u32 q, %2, 0; @q ld.global.u32 %0, [%1]; }" : "+r"(v) : "l"(p), "r"((uint32_t)pred));
    return v;
}
__device__ __forceinline__ float2 ld_if(const float2 *p, bool pred) {
    float2 v = make_float2(0.f, 0.f);
    asm("{ .reg .pred q; setp.ne.u32 q, %3, 0; @q ld.global.v2.f32 {%0, %1}, [%2]; }"
        : "+f"(v.x), "+f"(v.y) : "l"(p), "r"((uint32_t)pred));
    return v;
}
__device__ __forceinline__ int ld_if(const int16_t *p, bool pred, int dflt) {
    int v = dflt;
    asm("{ .reg .pred q; setp.ne.u32 q, %2, 0; @q ld.global.s16 %0, [%1]; }" : "+r"(v) : "l"(p), "r"((uint32_t)pred));
    return v;
}

// For this lane's row (when act), sum[a] = the sum of contribution a over the
// row's entries in entry order, with compensated summation; f(j, w, valid, out, take)
// writes the NARR contributions of the entry with column j and weight w and whether
// each is added (it is also called for invalid entries -- padding, other rows'
// tails -- and must then touch no memory beyond the slice and take nothing), and
// want[a] says whether sum a is taken for this row.  A sum of marked neighbours'
// infectiousness takes the marked entries only: the compensated sum of a row is then
// a function of its marked entries in entry order, however they are visited
// (row_sums here, or a warp walking one row).  Called by all 32 lanes; the batch runs
// without branches.
// No all-taken contribution: every batch goes through f.
struct NoFull {};

template <int NARR, class F, class FF = NoFull>
__device__ __forceinline__ void row_sums(const Sell &m, uint32_t p0, uint32_t len, bool act, int lane, F f,
                                         const bool (&want)[NARR], float (&sum)[NARR], FF ff = NoFull{}) {
    constexpr bool HAS_FULL = !std::is_same<FF, NoFull>::value;
    static_assert(!HAS_FULL || NARR == 1, "the all-taken path sums one contribution");
    float comp[NARR];
#pragma unroll
    for (int a = 0; a < NARR; ++a) { sum[a] = 0.f; comp[a] = 0.f; }
    const unsigned amask = __ballot_sync(0xffffffffu, act);
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, act ? len : 0u);
    // Mostly-active slices are read whole (padding and inactive rows included: every
    // entry below kmax lies inside the slice); sparse ones with predicated loads.
    const bool dense = __popc(amask) >= 24;
    // Batches wholly below every lane's row length (all lanes summing) have every entry
    // valid: with ff (the contribution of a valid entry when every valid entry is taken,
    // ff(j, w) = what f gives) they run without predicates or selects; the operations
    // and their order are those of the predicated path, so the sums are bitwise equal.
    uint32_t kfull = 0u;
    if constexpr (HAS_FULL) {
        const unsigned fmask = __ballot_sync(0xffffffffu, act && want[0]);
        kfull = __reduce_min_sync(0xffffffffu, (fmask == 0xffffffffu) ? len : 0u);
    }
    auto load_batch = [&](uint32_t k0, uint32_t (&jv)[kUnroll], float (&wv)[kUnroll]) {
        if (HAS_FULL && dense && k0 + (uint32_t)kUnroll <= kmax) {   // inside the slice: no predicates
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const uint32_t idx = p0 + (k0 + (uint32_t)u) * 32u + (uint32_t)lane;
                jv[u] = __ldcs(m.col + idx);
                wv[u] = __ldcs(m.w + idx);
            }
            return;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint32_t k = k0 + (uint32_t)u;
            const uint32_t idx = p0 + k * 32u + (uint32_t)lane;
            if (dense) {
                const bool in = k < kmax;
                jv[u] = ld_cs_if(m.col + idx, in);
                wv[u] = ld_cs_if(m.w + idx, in);
            } else {
                const bool v = act && k < len;
                jv[u] = ld_cs_if(m.col + idx, v);
                wv[u] = ld_cs_if(m.w + idx, v);
            }
        }
    };
    auto use_batch = [&](uint32_t k0, const uint32_t (&jv)[kUnroll], const float (&wv)[kUnroll]) {
        if constexpr (HAS_FULL) {
            if (k0 + (uint32_t)kUnroll <= kfull) {
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) kahan_add(sum[0], comp[0], ff(jv[u], wv[u]));
                return;
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint32_t k = k0 + (uint32_t)u;
            const bool valid = act && k < len;
            float out[NARR];
            bool take[NARR];
            f(jv[u], wv[u], valid, out, take);
#pragma unroll
            for (int a = 0; a < NARR; ++a) kahan_add_if(sum[a], comp[a], out[a], take[a] && want[a]);
        }
    };
    if (GABM_PIPE) {
        // the next batch is in flight while the current one is used
        uint32_t ja[kUnroll], jb[kUnroll];
        float wa[kUnroll], wb[kUnroll];
        if (kmax > 0) load_batch(0, ja, wa);
        for (uint32_t k0 = 0; k0 < kmax; k0 += 2 * kUnroll) {
            if (k0 + kUnroll < kmax) load_batch(k0 + kUnroll, jb, wb);
            use_batch(k0, ja, wa);
            if (k0 + kUnroll >= kmax) break;
            if (k0 + 2 * kUnroll < kmax) load_batch(k0 + 2 * kUnroll, ja, wa);
            use_batch(k0 + kUnroll, jb, wb);
        }
    } else {
        for (uint32_t k0 = 0; k0 < kmax; k0 += kUnroll) {
            uint32_t jv[kUnroll];
            float wv[kUnroll];
            load_batch(k0, jv, wv);
            use_batch(k0, jv, wv);
        }
    }
}

// Tiles with at most this many summing rows have them summed one row at a time by the
// whole warp (warp_row_sum) instead of lane by lane over the tile's longest row.
#ifndef GABM_COOP_ROWS
#define GABM_COOP_ROWS 4
#endif

// The sum of one row's taken contributions by the whole warp: the row of tile lane r
// (entries [0, len) at p0 + 32 k + r), the result in lane r's sum / comp.  The lanes
// load 32 entries at a time and evaluate f as row_sums does; lane r then adds the taken
// ones in entry order with the same compensated addition, so the value is row_sums'.
// Called by all 32 lanes.
template <class F>
__device__ __forceinline__ void warp_row_sum_from(const Sell &m, uint32_t p0, uint32_t len, uint32_t k_first, int r,
                                                  int lane, F f, float &sum, float &comp) {
    for (uint32_t k0 = k_first; k0 < len; k0 += 32u) {
        const uint32_t k = k0 + (uint32_t)lane;
        const bool valid = k < len;
        const uint32_t idx = p0 + k * 32u + (uint32_t)r;
        const uint32_t j = ld_cs_if(m.col + idx, valid);
        const float w = ld_cs_if(m.w + idx, valid);
        float out[1];
        bool take[1];
        f(j, w, valid, out, take);
        unsigned mm = __ballot_sync(0xffffffffu, take[0]);
        while (mm) {
            const int src = __ffs(mm) - 1;
            mm &= mm - 1u;
            const float v = __shfl_sync(0xffffffffu, out[0], src);
            if (lane == r) kahan_add(sum, comp, v);
        }
    }
}

template <class F>
__device__ __forceinline__ void warp_row_sum(const Sell &m, uint32_t p0, uint32_t len, int r, int lane, F f,
                                             float &sum, float &comp) {
    warp_row_sum_from(m, p0, len, 0u, r, lane, f, sum, comp);
}

// warp_row_sum for up to GABM_COOP_ROWS rows of a tile at once (the rows of `amask`), so
// that their loads overlap: the first 32 entries of every row are loaded, tested and
// gathered together, then each row's lane adds its taken contributions in entry order;
// entries past the first 32 go through warp_row_sum.  Each row's value is row_sums'.
// sum / comp: this lane's row (lanes without a row keep 0).  Called by all 32 lanes.
template <class F>
__device__ __forceinline__ void few_row_sums(const Sell &m, uint32_t p0, uint32_t my_len, unsigned amask, int lane,
                                             F f, float &sum, float &comp) {
    constexpr int K = GABM_COOP_ROWS;
    int r[K];
    uint32_t len[K], j[K];
    float w[K], out[K];
    bool take[K];
    unsigned mm = amask;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        r[i] = mm ? __ffs(mm) - 1 : -1;
        mm &= mm - 1u;
        len[i] = __shfl_sync(0xffffffffu, my_len, r[i] < 0 ? 0 : r[i]);
        if (r[i] < 0) len[i] = 0u;
        const bool valid = (uint32_t)lane < len[i];
        const uint32_t idx = p0 + (uint32_t)lane * 32u + (uint32_t)(r[i] < 0 ? 0 : r[i]);
        j[i] = ld_cs_if(m.col + idx, valid);
        w[i] = ld_cs_if(m.w + idx, valid);
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
        float o[1];
        bool tk[1];
        f(j[i], w[i], (uint32_t)lane < len[i], o, tk);
        out[i] = o[0];
        take[i] = tk[0];
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
        unsigned tm = __ballot_sync(0xffffffffu, take[i]);
        while (tm) {
            const int src = __ffs(tm) - 1;
            tm &= tm - 1u;
            const float v = __shfl_sync(0xffffffffu, out[i], src);
            if (lane == r[i]) kahan_add(sum, comp, v);
        }
    }
#pragma unroll
    for (int i = 0; i < K; ++i)
        if (__shfl_sync(0xffffffffu, len[i], 0) > 32u)   // len[i] is warp-uniform
            warp_row_sum_from(m, p0, len[i], 32u, r[i], lane, f, sum, comp);
}

}  // namespace gabm
