// batched.cu -- day kernels for B parameter sets sharing each contact graph.
//
// The model step is the one of forward.cu / backward.cu (Sec. 3.1, Eq. 1-3;
// adjoint of App. B) applied to B independent instances that differ only in
// their parameters (R_t, m_t, S_a) and Philox stream.  The graph is read once
// per row for all sets: exposure days, adjoints and coefficients are stored
// agent-major, [n_rows][Bp], so a neighbour's values for every set are one
// contiguous gather (Bp * 2 bytes of e, Bp * 4 bytes of r).
//
// A warp works on a 32-row tile.  A "group" of LPR = Bp/SPL lanes shares one
// row, lane q of the group owning the SPL sets [q SPL, (q+1) SPL); 32/LPR rows
// are in flight per warp and the tile takes LPR passes.  For each chunk of LPR
// entries of the row, the group loads the columns and weights coalesced, tests
// each neighbour against the day's bitmap (rows infectious in some set, or
// susceptible in some set in the backward), compacts the marked entries with a
// ballot and broadcasts them one by one; every lane gathers its SPL sets'
// values with one vector load and accumulates them in entry order.  Unmarked
// entries contribute nothing in any set, so skipping them changes no sum.
//
// Summation: compensated (as in the single-set kernels) when some row has more
// than kPlainSumMaxDegree entries, else fused multiply-add in entry order,
// whose relative error is below (entries + 3) * 2^-24 < 1e-5 for a sum of
// non-negative terms.
//
// Counting (Aggregate, Sec. 3.1): the forward writes, per tile and set, how
// many agents were exposed that day (tile_new, one byte each); the stage
// counts and newRM of every day follow from those and the exposure-day
// histogram of the starting state (k_counts_b), with no atomics in the day
// kernel.
#include <algorithm>

#include "gabm_internal.cuh"
#include "rowsum.cuh"

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

// For this lane's group row (entries [p0, p0 + len)), sum[h] = sum over the
// entries whose column is marked in `bits` of w * x_h(j), in entry order, where
// ld(j, ok, raw) gathers column j's values for this lane's sets (predicated by
// ok) and val(raw, h) is set h's value.  (j0, w0) is the row's entry q, loaded
// by the caller; each later chunk of LPR entries is in flight while the one
// before it is used.  Called by all 32 lanes.
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
        for (int i0 = 0; i0 < nmax; i0 += U) {
            uint32_t jv[U];
            float wv[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                ok[u] = mm != 0u;
                const int src = ok[u] ? __ffs(mm) - 1 : 0;
                mm &= mm - 1u;
                jv[u] = __shfl_sync(kFull, j, src, LPR);
                const float ws = __shfl_sync(kFull, w, src, LPR);
                wv[u] = ok[u] ? ws : 0.f;   // a zero weight leaves a plain sum unchanged
            }
            Raw rv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) ld(jv[u], ok[u], rv[u]);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int h = 0; h < SPL; ++h) acc_add<KAHAN>(sum[h], comp[h], wv[u], val(rv[u], h), ok[u]);
        }
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

// ---------------------------------------------------------------------------
// Forward day t for every set (Transmit, draw, Progress).
// ---------------------------------------------------------------------------
template <int LPR, int SPL, bool KAHAN>
__global__ void __launch_bounds__(kBlock, 2) k_fwd_day_b(const FwdBatchArgs a) {
    constexpr int RPW = 32 / LPR;
    constexpr int Bp = LPR * SPL;
    constexpr int NW = kBlock / 32;
    __shared__ float c_s[kMaxL + 1];
    if (threadIdx.x <= kMaxL) c_s[threadIdx.x] = threadIdx.x < kMaxL ? a.c[threadIdx.x] : 0.f;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int grp = lane / LPR, q = lane % LPR;
    const int t = a.t, L = a.L, B = a.B, ntiles = a.ntiles;
    uint32_t *e32 = reinterpret_cast<uint32_t *>(a.e);
    const uint32_t *e32r = e32;
    constexpr int WPR = Bp / 2;   // 32-bit words per row of e

    auto ld = [&](uint32_t j, bool ok, EWords<SPL> &r) { ld_words<SPL>(e32r + (size_t)j * WPR + q * (SPL / 2), ok, r.w); };
    auto val = [&](const EWords<SPL> &r, int h) { return infect_lut(half_of(r.w[h >> 1], h & 1), c_s, t, (unsigned)L); };

    int cur_g = -1;
    float Rt[SPL];
#pragma unroll
    for (int h = 0; h < SPL; ++h) Rt[h] = 0.f;
    TileDispenser disp;
    disp.init(a.tile_ctr, ntiles, gridDim.x * NW, lane);
    // row bounds of the tile's 32 rows (lane r: rows r and r + 1), one tile ahead
    int tile = disp.get();
    uint32_t rp_lo = 0u, rp_hi = 0u;
    if (tile < ntiles) {
        rp_lo = a.m.rowptr[tile * kTile + lane];
        rp_hi = a.m.rowptr[tile * kTile + lane + 1];
    }
    while (tile < ntiles) {
        const int ntile = disp.get();
        uint32_t nrp_lo = 0u, nrp_hi = 0u;
        if (ntile < ntiles) {
            nrp_lo = a.m.rowptr[ntile * kTile + lane];
            nrp_hi = a.m.rowptr[ntile * kTile + lane + 1];
        }
        const int g = a.gr.tile_graph ? (int)a.gr.tile_graph[tile] : 0;
        if (g != cur_g) {
            cur_g = g;
#pragma unroll
            for (int h = 0; h < SPL; ++h) {
                const int s = q * SPL + h;
                Rt[h] = (s < B) ? a.R[(size_t)(g * B + s) * a.ldP + t] : 0.f;
            }
        }
        const float inv_D = a.gr.inv_Dbar[g];
        uint32_t word = 0u;
        int nnew[SPL];
#pragma unroll
        for (int h = 0; h < SPL; ++h) nnew[h] = 0;
        PassRow<SPL> nx;
        load_pass_row<SPL>(a.m, e32 + (size_t)(tile * kTile + grp) * WPR + q * (SPL / 2), rp_lo, rp_hi, grp, q, nx);
        for (int pass = 0; pass < LPR; ++pass) {
            const int row = tile * kTile + pass * RPW + grp;
            uint32_t *mine_p = e32 + (size_t)row * WPR + q * (SPL / 2);
            const PassRow<SPL> cu = nx;
            if (pass + 1 < LPR)   // the next pass's row in flight while this one is summed
                load_pass_row<SPL>(a.m, mine_p + (size_t)RPW * WPR, rp_lo, rp_hi, (pass + 1) * RPW + grp, q, nx);
            uint32_t ew[SPL / 2];
#pragma unroll
            for (int k = 0; k < SPL / 2; ++k) ew[k] = cu.ew[k];
            bool sS[SPL];
            bool mine = false;
#pragma unroll
            for (int h = 0; h < SPL; ++h) {
                sS[h] = half_of(ew[h >> 1], h & 1) == kNever;
                mine |= sS[h];
            }
            const bool act = (group_bits<LPR>(__ballot_sync(kFull, mine)) >> grp) & 1u;
            float sum[SPL];
            group_row_sums<LPR, SPL, KAHAN, EWords<SPL>>(a.m, cu.p0, act ? cu.len : 0u, cu.j0, cu.w0, a.bits_cur, lane,
                                                         ld, val, sum);

            bool inf = false;
            if (mine) {
                const int ai = a.age[row];
                const uint32_t id = caller_id(a.gr, row, g);
                float Lam[SPL];
                uint32_t nw[SPL / 2];
#pragma unroll
                for (int k = 0; k < SPL / 2; ++k) nw[k] = ew[k];
                bool changed = false;
#pragma unroll
                for (int h = 0; h < SPL; ++h) {
                    Lam[h] = 0.f;
                    if (!sS[h] || sum[h] == 0.f) continue;   // lambda = 0: p = 0, no draw
                    const int inst = g * B + q * SPL + h;
                    Lam[h] = sum[h] * inv_D;
                    const float lam = (Rt[h] * a.S[inst * kAges + ai]) * Lam[h];
                    const float p = -expm1f(-lam);
                    if (p > kUmin) {
                        const float u = uniform_from_word(philox_word(a.seed, id, (uint32_t)t, (uint32_t)inst, 0u));
                        if (u < p) {
                            const uint32_t tv = (uint32_t)(uint16_t)(int16_t)t;
                            nw[h >> 1] = (h & 1) ? ((nw[h >> 1] & 0xffffu) | (tv << 16)) : ((nw[h >> 1] & 0xffff0000u) | tv);
                            ++nnew[h];
                            changed = true;
                        }
                    }
                }
                if (changed) st_words<SPL>(mine_p, nw);
                if (a.lam_out) st_floats<SPL>(a.lam_out + (size_t)row * Bp + q * SPL, Lam);
#pragma unroll
                for (int k = 0; k < SPL / 2; ++k) ew[k] = nw[k];
            }
#pragma unroll
            for (int h = 0; h < SPL; ++h) {
                const int kn = t + 1 - half_of(ew[h >> 1], h & 1);
                inf |= (unsigned)(kn - 1) < (unsigned)(L - 1);
            }
            word |= group_bits<LPR>(__ballot_sync(kFull, inf)) << (pass * RPW);
        }
        if (lane == 0) a.bits_next[tile] = word;
        // exposures of this tile by set (at most 32 each)
#pragma unroll
        for (int h = 0; h < SPL; ++h) nnew[h] = group_reduce<LPR>(nnew[h]);
        if (grp == 0) {
            uint8_t *dst = a.tile_new + (size_t)tile * Bp + q * SPL;
#pragma unroll
            for (int h = 0; h < SPL; ++h) dst[h] = (uint8_t)nnew[h];
        }
        tile = ntile;
        rp_lo = nrp_lo;
        rp_hi = nrp_hi;
    }
}

// ---------------------------------------------------------------------------
// Reverse day t for every set: the transpose gather of day t+1 and the
// straight-through adjoint of day t's draws (the per-set steps of backward.cu).
// ---------------------------------------------------------------------------
// DC: also accumulate the adjoint of the infectiousness table (a.dc_tile), a separate
// instance so that the plain sweep carries none of its code.
template <int LPR, int SPL, bool KAHAN, bool DC>
__global__ void __launch_bounds__(kBlock, 2) k_bwd_day_b(const BwdBatchArgs a) {
    constexpr int RPW = 32 / LPR;
    constexpr int Bc = LPR * SPL;        // sets of this launch (a chunk of the row's Bw)
    constexpr int NW = kBlock / 32;
    // DC: per-warp tile sums [L][Bc] of gx at the rows' infectious days, by k = t + 1 - E
    extern __shared__ float dcs_all[];
    __shared__ float c_s[kMaxL];
    __shared__ int slot_k[kMaxL];
    __shared__ float pacc[NW][kAges][Bc];   // per-warp tile sums of gl * Lam by age and set
    __shared__ float fac_s[NW][kMaxL];       // 2^(sigma(t+k) - sigma(t)) of the warp's graph
    if (threadIdx.x < kMaxL) {
        c_s[threadIdx.x] = a.c[threadIdx.x];
        slot_k[threadIdx.x] = a.ring_slot[threadIdx.x];
    }
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int i = lane; i < kAges * Bc; i += 32) (&pacc[wib][0][0])[i] = 0.f;
    float *dcs = dcs_all + (size_t)wib * a.L * Bc;
    if constexpr (DC)
        for (int i = lane; i < a.L * Bc; i += 32) dcs[i] = 0.f;
    __syncthreads();

    const int grp = lane / LPR, q = lane % LPR;
    const int t = a.t, T = a.T, L = a.L, B = a.B, ntiles = a.ntiles;
    const bool has_next = t + 1 < T;
    const uint32_t *E32 = reinterpret_cast<const uint32_t *>(a.E);
    const int Bw = a.Bw;                 // row width of the per-agent arrays
    const int s0 = a.s0 + q * SPL;       // this lane's first set
    const size_t stride = a.ring_stride;

    auto ld = [&](uint32_t j, bool ok, FVec<SPL> &r) { ld_floats<SPL>(a.r_next + (size_t)j * Bw + s0, ok, r.v); };
    auto val = [](const FVec<SPL> &r, int h) { return r.v[h]; };

    int cur_g = -1;
    float Rt[SPL], Gtail[SPL];
#pragma unroll
    for (int h = 0; h < SPL; ++h) Rt[h] = Gtail[h] = 0.f;
    const int32_t *sg = nullptr;   // scale exponents of the current graph (shared by its sets)
    int sig_t = 0;
    unsigned emax_w = 0u;          // largest exponent stored by this warp (+128)
    uint32_t touched = 0u;         // DC: the k rows of dcs this lane added to in the current tile
    TileDispenser disp;
    disp.init(a.tile_ctr, ntiles, gridDim.x * NW, lane);
    // row bounds of the tile's 32 rows (lane r: rows r and r + 1), one tile ahead
    int tile = disp.get();
    uint32_t rp_lo = 0u, rp_hi = 0u;
    if (tile < ntiles) {
        rp_lo = a.m.rowptr[tile * kTile + lane];
        rp_hi = a.m.rowptr[tile * kTile + lane + 1];
    }
    while (tile < ntiles) {
        const int ntile = disp.get();
        uint32_t nrp_lo = 0u, nrp_hi = 0u;
        if (ntile < ntiles) {
            nrp_lo = a.m.rowptr[ntile * kTile + lane];
            nrp_hi = a.m.rowptr[ntile * kTile + lane + 1];
        }
        const int g = a.gr.tile_graph ? (int)a.gr.tile_graph[tile] : 0;
        if (g != cur_g) {
            if (cur_g >= 0) {
                flush_emax(a.emax + (size_t)cur_g * a.ld_sig + t, emax_w);
                emax_w = 0u;
            }
            cur_g = g;
            sg = a.sig + (size_t)g * a.ld_sig;
            sig_t = next_sigma(sg[t + 1], a.emax[(size_t)g * a.ld_sig + t + 1]);
            if (lane == 0 && tile * kTile == a.gr.row0[g]) a.sig[(size_t)g * a.ld_sig + t] = sig_t;  // one writer
            if (lane < kMaxL)
                fac_s[wib][lane] = (lane >= 1 && lane < L && t + lane <= T) ? exp2i(sg[t + lane] - sig_t) : 0.f;
            __syncwarp();
#pragma unroll
            for (int h = 0; h < SPL; ++h) {
                const int s = s0 + h;
                const size_t pi = (size_t)(g * B + s) * a.ldP;
                Rt[h] = (s < B) ? a.R[pi + t] : 0.f;
                Gtail[h] = (s < B && t + L < T) ? a.m_t[pi + t + L] * (float)a.gD[pi + t + L] * exp2i(-sig_t) : 0.f;
            }
        }
        const float inv_D = a.gr.inv_Dbar[g];
        uint32_t word = 0u;
        PassRow<SPL> nx;
        load_pass_row<SPL>(a.m, E32 + ((size_t)(tile * kTile + grp) * Bw + s0) / 2, rp_lo, rp_hi, grp, q, nx);
        for (int pass = 0; pass < LPR; ++pass) {
            const int row = tile * kTile + pass * RPW + grp;
            const size_t xo = (size_t)row * Bw + s0;   // this lane's first slot
            const PassRow<SPL> cu = nx;
            if (pass + 1 < LPR)   // the next pass's row in flight while this one is summed
                load_pass_row<SPL>(a.m, E32 + (xo + (size_t)RPW * Bw) / 2, rp_lo, rp_hi, (pass + 1) * RPW + grp, q, nx);
            uint32_t ew[SPL / 2];
#pragma unroll
            for (int k = 0; k < SPL / 2; ++k) ew[k] = cu.ew[k];
            bool isS[SPL];
            bool needA_any = false, anyS = false;
#pragma unroll
            for (int h = 0; h < SPL; ++h) {
                const int Eh = half_of(ew[h >> 1], h & 1);
                const bool never = Eh == kNever;
                const bool live = (Eh != kPad) && (never || Eh >= 0);   // seeds are constants
                isS[h] = live && (never || Eh >= t);
                needA_any |= has_next && live && (never || Eh >= t + 2 - L);
                anyS |= isS[h];
            }
            // table adjoint: sets in which the row is infectious on day t+1 (k = t+1-E in
            // [1, L-1]) add gx(t+1) to dc[k]; seeds are gathered for this alone
            bool dch[SPL];
            int kdh[SPL];
            bool dc_any = false;
#pragma unroll
            for (int h = 0; h < SPL; ++h) {
                const int Eh = half_of(ew[h >> 1], h & 1);
                kdh[h] = t + 1 - Eh;
                dch[h] = DC && has_next && Eh != kPad && Eh != kNever && kdh[h] >= 1 && kdh[h] <= L - 1;
                dc_any |= dch[h];
            }
            const bool act = (group_bits<LPR>(__ballot_sync(kFull, needA_any || dc_any)) >> grp) & 1u;
            float gx[SPL];
            group_row_sums<LPR, SPL, KAHAN, FVec<SPL>>(a.m, cu.p0, act ? cu.len : 0u, cu.j0, cu.w0, a.rbits_next, lane,
                                                       ld, val, gx);
            if (needA_any) st_floats<SPL>(a.ring + (size_t)slot_k[1] * stride + xo, gx);
            if constexpr (DC) {
                // the groups add their rows in a fixed order
#pragma unroll
                for (int gi = 0; gi < RPW; ++gi) {
                    if (grp == gi)
#pragma unroll
                        for (int h = 0; h < SPL; ++h)
                            if (dch[h]) {
                                dcs[kdh[h] * Bc + q * SPL + h] += gx[h];
                                touched |= 1u << kdh[h];
                            }
                    __syncwarp();
                }
            }

            float v[SPL];
            int ai = 0;
#pragma unroll
            for (int h = 0; h < SPL; ++h) v[h] = 0.f;
            if (anyS) {
                ai = a.age[row];
                const uint32_t id = caller_id(a.gr, row, g);
                // loads that do not depend on G first, then the ring in batches of 4 slots
                bool readA = false, writeA = false;
#pragma unroll
                for (int h = 0; h < SPL; ++h) {
                    const int Eh = half_of(ew[h >> 1], h & 1);
                    readA |= isS[h] && Eh != kNever && Eh != t;
                    writeA |= isS[h] && Eh == t;
                }
                float Av[SPL];
                ld_floats<SPL>(a.A + xo, readA || writeA, Av);
                float Lv[SPL];
                ld_floats<SPL>(a.lam_t + xo, true, Lv);
                float G[SPL];
#pragma unroll
                for (int h = 0; h < SPL; ++h)
                    G[h] = has_next ? __fmaf_rn(c_s[1], gx[h] * fac_s[wib][1], Gtail[h]) : Gtail[h];
                for (int k0 = 2; k0 < L; k0 += 4) {
                    float rv[4][SPL];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = k0 + u;
                        const bool ok = k < L && t + k < T;
                        ld_floats<SPL>(a.ring + (size_t)slot_k[ok ? k : 0] * stride + xo, ok, rv[u]);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = k0 + u;
                        if (k < L && t + k < T)
#pragma unroll
                            for (int h = 0; h < SPL; ++h) G[h] = __fmaf_rn(c_s[k], rv[u][h] * fac_s[wib][k], G[h]);
                    }
                }
                float rc[SPL];
                float stored = 0.f;
#pragma unroll
                for (int h = 0; h < SPL; ++h) {
                    rc[h] = 0.f;
                    if (!isS[h]) continue;
                    const int Eh = half_of(ew[h >> 1], h & 1);
                    float dy;
                    if (Eh == t) { Av[h] = G[h]; dy = G[h]; }
                    else if (Eh == kNever) dy = G[h];
                    else dy = G[h] - Av[h] * exp2i(sg[Eh] - sig_t);   // A was stored on day Eh
                    stored = fmaxf(stored, fabsf(G[h]));
                    const int inst = g * B + s0 + h;
                    const float RS = Rt[h] * a.S[inst * kAges + ai];
                    const float lam = RS * Lv[h];
                    const float qv = expf(-lam);
                    const float p = -expm1f(-lam);
                    const float u = uniform_from_word(philox_word(a.seed, id, (uint32_t)t, (uint32_t)inst, 0u));
                    const float den = __fmaf_rn(p, 1.f - u, qv * u);
                    const float dydl = (u * (1.f - u)) * qv / (den * den);
                    const float glam = dy * dydl;
                    rc[h] = RS * glam * inv_D;
                    v[h] = glam * Lv[h];
                    stored = fmaxf(stored, fabsf(rc[h]));
                }
                emax_w = max(emax_w, (unsigned)(float_exponent(stored) + 128));
                if (writeA) st_floats<SPL>(a.A + xo, Av);
                st_floats<SPL>(a.r_cur + xo, rc);
            }
            // tile sums by age: the groups add their rows in a fixed order
#pragma unroll
            for (int gi = 0; gi < RPW; ++gi) {
                if (grp == gi && anyS)
#pragma unroll
                    for (int h = 0; h < SPL; ++h) pacc[wib][ai][q * SPL + h] += v[h];
                __syncwarp();
            }
            word |= group_bits<LPR>(__ballot_sync(kFull, anyS)) << (pass * RPW);
        }
        // per-tile sums by age and set: fp32 over the tile's 32 rows, FP64 from here on
        double *Pt = a.P_t + (size_t)tile * kAges * Bw + a.s0;
        for (int i = lane; i < kAges * Bc; i += 32) {
            float *cell = &pacc[wib][0][0] + i;
            Pt[(i / Bc) * Bw + (i % Bc)] = (double)*cell;
            *cell = 0.f;
        }
        __syncwarp();
        if (lane == 0) a.rbits_cur[tile] = word;
        if constexpr (DC) {
            // the tile's sums of the table adjoint, at the scale of day t+1, into FP64 (the
            // warp holding the tile is the only writer of its accumulators on this day)
            uint32_t tm = __reduce_or_sync(kFull, touched);
            touched = 0u;
            if (tm) {
                const double scale = ldexp(1.0, sg[t + 1]);
                double *dt = a.dc_tile + (size_t)tile * L * Bw + a.s0;
                while (tm) {
                    const int k = __ffs(tm) - 1;
                    tm &= tm - 1u;
                    for (int i = lane; i < Bc; i += 32) {
                        const float v = dcs[k * Bc + i];
                        if (v != 0.f) {
                            dt[(size_t)k * Bw + i] += (double)v * scale;
                            dcs[k * Bc + i] = 0.f;
                        }
                    }
                }
                __syncwarp();
            }
        }
        tile = ntile;
        rp_lo = nrp_lo;
        rp_hi = nrp_hi;
    }
    if (cur_g >= 0) flush_emax(a.emax + (size_t)cur_g * a.ld_sig + t, emax_w);
}

// One warp per tile: rows infectious on day t0 (1 <= t0 - e < L) in any set.
__global__ void k_infectious_bits_b(const int16_t *e, int Bp, int t0, int L, int ntiles, uint32_t *bits) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < ntiles; tile += warps) {
        const int16_t *er = e + (size_t)(tile * kTile + lane) * Bp;
        bool inf = false;
        for (int b = 0; b < Bp; ++b) {
            const int k = t0 - er[b];
            inf |= (unsigned)(k - 1) < (unsigned)(L - 1);
        }
        const unsigned w = __ballot_sync(kFull, inf);
        if (lane == 0) bits[tile] = w;
    }
}

// Exposure-day histogram of the starting state of day t0, per instance (bin 0,
// the susceptible agents, is left to k_counts_b: it is the graph's agents minus
// the others): bin 1 = exposed on or before day t0 - L - 1, bin 2 + d - (t0 - L)
// = exposed on day d for t0 - L <= d < t0.
__global__ void k_exposure_hist_b(const int16_t *e, GraphRef gr, int64_t n_rows, int B, int Bp, int t0, int L,
                                  int32_t *H) {
    const int nb = L + 2;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_rows * Bp;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / Bp;
        const int s = (int)(idx - r * Bp);
        const int v = e[idx];
        if (s >= B || v == kPad || v == kNever) continue;
        const int g = gr.tile_graph ? (int)gr.tile_graph[r / kTile] : 0;
        const int bin = (v < t0 - L) ? 1 : 2 + v - (t0 - L);
        if (bin < nb) atomicAdd(H + (size_t)(g * B + s) * nb + bin, 1);
    }
}

// New exposures per instance and day: sum of the per-tile bytes over the tiles of
// a chunk, added to newinf[inst][t] (integer sums: the order does not matter).
__global__ void k_newinf_b(const uint8_t *tile_new, int ntiles, const int32_t *tile0, const int32_t *ntl, int B,
                           int Bp, int t0, int ldP, int32_t *newinf) {
    const int c = blockIdx.x, d = blockIdx.y, g = blockIdx.z;
    const int t = t0 + d;
    const int nt = ntl[g];
    const int i0 = c * kReduceChunkTiles * 4, i1 = min(nt, i0 + kReduceChunkTiles * 4);
    if (i0 >= nt) return;
    const uint8_t *base = tile_new + ((size_t)t * ntiles + tile0[g]) * Bp;
    for (int s = threadIdx.x; s < B; s += blockDim.x) {
        int acc = 0;
        for (int i = i0; i < i1; ++i) acc += base[(size_t)i * Bp + s];
        if (acc) atomicAdd(newinf + (size_t)(g * B + s) * ldP + t, acc);
    }
}

// Stage counts and newRM of days t0..T-1 from the starting histogram and the
// daily exposures (one thread per instance).
__global__ void k_counts_b(const int32_t *H, const int32_t *newinf, const int32_t *rows, int B, int I, int ldP,
                           int t0, int T, int tau_EI, int L, int32_t *counts, int32_t *newRM) {
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= I) return;
    const int nb = L + 2;
    const int32_t *h = H + (size_t)inst * nb;
    const int32_t *ni = newinf + (size_t)inst * ldP;
    // exposures on day d (d >= t0 - L)
    auto cnt = [&](int d) -> int32_t { return d >= t0 ? ni[d] : h[2 + d - (t0 - L)]; };
    int32_t S = rows[inst / B];
    for (int b = 1; b < nb; ++b) S -= h[b];
    for (int t = t0; t < T; ++t) {
        int32_t E = 0, In = 0, RM = h[1];
        for (int d = t - tau_EI + 1; d <= t - 1; ++d) E += cnt(d);
        for (int d = t - L + 1; d <= t - tau_EI; ++d) In += cnt(d);
        for (int d = t0 - L; d <= t - L; ++d) RM += cnt(d);
        int32_t *cp = counts + ((size_t)inst * ldP + t) * 4;
        cp[0] = S;
        cp[1] = E;
        cp[2] = In;
        cp[3] = RM;
        newRM[(size_t)inst * ldP + t] = cnt(t - L);
        S -= ni[t];
    }
}

// Level 1 of the parameter-gradient reduction: Pc[t][g][c][a][s] = sum over the
// tiles [c K, min((c+1) K, ntiles_g)) of graph g of P[t][tile][a][s], K = kReduceChunkTiles.
__global__ void k_reduce_b1(const double *P, int ntiles, const int32_t *tile0, const int32_t *ntl, int G, int Bp,
                            int max_chunks, double *Pc) {
    const int c = blockIdx.x, t = blockIdx.y, g = blockIdx.z;
    const int wdt = kAges * Bp;
    const int nt = ntl[g];
    const int i0 = c * kReduceChunkTiles, i1 = min(nt, i0 + kReduceChunkTiles);
    const double *base = P + ((size_t)t * ntiles + tile0[g]) * wdt;
    for (int k = threadIdx.x; k < wdt; k += blockDim.x) {
        double acc = 0.0;
        for (int i = i0; i < i1; ++i) acc += base[(size_t)i * wdt + k];
        Pc[(((size_t)t * G + g) * max_chunks + c) * wdt + k] = acc;
    }
}

// Level 2: Q[g*B+s][t][a] = sum over the chunks, in order.
__global__ void k_reduce_b2(const double *Pc, int G, int B, int Bp, int T, int max_chunks, const int32_t *sig,
                            int ld_sig, double *Q) {
    const int t = blockIdx.x, g = blockIdx.y;
    const int wdt = kAges * Bp;
    for (int k = threadIdx.x; k < wdt; k += blockDim.x) {
        const int b = k / Bp, s = k - b * Bp;
        double acc = 0.0;
        const double *p = Pc + ((size_t)t * G + g) * max_chunks * wdt + k;
        for (int c = 0; c < max_chunks; ++c) acc += p[(size_t)c * wdt];
        if (s < B) Q[((size_t)(g * B + s) * T + t) * kAges + b] = ldexp(acc, sig[(size_t)g * ld_sig + t]);
    }
}

// The seeds' share of the table adjoint through day 0, one thread per (tile, set): a
// seed exposed on day E < 0 is infectious on day 0 with k = -E, and gx(0) = sum over its
// out-edges of w r(0) (r(0) at scale 2^sigma(0) of its graph).  The thread adds its
// tile's seeds in row order, so the sums do not depend on scheduling.
__global__ void k_dc_seeds_b(Csr m, const int16_t *E, const float *r0, GraphRef gr, const int32_t *sig,
                             int ld_sig, int ntiles, int L, int B, int Bp, double *dc_tile) {
    const int64_t total = (int64_t)ntiles * B;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int tile = (int)(idx / B), s = (int)(idx - (int64_t)tile * B);
        const int g = gr.tile_graph ? (int)gr.tile_graph[tile] : 0;
        const double scale = ldexp(1.0, sig[(size_t)g * ld_sig]);
        for (int r = 0; r < kTile; ++r) {
            const int row = tile * kTile + r;
            const int Eh = E[(size_t)row * Bp + s];
            if (Eh == kPad || Eh >= 0 || -Eh > L - 1) continue;
            float gx = 0.f;
            for (uint32_t p = m.rowptr[row]; p < m.rowptr[row + 1]; ++p)
                gx = __fmaf_rn(m.w[p], r0[(size_t)m.col[p] * Bp + s], gx);
            dc_tile[((size_t)tile * L - Eh) * Bp + s] += (double)gx * scale;
        }
    }
}

// dc[g*B+s][k] = sum over the tiles of graph g of dc_tile[tile][k][s] (fixed order, FP64).
__global__ void __launch_bounds__(256) k_dc_reduce_b(const double *dc_tile, const int32_t *graph_tile0,
                                                     const int32_t *graph_ntiles, int B, int Bp, int L, double *dc) {
    __shared__ double sh[256];
    const int inst = blockIdx.x, k = blockIdx.y;
    const int g = inst / B, s = inst - g * B;
    const int tile0 = graph_tile0[g], nt = graph_ntiles[g];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) acc += dc_tile[((size_t)(tile0 + i) * L + k) * Bp + s];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) dc[(size_t)inst * L + k] = (k == 0) ? 0.0 : sh[0];
}

// ---- dispatch over (lanes per row, sets per lane) -------------------------
template <int LPR, int SPL>
cudaError_t launch_fwd_cfg(const FwdBatchArgs &a, bool kahan, int grid, cudaStream_t s) {
    if (kahan) k_fwd_day_b<LPR, SPL, true><<<grid, kBlock, 0, s>>>(a);
    else k_fwd_day_b<LPR, SPL, false><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <int LPR, int SPL, bool KAHAN>
cudaError_t launch_bwd_dc(const BwdBatchArgs &a, int grid, cudaStream_t s) {
    const size_t bytes = sizeof(float) * (size_t)(kBlock / 32) * a.L * (LPR * SPL);
    if (bytes > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_bwd_day_b<LPR, SPL, KAHAN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
        if (e != cudaSuccess) return e;
    }
    k_bwd_day_b<LPR, SPL, KAHAN, true><<<grid, kBlock, bytes, s>>>(a);
    return cudaGetLastError();
}

template <int LPR, int SPL>
cudaError_t launch_bwd_cfg(const BwdBatchArgs &a, bool kahan, int grid, cudaStream_t s) {
    if (a.dc_tile) return kahan ? launch_bwd_dc<LPR, SPL, true>(a, grid, s) : launch_bwd_dc<LPR, SPL, false>(a, grid, s);
    if (kahan) k_bwd_day_b<LPR, SPL, true, false><<<grid, kBlock, 0, s>>>(a);
    else k_bwd_day_b<LPR, SPL, false, false><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <class K>
int blocks_of(K kernel) {
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, kBlock, 0);
    return blocks > 0 ? blocks : 1;
}

template <int LPR, int SPL>
int occ_cfg(bool fwd, bool kahan) {
    if (fwd) return kahan ? blocks_of(k_fwd_day_b<LPR, SPL, true>) : blocks_of(k_fwd_day_b<LPR, SPL, false>);
    return kahan ? blocks_of(k_bwd_day_b<LPR, SPL, true, false>) : blocks_of(k_bwd_day_b<LPR, SPL, false, false>);
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

bool batch_config_ok(int Bp, int spl) {
#define X(bp, sp) if (Bp == bp && spl == sp) return true;
    GABM_BATCH_CONFIGS(X)
#undef X
    return false;
}

cudaError_t launch_fwd_day_b(const FwdBatchArgs &a, int Bp, int spl, bool kahan, int grid, cudaStream_t s) {
#define X(bp, sp) if (Bp == bp && spl == sp) return launch_fwd_cfg<bp / sp, sp>(a, kahan, grid, s);
    GABM_BATCH_CONFIGS(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_bwd_day_b(const BwdBatchArgs &a, int Bc, int spl, bool kahan, int grid, cudaStream_t s) {
#define X(bp, sp) if (Bc == bp && spl == sp) return launch_bwd_cfg<bp / sp, sp>(a, kahan, grid, s);
    GABM_BATCH_CONFIGS(X)
#undef X
    return cudaErrorInvalidValue;
}

int occupancy_fwd_b(int Bp, int spl, bool kahan) {
#define X(bp, sp) if (Bp == bp && spl == sp) return occ_cfg<bp / sp, sp>(true, kahan);
    GABM_BATCH_CONFIGS(X)
#undef X
    return 1;
}

int occupancy_bwd_b(int Bc, int spl, bool kahan) {
#define X(bp, sp) if (Bc == bp && spl == sp) return occ_cfg<bp / sp, sp>(false, kahan);
    GABM_BATCH_CONFIGS(X)
#undef X
    return 1;
}

cudaError_t launch_infectious_bits_b(const int16_t *e, int Bp, int t0, int L, int ntiles, uint32_t *bits,
                                     cudaStream_t s) {
    int grid = (ntiles + 7) / 8;
    if (grid > 65535) grid = 65535;
    k_infectious_bits_b<<<grid > 0 ? grid : 1, 256, 0, s>>>(e, Bp, t0, L, ntiles, bits);
    return cudaGetLastError();
}

cudaError_t launch_exposure_hist_b(const int16_t *e, GraphRef gr, int64_t n_rows, int B, int Bp, int t0, int L,
                                   int32_t *H, cudaStream_t s) {
    int64_t grid = (n_rows * Bp + 255) / 256;
    if (grid > 4096) grid = 4096;
    k_exposure_hist_b<<<(int)(grid > 0 ? grid : 1), 256, 0, s>>>(e, gr, n_rows, B, Bp, t0, L, H);
    return cudaGetLastError();
}

cudaError_t launch_counts_b(const uint8_t *tile_new, int ntiles, const int32_t *d_tile0, const int32_t *d_ntiles,
                            const int32_t *d_rows, int G, int B, int Bp, int max_tiles, int t0, int T, int ldP,
                            int tau_EI, int L, const int32_t *H, int32_t *newinf, int32_t *counts, int32_t *newRM,
                            cudaStream_t s) {
    if (T > t0) {
        const int chunks = (max_tiles + kReduceChunkTiles * 4 - 1) / (kReduceChunkTiles * 4);
        k_newinf_b<<<dim3(std::max(chunks, 1), T - t0, G), 64, 0, s>>>(tile_new, ntiles, d_tile0, d_ntiles, B, Bp, t0,
                                                                        ldP, newinf);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int I = G * B;
    k_counts_b<<<(I + 127) / 128, 128, 0, s>>>(H, newinf, d_rows, B, I, ldP, t0, T, tau_EI, L, counts, newRM);
    return cudaGetLastError();
}

cudaError_t launch_bwd_reduce_b(const double *P, int ntiles, const int32_t *d_tile0, const int32_t *d_ntiles, int G,
                                int B, int Bp, int T, double *scratch, int max_chunks, const int32_t *sig,
                                int ld_sig, double *Q, cudaStream_t s) {
    const int wdt = kAges * Bp;
    const int threads = std::min(1024, (wdt + 31) / 32 * 32);
    k_reduce_b1<<<dim3(max_chunks, T, G), threads, 0, s>>>(P, ntiles, d_tile0, d_ntiles, G, Bp, max_chunks, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_b2<<<dim3(T, G), threads, 0, s>>>(scratch, G, B, Bp, T, max_chunks, sig, ld_sig, Q);
    return cudaGetLastError();
}

cudaError_t launch_dc_seeds_b(Csr m_out, const int16_t *E, const float *r0, GraphRef gr, const int32_t *sig,
                              int ld_sig, int ntiles, int L, int B, int Bp, double *dc_tile, cudaStream_t s) {
    const int64_t total = (int64_t)ntiles * B;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 65535));
    k_dc_seeds_b<<<grid, 256, 0, s>>>(m_out, E, r0, gr, sig, ld_sig, ntiles, L, B, Bp, dc_tile);
    return cudaGetLastError();
}

cudaError_t launch_dc_reduce_b(const double *dc_tile, const int32_t *graph_tile0, const int32_t *graph_ntiles, int G,
                               int B, int Bp, int L, double *dc, cudaStream_t s) {
    k_dc_reduce_b<<<dim3(G * B, L), 256, 0, s>>>(dc_tile, graph_tile0, graph_ntiles, B, Bp, L, dc);
    return cudaGetLastError();
}

}  // namespace gabm
