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
#include "batched_common.cuh"

namespace gabm {

namespace {

// ---------------------------------------------------------------------------
// Forward day t for every set (Transmit, draw, Progress).
// ---------------------------------------------------------------------------
template <int LPR, int SPL, bool KAHAN>
__global__ void __launch_bounds__(kBlock, GABM_BFWD_MINBLOCKS) k_fwd_day_b(const FwdBatchArgs a) {
    constexpr int RPW = 32 / LPR;
    constexpr int Bp = LPR * SPL;
    constexpr int NW = kBlock / 32;
    __shared__ float c_s[kMaxL + 1];
    __shared__ float lam_s[NW][SPL * 32];   // a pass's lambdas, by set position and lane
    __shared__ int hit_s[NW][SPL * 32];     // draws that exposed, by set position and lane
    const int lane = threadIdx.x & 31;
    float *lam_w = lam_s[threadIdx.x >> 5];
    int *hit_w = hit_s[threadIdx.x >> 5];
    if (threadIdx.x <= kMaxL) c_s[threadIdx.x] = threadIdx.x < kMaxL ? a.c[threadIdx.x] : 0.f;
#pragma unroll
    for (int h = 0; h < SPL; ++h) hit_w[h * 32 + lane] = 0;
    __syncthreads();

    const int grp = lane / LPR, q = lane % LPR;
    const int t = a.t, L = a.L, B = a.B, ntiles = a.ntiles;
    uint32_t *e32 = reinterpret_cast<uint32_t *>(a.e);
    const uint32_t *e32r = e32;
    constexpr int WPR = Bp / 2;   // 32-bit words per row of e

    auto ld = [&](uint32_t j, bool ok, EWords<SPL> &r) { ld_words<SPL>(e32r + (size_t)j * WPR + q * (SPL / 2), ok, r.w); };
    auto val = [&](const EWords<SPL> &r, int h) { return infect_lut(half_of(r.w[h >> 1], h & 1), c_s, t, (unsigned)L); };

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

            // lambda of each susceptible set with an infectious neighbour; only those draw
            float Lam[SPL];
            uint32_t dmask[SPL];
            int ndraw = 0;
#pragma unroll
            for (int h = 0; h < SPL; ++h) {
                const bool need = sS[h] && sum[h] != 0.f;   // lambda = 0: p = 0, no draw
                Lam[h] = need ? sum[h] * inv_D : 0.f;
                dmask[h] = __ballot_sync(kFull, need);
                ndraw += __popc(dmask[h]);
            }
            // The pass's draws (expm1f and Philox) are dealt to the lanes 32 at a time.  Drawn
            // where they sit, they would run once for every set position in which any lane of
            // the warp draws, with most lanes idle.  A draw's result returns to its lane through
            // shared memory; each draw computes exactly what the lane owning the set would.
            uint32_t drew = 0u;   // bit h: set h of this lane exposed today
            if (ndraw) {
#pragma unroll
                for (int h = 0; h < SPL; ++h) lam_w[h * 32 + lane] = Lam[h];
                __syncwarp();
                for (int base = 0; base < ndraw; base += 32) {
                    const int pi = base + lane;
                    // set position hs of draw pi and its index among that position's draws
                    int hs = 0, before = 0;
                    uint32_t msel = dmask[0];
#pragma unroll
                    for (int h = 0; h + 1 < SPL; ++h) {
                        const int upto = before + __popc(dmask[h]);
                        if (hs == h && pi >= upto) {
                            hs = h + 1;
                            before = upto;
                            msel = dmask[h + 1];
                        }
                    }
                    if (pi < ndraw) {
                        const int src = nth_set_bit(msel, pi - before);
                        const int srow = tile * kTile + pass * RPW + src / LPR;
                        const int inst = g * B + (src % LPR) * SPL + hs;
                        const float lam = (a.R[(size_t)inst * a.ldP + t] * a.S[inst * kAges + a.age[srow]]) *
                                          lam_w[hs * 32 + src];
                        const float p = -expm1f(-lam);
                        if (p > kUmin) {
                            const uint32_t id = caller_id(a.gr, srow, g);
                            if (uniform_from_word(philox_word(a.seed, id, (uint32_t)t, (uint32_t)inst, 0u)) < p)
                                hit_w[hs * 32 + src] = 1;
                        }
                    }
                }
                __syncwarp();
#pragma unroll
                for (int h = 0; h < SPL; ++h) {
                    if (hit_w[h * 32 + lane]) {
                        drew |= 1u << h;
                        hit_w[h * 32 + lane] = 0;
                    }
                }
                __syncwarp();
            }

            bool inf = false;
            if (mine) {
                uint32_t nw[SPL / 2];
#pragma unroll
                for (int k = 0; k < SPL / 2; ++k) nw[k] = ew[k];
#pragma unroll
                for (int h = 0; h < SPL; ++h) {
                    if ((drew >> h) & 1u) {
                        const uint32_t tv = (uint32_t)(uint16_t)(int16_t)t;
                        nw[h >> 1] = (h & 1) ? ((nw[h >> 1] & 0xffffu) | (tv << 16)) : ((nw[h >> 1] & 0xffff0000u) | tv);
                        ++nnew[h];
                    }
                }
                if (drew) st_words<SPL>(mine_p, nw);
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

template <int LPR, int SPL>
cudaError_t launch_fwd_cfg(const FwdBatchArgs &a, bool kahan, int grid, cudaStream_t s) {
    if (kahan) k_fwd_day_b<LPR, SPL, true><<<grid, kBlock, 0, s>>>(a);
    else k_fwd_day_b<LPR, SPL, false><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <int LPR, int SPL>
int occ_fwd_cfg(bool kahan) {
    return kahan ? blocks_of(k_fwd_day_b<LPR, SPL, true>) : blocks_of(k_fwd_day_b<LPR, SPL, false>);
}

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

int occupancy_fwd_b(int Bp, int spl, bool kahan) {
#define X(bp, sp) if (Bp == bp && spl == sp) return occ_fwd_cfg<bp / sp, sp>(kahan);
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
