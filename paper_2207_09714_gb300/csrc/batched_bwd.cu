// batched_bwd.cu -- the reverse day kernel of the batched instances (B parameter sets
// sharing each graph; layout and schedules as described in batched.cu): the transpose
// gather of day t+1 and the straight-through adjoint of day t's draws for every set,
// with the table adjoint as a separate instance.
#include "batched_common.cuh"

namespace gabm {

namespace {

// ---------------------------------------------------------------------------
// Reverse day t for every set: the transpose gather of day t+1 and the
// straight-through adjoint of day t's draws (the per-set steps of backward.cu).
// ---------------------------------------------------------------------------
// DC: also accumulate the adjoint of the infectiousness table (a.dc_tile), a separate
// instance so that the plain sweep carries none of its code.  REC (recompute policy,
// symmetric weights): lambda is not stored but summed again from the final exposure
// days over the same entries, with the forward's marking (a.bits_t) and order, so it
// is bitwise the forward's.
template <int LPR, int SPL, bool KAHAN, bool DC, bool REC = false>
__global__ void __launch_bounds__(kBlock, GABM_BBWD_MINBLOCKS) k_bwd_day_b(const BwdBatchArgs a) {
    constexpr int RPW = 32 / LPR;
    constexpr int Bc = LPR * SPL;        // sets of this launch (a chunk of the row's Bw)
    constexpr int NW = kBlock / 32;
    // DC: per-warp tile sums [L][Bc] of gx at the rows' infectious days, by k = t + 1 - E
    extern __shared__ float dcs_all[];
    __shared__ float c_s[kMaxL + 1];    // c_s[k] = 0 for k >= L (the clamped lookup)
    __shared__ int slot_k[kMaxL];
    __shared__ float pacc[NW][kAges][Bc];   // per-warp tile sums of gl * Lam by age and set
    __shared__ float fac_s[NW][kMaxL];       // 2^(sigma(t+k) - sigma(t)) of the warp's graph
    if (threadIdx.x < kMaxL) {
        c_s[threadIdx.x] = a.c[threadIdx.x];
        slot_k[threadIdx.x] = a.ring_slot[threadIdx.x];
    }
    if (threadIdx.x == kMaxL) c_s[kMaxL] = 0.f;
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

            // REC: the day's lambda sums of the row's susceptible sets, from the final state
            float Lrec[SPL];
            if constexpr (REC) {
                const bool actl = (group_bits<LPR>(__ballot_sync(kFull, anyS)) >> grp) & 1u;
                auto lde = [&](uint32_t j, bool ok, EWords<SPL> &rw) {
                    ld_words<SPL>(E32 + ((size_t)j * Bw + s0) / 2, ok, rw.w);
                };
                auto vale = [&](const EWords<SPL> &rw, int h) {
                    return infect_lut(half_of(rw.w[h >> 1], h & 1), c_s, t, (unsigned)L);
                };
                group_row_sums<LPR, SPL, KAHAN, EWords<SPL>>(a.m, cu.p0, actl ? cu.len : 0u, cu.j0, cu.w0, a.bits_t,
                                                             lane, lde, vale, Lrec);
#pragma unroll
                for (int h = 0; h < SPL; ++h) Lrec[h] = Lrec[h] * inv_D;
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
                if constexpr (REC) {
#pragma unroll
                    for (int h = 0; h < SPL; ++h) Lv[h] = Lrec[h];
                } else {
                    ld_floats<SPL>(a.lam_t + xo, true, Lv);
                }
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
    if (!a.lam_t) {   // recompute policy (no table adjoint)
        if (a.dc_tile) return cudaErrorInvalidValue;
        if (kahan) k_bwd_day_b<LPR, SPL, true, false, true><<<grid, kBlock, 0, s>>>(a);
        else k_bwd_day_b<LPR, SPL, false, false, true><<<grid, kBlock, 0, s>>>(a);
        return cudaGetLastError();
    }
    if (a.dc_tile) return kahan ? launch_bwd_dc<LPR, SPL, true>(a, grid, s) : launch_bwd_dc<LPR, SPL, false>(a, grid, s);
    if (kahan) k_bwd_day_b<LPR, SPL, true, false><<<grid, kBlock, 0, s>>>(a);
    else k_bwd_day_b<LPR, SPL, false, false><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <int LPR, int SPL>
int occ_bwd_cfg(bool kahan) {
    return kahan ? blocks_of(k_bwd_day_b<LPR, SPL, true, false>) : blocks_of(k_bwd_day_b<LPR, SPL, false, false>);
}

}  // namespace

cudaError_t launch_bwd_day_b(const BwdBatchArgs &a, int Bc, int spl, bool kahan, int grid, cudaStream_t s) {
#define X(bp, sp) if (Bc == bp && spl == sp) return launch_bwd_cfg<bp / sp, sp>(a, kahan, grid, s);
    GABM_BATCH_CONFIGS(X)
#undef X
    return cudaErrorInvalidValue;
}

int occupancy_bwd_b(int Bc, int spl, bool kahan) {
#define X(bp, sp) if (Bc == bp && spl == sp) return occ_bwd_cfg<bp / sp, sp>(kahan);
    GABM_BATCH_CONFIGS(X)
#undef X
    return 1;
}

}  // namespace gabm
