// backward.cu -- hand-written straight-through adjoint of the day loop (App. B).
//
// The reverse sweep runs one launch per day t = T-1 .. 0.  Launch t fuses two
// steps that touch the same rows:
//   (1) the transpose gather of day t+1: gx_i(t+1) = sum_{j in out(i)} w_ij r_j(t+1),
//       a pull over the source-sorted CSR (the forward CSR itself when the
//       weights are symmetric), so no atomics; written to a ring of the last
//       L-1 days;
//   (2) for every agent susceptible on day t, the adjoint of its draw:
//       G_i(t) = m_{t+L} gD_{t+L} + sum_{k=1}^{L-1} c[k] gx_i(t+k),
//       dL/dy = G (t = E_i or never infected) or G - A_i (t < E_i), A_i = G_i(E_i),
//       gl = dL/dy * dy_soft/dlambda (Gumbel-softmax, tau = 1, straight-through),
//       r_i(t) = R_t S[a_i] gl / Dbar and per-tile, per-age sums of gl * Lam.
// lambda_i(t) comes from the forward's store or is recomputed from the final
// exposure days E (no reinfection, A3/A4 of App. A, so E determines every
// day's state and no checkpoints are needed): in the same pass when in- and
// out-edges coincide, else by k_lam_day over the in-edges first.  Each warp
// prefetches the next tile's id, row data and (into L2) its edge range while
// it works on the current tile.
#include "gabm_internal.cuh"
#include "rowsum.cuh"

namespace gabm {

namespace {

// Adds this tile's share of the table adjoint dL/dc[k] = sum_j gx_j(E_j + k): every lane
// with `has` holds gx of its row for the day that is k = kd days after the row's
// exposure, at scale 2^sigma of that day.  Rows with equal k are summed over the warp
// (fp32, fixed tree), then added in FP64 to the tile's accumulator, whose only writer
// is the warp holding the tile (days are sequential launches).  Called by all 32 lanes.
__device__ __forceinline__ void dc_accumulate(double *dc_tile, int tile, bool has, int kd, float gx, int sigma,
                                              int lane) {
    unsigned pend = __ballot_sync(0xffffffffu, has);
    if (!pend) return;
    // lane k keeps the sum for k (k < L <= 32), so the read-modify-writes of all k go out together
    float mine = 0.f;
    bool touched = false;
    while (pend) {
        const int k0 = __shfl_sync(0xffffffffu, kd, __ffs(pend) - 1);
        const bool sel = has && kd == k0;
        float v = sel ? gx : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == k0) {
            mine = v;
            touched = true;
        }
        pend &= ~__ballot_sync(0xffffffffu, sel);
    }
    if (touched) dc_tile[(size_t)tile * kMaxL + lane] += (double)mine * ldexp(1.0, sigma);
}

// DC: accumulate the table adjoint (a.dc_tile); a separate instance, so the plain sweep
// carries none of its code.
// Four resident blocks (64 registers) for the plain store sweep: the gathers of r want
// the warps (79 vs 82 us per day on the 1M-agent graph at three).  The fused, soft and
// table-adjoint instances, which spill at 64 registers, keep three.
#ifndef GABM_BWD_MINBLOCKS
#define GABM_BWD_MINBLOCKS 4
#endif
// EXIT = kExitFate (sampled R/M split, store policy): G of an exposure today takes the
// fate it would draw (window L_R or L_M; the death term gD_{t+L_M} only if M-fated), and
// the rows exposed today add H dphi/dm to day t + tau_EI's dL/dm, H = dL/dphi = sum over
// the days between the two exits of +-c[k] gx(t+k) plus gD_{t+L_M}.  Rows exposed before
// day 0 keep their gx in the ring for k_fate_seeds.
// EXIT = kExitDur (stochastic I-stage durations, store policy): G of an exposure today
// sums over the window L_i it would draw and takes the death term m gD of its own exit
// day; the exits recounted for dm are at each row's drawn L_i.
template <int MODE, bool DC, int EXIT = kExitBase>
__global__ void __launch_bounds__(kBlock, (MODE == kBwdStore && !DC) ? GABM_BWD_MINBLOCKS : GABM_MINBLOCKS)
    k_bwd_day(const BwdDayArgs a) {
    constexpr bool FATE = EXIT == kExitFate;
    constexpr bool DUR = EXIT == kExitDur;
    constexpr int NARR = (MODE == kBwdFused) ? 2 : 1;
    constexpr bool SOFT = MODE == kBwdSoft;
    constexpr int RB = 8;   // ring slots loaded together in the epilogue (16: 4% slower)
    __shared__ float c_s[kMaxL];
    __shared__ int slot_k[kMaxL];
    __shared__ int32_t red_s[kBlock / 32][2];
    __shared__ float fac_s[kBlock / 32][kMaxL];   // 2^(sigma(t+k) - sigma(t)) of the warp's graph
    __shared__ double F_s[kMaxL];
    if (threadIdx.x < kMaxL) {
        c_s[threadIdx.x] = a.c[threadIdx.x];
        slot_k[threadIdx.x] = a.ring_slot[threadIdx.x];
        if (DUR) F_s[threadIdx.x] = a.dur.F[threadIdx.x];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int t = a.t, T = a.T, L = a.L, ntiles = a.ntiles;
    const int32_t *sg = nullptr;   // scale exponents of the current graph
    int sig_t = 0;                 // sigma(t) of the current graph
    unsigned emax_w = 0u;          // largest exponent stored by this warp (+128)
    float gtail = 0.f;             // m_{t+L} gD_{t+L} at day t's scale
    const bool has_next = (t + 1 < T);
    const int16_t *E = a.E;
    const float *__restrict__ r_next = a.r_next;
    const uint32_t *bits = a.bits_t;
    // contribution 0: w * r_j(t+1) (transpose gather); contribution 1 (recompute):
    // w * c[t - E_j] for neighbours marked infectious on day t
    auto contrib = [&](uint32_t j, float w, bool valid, float (&out)[NARR], bool (&take)[NARR]) {
        out[0] = w * ld_if(r_next + j, valid);
        take[0] = valid;
        if constexpr (NARR == 2) {
            const bool mk = valid && marked(bits, j);
            const int Ej = ld_if(E + j, mk, kNever);
            out[1] = mk ? w * infectiousness(Ej, c_s, t, L) : 0.f;
            take[1] = mk;
        }
    };

    int cur_g = -1, cN = 0;
    BlockTiles disp;
    disp.init(ntiles, lane);
    TileRows cur, nxt;
    load_tile_rows(a.m, E, a.gr.tile_graph, ntiles, disp.get(), lane, cur);
    load_tile_rows(a.m, E, a.gr.tile_graph, ntiles, disp.get(), lane, nxt);
    prefetch_slice(a.m, cur.p0, cur.p1, lane);
    while (cur.tile < ntiles) {
        prefetch_slice(a.m, nxt.p0, nxt.p1, lane);
        TileRows nn;
        load_tile_rows(a.m, E, a.gr.tile_graph, ntiles, disp.get(), lane, nn);

        const int g = cur.g, tile = cur.tile, Ei = cur.e;
        if (g != cur_g) {
            if (cur_g >= 0) {
                const int sN = __reduce_add_sync(0xffffffffu, cN);
                if (lane == 0 && sN) atomicAdd(a.newRM + (size_t)cur_g * a.ldP + t, sN);
                flush_emax(a.emax + (size_t)cur_g * a.ld_sig + t, emax_w);
                emax_w = 0u;
            }
            // this day's scale for graph g (every warp computes the same value; the warp
            // holding the graph's first tile records it)
            sg = a.sig + (size_t)g * a.ld_sig;
            sig_t = next_sigma(sg[t + 1], a.emax[(size_t)g * a.ld_sig + t + 1]);
            if (lane == 0 && tile * kTile == a.gr.row0[g]) a.sig[(size_t)g * a.ld_sig + t] = sig_t;
            if (lane < kMaxL)
                fac_s[wib][lane] = (lane >= 1 && lane < L && t + lane <= T) ? exp2i(sg[t + lane] - sig_t) : 0.f;
            {
                const size_t pg = (size_t)g * a.ldP;
                if constexpr (FATE)   // deaths are counted: dL/d(one M entry on day t + L_M)
                    gtail = (t + a.fate.L_M < T) ? (float)a.gD[pg + t + a.fate.L_M] * exp2i(-sig_t) : 0.f;
                else
                    gtail = (t + L < T) ? a.m_t[pg + t + L] * (float)a.gD[pg + t + L] * exp2i(-sig_t) : 0.f;
            }
            __syncwarp();
            cur_g = g;
            cN = 0;
        }
        const int row = tile * kTile + lane;
        const bool agent = (Ei != kPad);
        const bool never = (Ei == kNever);
        const bool live = agent && (never || Ei >= 0);           // seeds are constants
        // soft relaxation: every agent carries susceptible mass and draws every day
        const bool isS = SOFT ? agent : live && (never || Ei >= t);
        // R/M split: rows exposed before day 0 keep gx while day t+1 is inside their window
        const bool needA = has_next && (SOFT ? agent : (live && (never || Ei >= t + 2 - L)) ||
                                                       (FATE && agent && !never && Ei < 0 && t + 1 - Ei < L));
        if constexpr (DUR) {
            // exits at the row's drawn L_i (its first possible day is tau_EI + 1)
            const int k = t - Ei;
            if (agent && !never && k > a.tau_EI && k <= L)
                cN += (k == dur_exit(a.dur, F_s, caller_id(a.gr, row, g), Ei, g));
        } else if (!SOFT) {
            cN += (agent && !never && t - Ei == L);
        }
        // table adjoint: rows infectious on day t+1 (k = t+1-E in [1, L-1]) add gx(t+1) to
        // dc[k]; the non-seed ones are already gathered (needA), the seeds only for this
        const int kd = t + 1 - Ei;
        const bool dc_row = DC && !SOFT && has_next && agent && !never && kd >= 1 && kd <= L - 1;

        // the epilogue's row loads that do not depend on the sums go out before them, so
        // that their latency overlaps the entry stream; A was stored on day E_i (soft:
        // dL/ds on day t+1) at that day's scale
        const bool readA = SOFT || (!never && Ei != t);
        const float A_ld = ld_if(a.A + row, isS && readA);
        float lam_ld = 0.f;
        if constexpr (MODE != kBwdFused) lam_ld = ld_if(a.lam_t + row, isS);
        const int age_ld = isS ? (int)a.age[row] : 0;

        float sum[NARR];
        {
            const bool act = (MODE == kBwdFused) ? (needA || isS || dc_row) : (needA || dc_row);
            bool want[NARR];
            want[0] = needA || dc_row;
            if constexpr (NARR == 2) want[1] = isS;
            if constexpr (NARR == 1)   // every valid entry's w r_j(t+1) is taken
                row_sums<1>(a.m, cur.p0, cur.len, act, lane, contrib, want, sum,
                            [&](uint32_t j, float w) { return w * r_next[j]; });
            else
                row_sums<NARR>(a.m, cur.p0, cur.len, act, lane, contrib, want, sum);
        }
        float gx_mine = sum[0];
        if (a.self_q) gx_mine = __fmaf_rn(-a.self_q[row], a.self_r[row], gx_mine);

        if (needA) a.ring[(size_t)slot_k[1] * a.ring_stride + row] = gx_mine;
        if constexpr (DC && !SOFT) dc_accumulate(a.dc_tile, tile, dc_row, kd, gx_mine, sg[t + 1], lane);
        if constexpr (DC && SOFT) {
            // soft: every agent's mass exposed k days before t+1 counts, n_j(d) = s_j(d) y_j(d)
            // for d >= 0 and the seeds' unit mass on their day E_j < 0 (lane k keeps k's sum)
            const bool on = has_next && agent;
            if (__any_sync(0xffffffffu, on)) {
                float mine = 0.f;
                for (int k = 1; k < L; ++k) {
                    const int d = t + 1 - k;
                    float nk = 0.f;
                    if (on)
                        nk = (d >= 0) ? a.s_hist[(size_t)d * a.hist_stride + row] * a.y_hist[(size_t)d * a.hist_stride + row]
                                      : (Ei == d ? 1.f : 0.f);
                    float v = nk * gx_mine;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == k) mine = v;
                }
                if (lane >= 1 && lane < L && mine != 0.f)
                    a.dc_tile[(size_t)tile * kMaxL + lane] += (double)mine * ldexp(1.0, sg[t + 1]);
            }
        }

        float v = 0.f, pm = 0.f;
        int ai = 0;
        if (isS) {
            ai = age_ld;
            const int inst = g;
            const size_t pi = (size_t)inst * a.ldP;
            const float Apre = readA ? A_ld * (SOFT ? fac_s[wib][1] : exp2i(sg[Ei] - sig_t)) : 0.f;
            float Lam;
            if constexpr (MODE == kBwdFused) Lam = sum[NARR - 1] * a.gr.inv_Dbar[g];
            else Lam = lam_ld;
            // R/M split: the fate an exposure today would draw on day t + tau_EI
            bool phi = false;
            float vf = 0.5f;
            int Lx = L;
            if constexpr (FATE) {
                if (t + a.tau_EI < T) {
                    vf = fate_uniform(a.fate, caller_id(a.gr, row, g), t + a.tau_EI, g);
                    phi = vf < a.m_t[(size_t)g * a.ldP + t + a.tau_EI];
                }
                Lx = phi ? a.fate.L_M : a.fate.L_R;
            }
            const int Lmin = FATE ? min(a.fate.L_R, a.fate.L_M) : L;
            const float sgn = (FATE && a.fate.L_M > a.fate.L_R) ? 1.f : -1.f;
            if constexpr (DUR) {
                // the window an exposure today would draw, and the death term of its exit day
                Lx = dur_exit(a.dur, F_s, caller_id(a.gr, row, g), t, g);
                const size_t pg = (size_t)g * a.ldP;
                gtail = (t + Lx < T) ? a.m_t[pg + t + Lx] * (float)a.gD[pg + t + Lx] * exp2i(-sig_t) : 0.f;
            }
            float G = (FATE && !phi) ? 0.f : gtail;
            float H = gtail;
            if (has_next) G = __fmaf_rn(c_s[1], gx_mine * fac_s[wib][1], G);
            for (int k0 = 2; k0 < L; k0 += RB) {
                float rv[RB];
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const int k = k0 + u;
                    const bool ok = k < L && t + k < T;
                    rv[u] = ld_if(a.ring + (size_t)slot_k[ok ? k : 0] * a.ring_stride + row, ok);
                }
#pragma unroll
                for (int u = 0; u < RB; ++u) {
                    const int k = k0 + u;
                    if (k < L && t + k < T) {
                        const float gk = rv[u] * fac_s[wib][k];
                        if (!(FATE || DUR) || k < Lx) G = __fmaf_rn(c_s[k], gk, G);
                        if (FATE && k >= Lmin) H = __fmaf_rn(sgn * c_s[k], gk, H);
                    }
                }
            }
            if constexpr (FATE) {
                // the fate draw of today's exposure: dphi_soft/dm = v (1-v) / (m (1-v) + (1-m) v)^2
                if (Ei == t && t + a.tau_EI < T) {
                    const float mI = a.m_t[(size_t)g * a.ldP + t + a.tau_EI];
                    const float den = __fmaf_rn(mI, 1.f - vf, (1.f - mI) * vf);
                    pm = H * ((vf * (1.f - vf)) / (den * den));
                }
            }
            float dy;
            float stored = fabsf(G);
            if (SOFT) {
                // dL/dy = s(t) (G - dL/ds(t+1));  dL/ds(t) = y G + (1 - y) dL/ds(t+1)
                const float ds = Apre;
                const float yv = a.y_hist_t[row];
                dy = a.s_hist_t[row] * (G - ds);
                const float dsn = __fmaf_rn(yv, G, (1.f - yv) * ds);
                a.A[row] = dsn;
                stored = fmaxf(stored, fabsf(dsn));
            } else if (Ei == t) { a.A[row] = G; dy = G; }
            else if (never) dy = G;
            else dy = G - Apre;
            const float RS = a.R[pi + t] * a.S[inst * kAges + ai];
            const float lam = RS * Lam;
            const float q = expf(-lam);
            const float p = -expm1f(-lam);
            const uint32_t id = caller_id(a.gr, row, g);
            const float u = uniform_from_word(philox_word(a.seed, id, (uint32_t)t, (uint32_t)inst, 0u));
            const float den = __fmaf_rn(p, 1.f - u, q * u);
            const float dydl = (u * (1.f - u)) * q / (den * den);
            const float glam = dy * dydl;
            const float rc = RS * glam * a.gr.inv_Dbar[g];
            a.r_cur[row] = rc;
            v = glam * Lam;
            stored = fmaxf(stored, fabsf(rc));
            emax_w = max(emax_w, (unsigned)(float_exponent(stored) + 128));
        }

        // per-tile sums of gl * Lam by age bin (fp32 over 32 rows, FP64 from here on)
        // (the recomputing instance keeps a butterfly per bin: with the reduce-scatter its
        // day took 1.37 ms against 0.92 on the 8M power-law workload)
        static_assert(kAges <= 16, "age bins fit the warp's bin sums");
        const unsigned smask = __ballot_sync(0xffffffffu, isS);
        if constexpr (NARR == 1) {
            float mine = 0.f;   // lanes 2b, 2b + 1: bin b
            if (smask) mine = warp_bin_sums16(isS ? v : 0.f, ai, lane);
            if (!(lane & 1) && (lane >> 1) < kAges) a.P_t[(size_t)tile * kAges + (lane >> 1)] = (double)mine;
        } else {
            double outv = 0.0;
            if (smask) {
                float vb[kAges];
#pragma unroll
                for (int b = 0; b < kAges; ++b) vb[b] = (isS && ai == b) ? v : 0.f;
#pragma unroll
                for (int b = 0; b < kAges; ++b)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) vb[b] += __shfl_xor_sync(0xffffffffu, vb[b], o);
                float mine = 0.f;
#pragma unroll
                for (int b = 0; b < kAges; ++b) if (lane == b) mine = vb[b];
                outv = (double)mine;
            }
            if (lane < kAges) a.P_t[(size_t)tile * kAges + lane] = outv;
        }
        if constexpr (FATE) {
            // dL/dm of day t + tau_EI from this tile's exposures today (fixed tree, FP64 out)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pm += __shfl_xor_sync(0xffffffffu, pm, o);
            if (lane == 0 && t + a.tau_EI < T) a.Pm_t[tile] = ldexp((double)pm, sig_t);
        }

        cur = nxt;
        nxt = nn;
    }

    const int sN = __reduce_add_sync(0xffffffffu, cN);
    if (cur_g >= 0) flush_emax(a.emax + (size_t)cur_g * a.ld_sig + t, emax_w);
    if (lane == 0) { red_s[wib][0] = cur_g; red_s[wib][1] = sN; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int g = -1;
        int32_t acc = 0;
        for (int w = 0; w <= kBlock / 32; ++w) {
            const int gw = (w < kBlock / 32) ? red_s[w][0] : -2;
            if (gw != g) {
                if (g >= 0 && acc) atomicAdd(a.newRM + (size_t)g * a.ldP + t, acc);
                g = gw;
                acc = 0;
            }
            if (w < kBlock / 32 && gw >= 0) acc += red_s[w][1];
        }
    }
}

// Normalised neighbour sums Lam_i(t) over the in-edges, recomputed from the final
// exposure days (used when the in- and out-edges differ, ahead of the backward day
// kernel of day t); the same per-row summation as the forward.
__global__ void __launch_bounds__(kBlock) k_lam_day(Sell m, const int16_t *E, const uint32_t *bits, GraphRef gr,
                                                    int t, int L, int ntiles, const float *c, float *lam_out) {
    __shared__ float c_s[kMaxL];
    if (threadIdx.x < kMaxL) c_s[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * (kBlock / 32);
    auto contrib = [&](uint32_t j, float w, bool valid, float (&out)[1], bool (&take)[1]) {
        const bool mk = valid && marked(bits, j);
        const int Ej = ld_if(E + j, mk, kNever);
        out[0] = mk ? w * infectiousness(Ej, c_s, t, L) : 0.f;
        take[0] = mk;
    };
    const bool want[1] = {true};
    for (int tile = blockIdx.x * (kBlock / 32) + wib; tile < ntiles; tile += nwarps) {
        const int row = tile * kTile + lane;
        const int Ei = E[row];
        const bool act = (Ei != kPad) && (Ei == kNever || Ei >= t);
        float sum[1];
        row_sums<1>(m, m.slice_ptr[tile], m.row_len[row], act, lane, contrib, want, sum);
        if (act) {
            const int g = gr.tile_graph ? (int)gr.tile_graph[tile] : 0;
            lam_out[row] = sum[0] * gr.inv_Dbar[g];
        }
    }
}

// The seeds' share of the table adjoint through day 0: a seed exposed on day E < 0 is
// infectious on day 0 with k = -E, and gx(0) = sum over its out-edges of w r(0) (r(0) at
// scale 2^sigma(0)).  Only tiles holding a seed do any work.
__global__ void __launch_bounds__(kBlock) k_dc_seeds(Sell m, const int16_t *E, const float *r0, GraphRef gr,
                                                     const int32_t *sig, int ld_sig, int ntiles, int L,
                                                     double *dc_tile) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * (kBlock / 32);
    auto contrib = [&](uint32_t j, float w, bool valid, float (&out)[1], bool (&take)[1]) {
        out[0] = w * ld_if(r0 + j, valid);
        take[0] = valid;
    };
    const bool want[1] = {true};
    for (int tile = blockIdx.x * (kBlock / 32) + wib; tile < ntiles; tile += nwarps) {
        const int row = tile * kTile + lane;
        const int Ei = E[row];
        const bool seed = Ei != kPad && Ei < 0 && -Ei <= L - 1;
        if (!__any_sync(0xffffffffu, seed)) continue;
        float sum[1];
        row_sums<1>(m, m.slice_ptr[tile], m.row_len[row], seed, lane, contrib, want, sum);
        const int g = gr.tile_graph ? (int)gr.tile_graph[tile] : 0;
        dc_accumulate(dc_tile, tile, seed, -Ei, sum[0], sig[(size_t)g * ld_sig], lane);
    }
}

// Sampled R/M split: the fate draws of agents exposed before day 0 (E < 0, drawn on day
// t_I = max(E + tau_EI, 0)).  H = gD_{E+L_M} + sum over k between the two exits of
// +-c[k] gx(E + k) over days 0..T-1: gx(0) gathered from r(0), later days from the ring
// (day d in slot d mod (L-1), written while the sweep ran).  Each tile adds its seeds'
// H dphi/dm per day t_I < tau_EI (warp tree in FP64) to Pm[t_I][tile], zeroed beforehand.
__global__ void __launch_bounds__(kBlock) k_fate_seeds(Sell m, const int16_t *E, const float *r0, const float *ring,
                                                       size_t ring_stride, int Lm1, GraphRef gr, FateRef f,
                                                       const double *gD, const int32_t *sig, int ld_sig, int ntiles,
                                                       int T, const float *c, double *Pm) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = gridDim.x * (kBlock / 32);
    const int L = Lm1 + 1;
    const int Lmin = min(f.L_R, f.L_M);
    const double sgn = f.L_M > f.L_R ? 1.0 : -1.0;
    auto contrib = [&](uint32_t j, float w, bool valid, float (&out)[1], bool (&take)[1]) {
        out[0] = w * ld_if(r0 + j, valid);
        take[0] = valid;
    };
    const bool want[1] = {true};
    for (int tile = blockIdx.x * (kBlock / 32) + wib; tile < ntiles; tile += nwarps) {
        const int row = tile * kTile + lane;
        const int Ei = E[row];
        const int tI = max(Ei + f.tau_EI, 0);
        const bool seed = Ei != kPad && Ei != kNever && Ei < 0 && tI < T;
        if (!__any_sync(0xffffffffu, seed)) continue;
        const int g = gr.tile_graph ? (int)gr.tile_graph[tile] : 0;
        const int32_t *sg = sig + (size_t)g * ld_sig;
        // gx(0), needed when day 0 lies between the two exits
        const bool at0 = seed && -Ei >= Lmin && -Ei < L;
        float sum[1];
        row_sums<1>(m, m.slice_ptr[tile], m.row_len[row], at0, lane, contrib, want, sum);
        double pm = 0.0;
        if (seed) {
            const size_t pg = (size_t)g * f.ldP;
            double H = (Ei + f.L_M >= 0 && Ei + f.L_M < T) ? gD[pg + Ei + f.L_M] : 0.0;
            for (int k = Lmin; k < L; ++k) {
                const int d = Ei + k;
                if (d < 0 || d >= T) continue;
                const float gxs = d == 0 ? sum[0] : ring[(size_t)(d % Lm1) * ring_stride + row];
                H += sgn * (double)c[k] * ldexp((double)gxs, sg[d]);
            }
            const float vf = fate_uniform(f, caller_id(gr, row, g), tI, g);
            const double mI = (double)f.mort[pg + tI], v = (double)vf;
            const double den = mI * (1.0 - v) + (1.0 - mI) * v;
            pm = H * (v * (1.0 - v) / (den * den));
        }
        for (int d = 0; d < f.tau_EI && d < T; ++d) {
            double x = (seed && tI == d) ? pm : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0 && x != 0.0) Pm[(size_t)d * ntiles + tile] = x;
        }
    }
}

// dm[g][t] = sum over the graph's tiles of Pm[t][tile] (fixed order, FP64).
__global__ void __launch_bounds__(256) k_fate_dm(const double *Pm, int ntiles, const int32_t *graph_tile0,
                                                 const int32_t *graph_ntiles, int T, double *dm) {
    __shared__ double s[256];
    const int t = blockIdx.x, g = blockIdx.y;
    const int tile0 = graph_tile0[g], nt = graph_ntiles[g];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) acc += Pm[(size_t)t * ntiles + tile0 + i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) dm[(size_t)g * T + t] = s[0];
}

// dc[g][k] = sum over the graph's tiles of dc_tile[tile][k] (fixed order, FP64), k < L.
__global__ void __launch_bounds__(256) k_dc_reduce(const double *dc_tile, const int32_t *graph_tile0,
                                                   const int32_t *graph_ntiles, int L, double *dc) {
    __shared__ double s[256];
    const int g = blockIdx.x, k = blockIdx.y;
    const int tile0 = graph_tile0[g], nt = graph_ntiles[g];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) acc += dc_tile[(size_t)(tile0 + i) * kMaxL + k];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) dc[(size_t)g * L + k] = s[0];
}

// Q[inst][t][a] = sum over the graph's tiles of P[t][tile][a], fixed order, FP64.
__global__ void __launch_bounds__(256) k_bwd_reduce(const double *P, int ntiles, const int32_t *graph_tile0,
                                                    const int32_t *graph_ntiles, int T, const int32_t *sig,
                                                    int ld_sig, double *Q) {
    __shared__ double s[256][kAges];
    const int t = blockIdx.x, inst = blockIdx.y;
    const int g = inst;
    const int tile0 = graph_tile0[g], nt = graph_ntiles[g];
    double acc[kAges];
#pragma unroll
    for (int b = 0; b < kAges; ++b) acc[b] = 0.0;
    const double *Pt = P + (size_t)t * ntiles * kAges;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        const double *p = Pt + (size_t)(tile0 + i) * kAges;
#pragma unroll
        for (int b = 0; b < kAges; ++b) acc[b] += p[b];
    }
#pragma unroll
    for (int b = 0; b < kAges; ++b) s[threadIdx.x][b] = acc[b];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int b = 0; b < kAges; ++b) s[threadIdx.x][b] += s[threadIdx.x + h][b];
        __syncthreads();
    }
    if (threadIdx.x < kAges)
        Q[((size_t)inst * T + t) * kAges + threadIdx.x] = ldexp(s[0][threadIdx.x], sig[(size_t)g * ld_sig + t]);
}

// dR_t = sum_a S_a Q[t][a];  dS_a = sum_t R_t Q[t][a];  dm_t = gD_t newRM(t) (not written
// when both counts are NULL: the sampled R/M split's dm comes from k_fate_dm).
__global__ void __launch_bounds__(256) k_bwd_finalize(const double *Q, const float *R, const float *S,
                                                      const double *gD, const int32_t *newRM,
                                                      const double *newRM_real, int ldP, int T, double *dR,
                                                      double *dm, double *dS) {
    const int inst = blockIdx.x;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const double *q = Q + ((size_t)inst * T + t) * kAges;
        double acc = 0.0;
        for (int b = 0; b < kAges; ++b) acc += (double)S[inst * kAges + b] * q[b];
        dR[(size_t)inst * T + t] = acc;
        const size_t pi = (size_t)inst * ldP + t;
        if (newRM_real || newRM) dm[(size_t)inst * T + t] = gD[pi] * (newRM_real ? newRM_real[pi] : (double)newRM[pi]);
    }
    if (threadIdx.x < kAges) {
        const int b = threadIdx.x;
        double acc = 0.0;
        for (int t = 0; t < T; ++t) acc += (double)R[(size_t)inst * ldP + t] * Q[((size_t)inst * T + t) * kAges + b];
        dS[inst * kAges + b] = acc;
    }
}

}  // namespace

cudaError_t launch_bwd_day(const BwdDayArgs &a, int grid, cudaStream_t s) {
    const bool dc = a.dc_tile != nullptr;
    if (a.fate.L_M > 0 || a.dur.n > 0) {   // store policy, plain instance only (checked at creation)
        if (a.mode != kBwdStore || dc) return cudaErrorInvalidValue;
        if (a.fate.L_M > 0) k_bwd_day<kBwdStore, false, kExitFate><<<grid, kBlock, 0, s>>>(a);
        else k_bwd_day<kBwdStore, false, kExitDur><<<grid, kBlock, 0, s>>>(a);
        return cudaGetLastError();
    }
    switch (a.mode) {
        case kBwdStore:
            if (dc) k_bwd_day<kBwdStore, true><<<grid, kBlock, 0, s>>>(a);
            else k_bwd_day<kBwdStore, false><<<grid, kBlock, 0, s>>>(a);
            break;
        case kBwdFused:
            if (dc) k_bwd_day<kBwdFused, true><<<grid, kBlock, 0, s>>>(a);
            else k_bwd_day<kBwdFused, false><<<grid, kBlock, 0, s>>>(a);
            break;
        case kBwdSoft:
            if (dc) k_bwd_day<kBwdSoft, true><<<grid, kBlock, 0, s>>>(a);
            else k_bwd_day<kBwdSoft, false><<<grid, kBlock, 0, s>>>(a);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_dc_seeds(Sell m_out, const int16_t *E, const float *r0, GraphRef gr, const int32_t *sig,
                            int ld_sig, int ntiles, int L, double *dc_tile, int grid, cudaStream_t s) {
    k_dc_seeds<<<grid, kBlock, 0, s>>>(m_out, E, r0, gr, sig, ld_sig, ntiles, L, dc_tile);
    return cudaGetLastError();
}

cudaError_t launch_fate_seeds(Sell m_out, const int16_t *E, const float *r0, const float *ring, size_t ring_stride,
                              int Lm1, GraphRef gr, FateRef f, const double *gD, const int32_t *sig, int ld_sig,
                              int ntiles, int T, const float *c, double *Pm, int grid, cudaStream_t s) {
    k_fate_seeds<<<grid, kBlock, 0, s>>>(m_out, E, r0, ring, ring_stride, Lm1, gr, f, gD, sig, ld_sig, ntiles, T, c, Pm);
    return cudaGetLastError();
}

cudaError_t launch_fate_dm(const double *Pm, int ntiles, const int32_t *graph_tile0, const int32_t *graph_ntiles,
                           int G, int T, double *dm, cudaStream_t s) {
    if (T > 0) k_fate_dm<<<dim3(T, G), 256, 0, s>>>(Pm, ntiles, graph_tile0, graph_ntiles, T, dm);
    return cudaGetLastError();
}

cudaError_t launch_dc_reduce(const double *dc_tile, const int32_t *graph_tile0, const int32_t *graph_ntiles, int G,
                             int L, double *dc, cudaStream_t s) {
    k_dc_reduce<<<dim3(G, L), 256, 0, s>>>(dc_tile, graph_tile0, graph_ntiles, L, dc);
    return cudaGetLastError();
}

cudaError_t launch_lam_day(Sell m, const int16_t *E, const uint32_t *bits, GraphRef gr, int t, int L, int ntiles,
                           const float *c, float *lam_out, int grid, cudaStream_t s) {
    k_lam_day<<<grid, kBlock, 0, s>>>(m, E, bits, gr, t, L, ntiles, c, lam_out);
    return cudaGetLastError();
}

int occupancy_bwd(int mode, bool dc, int exit_mode) {
    int blocks = 0;
    if (exit_mode != kExitBase) {
        if (exit_mode == kExitFate)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day<kBwdStore, false, kExitFate>, kBlock, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day<kBwdStore, false, kExitDur>, kBlock, 0);
        return blocks > 0 ? blocks : 1;
    }
    switch (mode) {
        case kBwdFused:
            if (dc) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day<kBwdFused, true>, kBlock, 0);
            else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day<kBwdFused, false>, kBlock, 0);
            break;
        case kBwdSoft:
            if (dc) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day<kBwdSoft, true>, kBlock, 0);
            else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day<kBwdSoft, false>, kBlock, 0);
            break;
        default:
            if (dc) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day<kBwdStore, true>, kBlock, 0);
            else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day<kBwdStore, false>, kBlock, 0);
            break;
    }
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_bwd_reduce(const double *P, int ntiles, int ldP, const int32_t *graph_tile0,
                              const int32_t *graph_ntiles, int T, int I, const int32_t *sig, int ld_sig,
                              double *Q, cudaStream_t s) {
    (void)ldP;
    k_bwd_reduce<<<dim3(T, I), 256, 0, s>>>(P, ntiles, graph_tile0, graph_ntiles, T, sig, ld_sig, Q);
    return cudaGetLastError();
}

cudaError_t launch_bwd_finalize(const double *Q, const float *R, const float *S, const double *gD,
                                const int32_t *newRM, const double *newRM_real, int ldP, int T, int I, double *dR,
                                double *dm, double *dS, cudaStream_t s) {
    k_bwd_finalize<<<I, 256, 0, s>>>(Q, R, S, gD, newRM, newRM_real, ldP, T, dR, dm, dS);
    return cudaGetLastError();
}

}  // namespace gabm
