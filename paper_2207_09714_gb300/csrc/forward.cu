// forward.cu -- forward day step of the hard GradABM model on sm_103a.
//
// One launch per day (Sec. 3.1, Eq. 1-3; A1: one-day steps).  Each block takes
// a contiguous range of 32-row tiles, its warps one tile at a time (neighbours
// stay in the SM's L1 this way); each lane sums its own susceptible
// row over the in-edges (a pull gather, no atomics) read from the tile's
// SELL-32 slice with coalesced loads: w_ji * c[t - e_j] for the neighbours
// marked infectious in today's bitmap (an L1-resident bit array), whose
// exposure days are gathered from the L2-resident state.  Each warp prefetches
// the next tile's id, row data and (into L2) its slice while it works on the
// current tile.  Each lane then runs the fused epilogue for its own
// row: lambda, p = 1 - exp(-lambda) (Eq. 3), the Philox uniform, the hard draw
// and the in-place state update e_i = t.
//
// The in-place update is race-free in effect: a neighbour that reads e_i
// during the same day sees either NEVER or t, and both give c = 0 (c[0] = 0 by
// assumption A2 of App. A), so every lambda uses the start-of-day state.
#include "gabm_internal.cuh"
#include "rowsum.cuh"

// The share (percent) of a graph's agents in E or I on the previous day from which the
// one-set forward gathers every entry's exposure day instead of testing the day's bitmap.
#ifndef GABM_DENSE_MARKS_PCT
#define GABM_DENSE_MARKS_PCT 25
#endif

namespace gabm {

namespace {

__device__ __forceinline__ void flush_counts_warp(int32_t *counts, int32_t *newRM, int ldP, int g,
                                                  int t, int cS, int cE, int cI, int cR, int cN,
                                                  int lane) {
    cS = __reduce_add_sync(0xffffffffu, cS);
    cE = __reduce_add_sync(0xffffffffu, cE);
    cI = __reduce_add_sync(0xffffffffu, cI);
    cR = __reduce_add_sync(0xffffffffu, cR);
    cN = __reduce_add_sync(0xffffffffu, cN);
    if (lane == 0) {
        int32_t *cp = counts + ((size_t)g * ldP + t) * 4;
        if (cS) atomicAdd(cp + 0, cS);
        if (cE) atomicAdd(cp + 1, cE);
        if (cI) atomicAdd(cp + 2, cI);
        if (cR) atomicAdd(cp + 3, cR);
        if (cN) atomicAdd(newRM + (size_t)g * ldP + t, cN);
    }
}

// SMEM_BITS: today's infectious bitmap is copied into shared memory (one large
// block per SM), so the per-edge test is a shared-memory lookup instead of a
// scattered L1 load; otherwise it is read through L1 from global memory.
// PULL (agent-location graphs): the row's entries are the agent's locations, and each
// contributes w_il * P_l from the day's location pressures (a.pull) instead of a marked
// neighbour's infectiousness.
// EXIT = kExitFate (sampled R/M split): a row's exit from I is L_R or L_M after exposure by
// its fate, drawn again where needed (the day before the earlier exit through the later
// one), and the deaths counted are the M entries.  EXIT = kExitDur (stochastic I-stage
// durations): the exit is the row's drawn L_i (drawn again from its first possible day
// on); deaths stay m_t newRM(t).
template <bool SMEM_BITS, int NT, int MINB, bool PULL = false, int EXIT = kExitBase>
__global__ void __launch_bounds__(NT, MINB) k_fwd_day(const FwdDayArgs a) {
    constexpr int NW = NT / 32;
    extern __shared__ uint32_t bits_s[];
    constexpr bool FATE = EXIT == kExitFate;
    __shared__ float c_s[kMaxL];
    __shared__ double F_s[kMaxL];
    __shared__ int32_t red_s[NW][6];
    if (threadIdx.x < kMaxL) c_s[threadIdx.x] = a.c[threadIdx.x];
    if (EXIT == kExitDur && threadIdx.x < kMaxL) F_s[threadIdx.x] = a.dur.F[threadIdx.x];
    if (SMEM_BITS)
        for (int i = threadIdx.x; i < a.ntiles; i += NT) bits_s[i] = __ldcg(a.bits_cur + i);
    __syncthreads();

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int t = a.t, L = a.L, tau_EI = a.tau_EI, ntiles = a.ntiles;
    const int16_t *e = a.e;
    const uint32_t *bits = a.bits_cur;
    // Only neighbours infectious today contribute; their exposure day is gathered.  While
    // few rows are infectious the day's bitmap spares the gathers of the others; once many
    // are (use_bits false, base model only), every entry's exposure day is gathered and
    // tested directly, which selects the same entries (an exposure during the day gives
    // c[0] = 0) at one scattered load per entry instead of two.
    bool use_bits = true;
    auto contrib = [&](uint32_t j, float w, bool valid, float (&out)[1], bool (&take)[1]) {
        if constexpr (PULL) {
            out[0] = w * ld_if(a.pull + j, valid);
            take[0] = valid;
        } else {
            const bool pre = valid && (!use_bits || (SMEM_BITS ? ((bits_s[j >> 5] >> (j & 31u)) & 1u) : marked(bits, j)));
            const int ej = ld_if(e + j, pre, kNever);
            const int k = t - ej;
            const bool mk = pre && (unsigned)(k - 1) < (unsigned)(L - 1);
            out[0] = mk ? w * c_s[k] : 0.f;
            take[0] = mk;
        }
    };
    const bool want[1] = {true};

    int cur_g = -1;
    int cS = 0, cE = 0, cI = 0, cR = 0, cN = 0;

    // Tiles come from the block's contiguous range; each tile's row data is loaded one
    // tile ahead of use (and, when enabled, its slice prefetched into L2).
    BlockTiles disp;
    disp.init(ntiles, lane);
    const uint8_t *flags = PULL ? nullptr : a.flag_cur;
    TileRows cur, nxt;
    load_tile_rows(a.m, e, a.gr.tile_graph, ntiles, disp.get(), lane, cur, flags);
    load_tile_rows(a.m, e, a.gr.tile_graph, ntiles, disp.get(), lane, nxt, flags);
    prefetch_slice(a.m, cur.p0, cur.p1, lane);
    while (cur.tile < ntiles) {
        prefetch_slice(a.m, nxt.p0, nxt.p1, lane);
        TileRows nn;
        load_tile_rows(a.m, e, a.gr.tile_graph, ntiles, disp.get(), lane, nn, flags);

        const int g = cur.g, tile = cur.tile, ei = cur.e;
        if (g != cur_g) {
            if (cur_g >= 0) flush_counts_warp(a.counts, a.newRM, a.ldP, cur_g, t, cS, cE, cI, cR, cN, lane);
            cur_g = g;
            cS = cE = cI = cR = cN = 0;
            if (!PULL && EXIT == kExitBase && t > a.t_first) {   // the graph's E + I share yesterday
                const int32_t *cp = a.counts + ((size_t)g * a.ldP + t - 1) * 4;
                const int32_t ei_cnt = cp[1] + cp[2], all = cp[0] + cp[1] + cp[2] + cp[3];
                use_bits = (int64_t)ei_cnt * 100 < (int64_t)GABM_DENSE_MARKS_PCT * all;
            }
        }
        const int row = tile * kTile + lane;
        const bool isS = (ei == kNever);
        int Lx = L;   // this row's exit from I
        if constexpr (FATE) {
            const int k = t - ei;
            bool phi = false;
            if (ei != kPad && !isS && k + 1 >= min(a.fate.L_R, a.fate.L_M) && k <= L)
                phi = fate_M(a.fate, caller_id(a.gr, row, g), ei, g, t + 1);
            Lx = phi ? a.fate.L_M : a.fate.L_R;
            if (ei != kPad && !isS) cN += (phi && k == a.fate.L_M);
        }
        if constexpr (EXIT == kExitDur) {
            const int k = t - ei;
            if (ei != kPad && !isS && k >= tau_EI && k <= L) Lx = dur_exit(a.dur, F_s, caller_id(a.gr, row, g), ei, g);
        }
        if (ei != kPad && !isS) {
            const int k = t - ei;
            if (k < tau_EI) ++cE; else if (k < Lx) ++cI; else ++cR;
            if (!FATE) cN += (k == Lx);
        }
        cS += isS;

        // A susceptible row with no infectious in-neighbour has lambda = 0 exactly (no
        // marked entry): it reads no entries and does not draw (u < p = 0 is false).
        const bool act = isS && cur.flag;
        // the draw's row loads go out before the sums, so that their latency overlaps them
        const int age_ld = act ? (int)a.age[row] : 0;
        const uint32_t id_ld = act ? caller_id(a.gr, row, g) : 0u;
        float sum[1];
        const unsigned amask = __ballot_sync(0xffffffffu, act);
        if (flags && __popc(amask) <= GABM_COOP_ROWS) {   // few summing rows: warp-wide, together
            float cs = 0.f;
            sum[0] = 0.f;
            if (amask) few_row_sums(a.m, cur.p0, cur.len, amask, lane, contrib, sum[0], cs);
        } else {
            row_sums<1>(a.m, cur.p0, cur.len, act, lane, contrib, want, sum);
        }

        int e_next = ei;
        if (act) {
            const float Lam = sum[0] * a.gr.inv_Dbar[g];
            const int inst = g;
            const float lam = (a.R[(size_t)inst * a.ldP + t] * a.S[inst * kAges + age_ld]) * Lam;
            const float p = -expm1f(-lam);
            const uint32_t id = id_ld;
            const float u = uniform_from_word(philox_word(a.seed, id, (uint32_t)t, (uint32_t)inst, 0u));
            if (u < p) {
                a.e[row] = (int16_t)t;
                e_next = t;
            }
            if (a.lam_out) a.lam_out[row] = Lam;
        } else if (isS && a.lam_out) {
            a.lam_out[row] = 0.f;
        }
        // rows infectious tomorrow (susceptible and padding rows fall outside the window)
        const int kn = t + 1 - e_next;
        const bool inf = (unsigned)(kn - 1) < (unsigned)(Lx - 1);
        const unsigned inf_next = __ballot_sync(0xffffffffu, inf);
        if (lane == 0) a.bits_next[tile] = inf_next;
        if (!PULL && flags) {   // tomorrow's flags: the out-neighbours of tomorrow's infectious rows
            push_flags(a.m_out, tile, lane, inf, a.flag_next);
            a.flag_clear[row] = 0;
        }

        cur = nxt;
        nxt = nn;
    }

    // block-level reduction of the last graph's counts, then one atomic per count
    cS = __reduce_add_sync(0xffffffffu, cS);
    cE = __reduce_add_sync(0xffffffffu, cE);
    cI = __reduce_add_sync(0xffffffffu, cI);
    cR = __reduce_add_sync(0xffffffffu, cR);
    cN = __reduce_add_sync(0xffffffffu, cN);
    if (lane == 0) {
        red_s[wib][0] = cur_g;
        red_s[wib][1] = cS; red_s[wib][2] = cE; red_s[wib][3] = cI; red_s[wib][4] = cR; red_s[wib][5] = cN;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int g = -1;
        int32_t acc[5] = {0, 0, 0, 0, 0};
        for (int w = 0; w <= NW; ++w) {
            const int gw = (w < NW) ? red_s[w][0] : -2;
            if (gw != g) {
                if (g >= 0) {
                    int32_t *cp = a.counts + ((size_t)g * a.ldP + t) * 4;
                    for (int s2 = 0; s2 < 4; ++s2) if (acc[s2]) atomicAdd(cp + s2, acc[s2]);
                    if (acc[4]) atomicAdd(a.newRM + (size_t)g * a.ldP + t, acc[4]);
                }
                g = gw;
                for (int s2 = 0; s2 < 5; ++s2) acc[s2] = 0;
            }
            if (w < NW && gw >= 0)
                for (int s2 = 0; s2 < 5; ++s2) acc[s2] += red_s[w][1 + s2];
        }
    }
}

// ---------------------------------------------------------------------------
// Fixed-noise soft relaxation (the smooth model whose gradient the
// straight-through estimator stands in for; used for finite-difference checks):
// every agent draws every day with y = sigmoid(logit p - logit u) (Gumbel-softmax,
// tau = 1, the same u as the hard draw), moving mass n = s y from S to E:
//   s_i(t+1) = s_i(t) - n_i(t),  x_i(t) = sum_{k=1}^{L-1} c[k] n_i(t-k),
//   newRM(t) = sum_i n_i(t-L),  D_t = m_t newRM(t).
// ---------------------------------------------------------------------------
__global__ void k_soft_init(const int16_t *e, int64_t n_rows, int L, const float *c, float *s, float *nh,
                            float *x_cur) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int ei = e[r];
        const bool seedr = (ei != kNever) && (ei != kPad);   // exposed before day 0 (e in [-L, -1])
        s[r] = (ei == kNever) ? 1.f : 0.f;
        float x = 0.f;
        for (int k = 0; k < L; ++k) {
            // slot k holds day d with d mod L == k, d in [-L, -1]
            const int d = k - L;
            const float v = (seedr && ei == d) ? 1.f : 0.f;
            nh[(size_t)k * n_rows + r] = v;
        }
        if (seedr && -ei >= 1 && -ei < L) x = c[-ei];
        x_cur[r] = x;
    }
}

__global__ void __launch_bounds__(kBlock, GABM_MINBLOCKS) k_fwd_day_soft(const SoftDayArgs a) {
    __shared__ float c_s[kMaxL];
    if (threadIdx.x < kMaxL) c_s[threadIdx.x] = a.c[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int t = a.t, L = a.L, ntiles = a.ntiles;
    const float *__restrict__ x_cur = a.x_cur;
    auto contrib = [&](uint32_t j, float w, bool valid, float (&out)[1], bool (&take)[1]) {
        out[0] = w * ld_if(x_cur + j, valid);
        take[0] = valid;
    };
    const bool want[1] = {true};
    const size_t n_rows = (size_t)ntiles * kTile;
    const int slot_t = t % L;   // holds n(t - L) before this launch overwrites it with n(t)
    BlockTiles disp;
    disp.init(ntiles, lane);
    for (int tile = disp.get(); tile < ntiles; tile = disp.get()) {
        const int row = tile * kTile + lane;
        const int ei = a.e[row];
        const bool agent = ei != kPad;
        const int g = a.gr.tile_graph ? (int)a.gr.tile_graph[tile] : 0;
        float sum[1];
        row_sums<1>(a.m, a.m.slice_ptr[tile], a.m.row_len[row], agent, lane, contrib, want, sum);
        float n_old = 0.f;
        if (agent) {
            const float Lam = sum[0] * a.gr.inv_Dbar[g];
            const float lam = (a.R[(size_t)g * a.ldP + t] * a.S[g * kAges + a.age[row]]) * Lam;
            const float q = expf(-lam);
            const float p = -expm1f(-lam);
            const uint32_t id = caller_id(a.gr, row, g);
            const float u = uniform_from_word(philox_word(a.seed, id, (uint32_t)t, (uint32_t)g, 0u));
            const float num = p * (1.f - u);
            const float y = num / __fmaf_rn(q, u, num);
            const float s_old = a.s[row];
            const float n = s_old * y;
            a.s[row] = s_old - n;
            n_old = a.nh[(size_t)slot_t * n_rows + row];
            a.nh[(size_t)slot_t * n_rows + row] = n;
            // x(t+1) = c[1] n(t) + sum_{k=2}^{L-1} c[k] n(t+1-k)
            float x = c_s[1] * n;
            for (int k = 2; k < L; ++k) x = __fmaf_rn(c_s[k], a.nh[(size_t)((t + 1 - k + L) % L) * n_rows + row], x);
            a.x_next[row] = x;
            a.s_hist_t[row] = s_old;
            a.y_hist_t[row] = y;
            a.lam_t[row] = Lam;
        } else {
            a.x_next[row] = 0.f;
        }
        float v = n_old;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) a.P_nrm_t[tile] = (double)v;
    }
}

// newRM_real[g][t] = sum over graph g's tiles of P_nrm[t][tile] (fixed order, FP64);
// D = m newRM in FP64, copied out when D_out is given ([G][T]).
__global__ void __launch_bounds__(256) k_soft_finalize(const double *P_nrm, int ntiles, const int32_t *tile0,
                                                       const int32_t *ntl, const float *m, int ldP, int T,
                                                       double *newRM_real, double *D_ctx, double *D_out) {
    __shared__ double sh[256];
    const int t = blockIdx.x, g = blockIdx.y;
    double acc = 0.0;
    const double *p = P_nrm + (size_t)t * ntiles + tile0[g];
    for (int i = threadIdx.x; i < ntl[g]; i += blockDim.x) acc += p[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const size_t pi = (size_t)g * ldP + t;
        newRM_real[pi] = sh[0];
        const double d = (double)m[pi] * sh[0];
        D_ctx[pi] = d;
        if (D_out) D_out[(size_t)g * T + t] = d;
    }
}

// One warp per tile: for every day d of the range, the ballot of rows with
// 1 <= d - e < L.
__global__ void k_infectious_bits_dur(const int16_t *e, GraphRef gr, const DurRef d, int t, int ntiles, uint32_t *bits) {
    __shared__ double F_s[kMaxL];
    if (threadIdx.x < kMaxL) F_s[threadIdx.x] = d.F[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int L = d.tau_EI + d.n;
    for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < ntiles; tile += warps) {
        const int row = tile * kTile + lane;
        const int ei = e[row];
        const int k = t - ei;
        int Lx = L;
        if (ei != kPad && ei != kNever && k > d.tau_EI && k < L) {
            const int g = gr.tile_graph ? (int)gr.tile_graph[tile] : 0;
            Lx = dur_exit(d, F_s, caller_id(gr, row, g), ei, g);
        }
        const unsigned b = __ballot_sync(0xffffffffu, (unsigned)(k - 1) < (unsigned)(Lx - 1));
        if (lane == 0) bits[tile] = b;
    }
}

__global__ void k_infectious_bits_fate(const int16_t *e, GraphRef gr, FateRef f, int t, int ntiles, uint32_t *bits) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < ntiles; tile += warps) {
        const int row = tile * kTile + lane;
        const int ei = e[row];
        const int k = t - ei;
        int Lx = f.L_R;
        if (ei != kPad && ei != kNever && k >= min(f.L_R, f.L_M) && k < max(f.L_R, f.L_M)) {
            const int g = gr.tile_graph ? (int)gr.tile_graph[tile] : 0;
            Lx = fate_M(f, caller_id(gr, row, g), ei, g, t + 1) ? f.L_M : f.L_R;
        }
        const unsigned b = __ballot_sync(0xffffffffu, (unsigned)(k - 1) < (unsigned)(Lx - 1));
        if (lane == 0) bits[tile] = b;
    }
}

__global__ void k_infectious_bits(const int16_t *e, int t0, int ndays, int L, int ntiles, uint32_t *bits,
                                  size_t day_stride) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < ntiles; tile += warps) {
        const int ei = e[tile * kTile + lane];
        for (int d = 0; d < ndays; ++d) {
            const int k = t0 + d - ei;
            const unsigned b = __ballot_sync(0xffffffffu, (unsigned)(k - 1) < (unsigned)(L - 1));
            if (lane == 0) bits[(size_t)d * day_stride + tile] = b;
        }
    }
}

// ---------------------------------------------------------------------------
// State initialisation and seeding (initial infections i^0, Sec. 3.1):
// the n_seed agents of each instance with the smallest 64-bit key
// (Philox word at (id, 0, inst, 1) << 32 | id).  Exact radix select on the
// 32-bit word in three digits (11, 11, 10 bits), then ties on the final word
// are broken by id.
// ---------------------------------------------------------------------------
__global__ void k_init_state(int16_t *e, const int32_t *row0, const int32_t *rows, int G, int64_t n_rows,
                             int B, int Bp) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        // binary search the graph of row r
        int lo = 0, hi = G - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (row0[mid] <= r) lo = mid; else hi = mid - 1;
        }
        const bool agent = r - row0[lo] < rows[lo];
        for (int b = 0; b < Bp; ++b)
            e[(size_t)r * Bp + b] = (agent && b < B) ? (int16_t)kNever : (int16_t)kPad;
    }
}

__global__ void k_seed_reset(SeedState *st, const int32_t *n_seed, int I) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    SeedState s;
    s.prefix = 0u;
    s.k_rem = (uint32_t)n_seed[i];
    s.eq_count = 0u;
    s.tie_n = 0u;
    s.none = (n_seed[i] == 0);
    s.overflow = 0;
    st[i] = s;
}

__device__ __forceinline__ void digit_of_pass(int pass, int &shift, int &nbins, uint32_t &himask) {
    if (pass == 0) { shift = 21; nbins = 2048; himask = 0u; }
    else if (pass == 1) { shift = 10; nbins = 2048; himask = 0xFFE00000u; }
    else { shift = 0; nbins = 1024; himask = 0xFFFFFC00u; }
}

__global__ void __launch_bounds__(256) k_seed_hist(const SeedArgs a) {
    __shared__ uint32_t h_s[kHistBins];
    const int inst = blockIdx.y;
    const SeedState st = a.st[inst];
    if (st.none) return;
    int shift, nbins; uint32_t himask;
    digit_of_pass(a.pass, shift, nbins, himask);
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) h_s[b] = 0u;
    __syncthreads();
    const int g = inst / a.B;
    const int32_t r0 = a.row0[g], nr = a.rows[g];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
        const uint32_t id = a.orig_id ? a.orig_id[r0 + i] : (uint32_t)i;
        const uint32_t h = philox_word(a.seed, id, 0u, (uint32_t)inst, 1u);
        if ((h & himask) == st.prefix) atomicAdd(&h_s[(h >> shift) & (nbins - 1)], 1u);
    }
    __syncthreads();
    uint32_t *gh = a.hist + (size_t)inst * kHistBins;
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (h_s[b]) atomicAdd(gh + b, h_s[b]);
}

// One warp per instance: find the digit bin holding the k_rem-th smallest key.
__global__ void k_seed_scan(const SeedArgs a) {
    const int inst = blockIdx.x;
    const int lane = threadIdx.x;
    SeedState st = a.st[inst];
    int shift, nbins; uint32_t himask;
    digit_of_pass(a.pass, shift, nbins, himask);
    uint32_t *gh = a.hist + (size_t)inst * kHistBins;
    if (!st.none) {
        const int per = nbins / 32;
        uint32_t mine = 0;
        for (int b = 0; b < per; ++b) mine += gh[lane * per + b];
        uint32_t incl = mine;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t excl = incl - mine;
        const bool here = (excl < st.k_rem) && (st.k_rem <= incl);
        const unsigned who = __ballot_sync(0xffffffffu, here);
        const int src = __ffs(who) - 1;
        uint32_t digit = 0, below = 0, eq = 0;
        if (lane == src) {
            uint32_t cum = excl;
            for (int b = 0; b < per; ++b) {
                const uint32_t hb = gh[lane * per + b];
                if (st.k_rem <= cum + hb) { digit = (uint32_t)(lane * per + b); below = cum; eq = hb; break; }
                cum += hb;
            }
        }
        digit = __shfl_sync(0xffffffffu, digit, src);
        below = __shfl_sync(0xffffffffu, below, src);
        eq = __shfl_sync(0xffffffffu, eq, src);
        __syncwarp();
        if (lane == 0) {
            st.prefix |= digit << shift;
            st.k_rem -= below;
            if (a.pass == 2) st.eq_count = eq;
            a.st[inst] = st;
        }
    }
    for (int b = lane; b < nbins; b += 32) gh[b] = 0u;
}

__global__ void k_seed_mark(const SeedArgs a) {
    const int inst = blockIdx.y;
    const SeedState st = a.st[inst];
    if (st.none) return;
    const int g = inst / a.B;
    const size_t set = (size_t)(inst - g * a.B);
    const int32_t r0 = a.row0[g], nr = a.rows[g];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
        const uint32_t id = a.orig_id ? a.orig_id[r0 + i] : (uint32_t)i;
        const uint32_t h = philox_word(a.seed, id, 0u, (uint32_t)inst, 1u);
        bool mark = h < st.prefix;
        if (h == st.prefix) {
            if (st.eq_count == st.k_rem) {
                mark = true;
            } else {
                const uint32_t slot = atomicAdd(&a.st[inst].tie_n, 1u);
                if (slot < (uint32_t)kTieCap) a.ties[(size_t)inst * kTieCap + slot] = (uint32_t)i;
                else a.st[inst].overflow = 1;
            }
        }
        if (mark) a.e[(size_t)(r0 + i) * a.Bp + set] = (int16_t)(-a.tau_EI);
    }
}

// Ties on the threshold word: the k_rem candidates with the smallest caller ids win.
// The tie list holds local row indices.
__global__ void k_seed_ties(const SeedArgs a) {
    const int inst = blockIdx.x;
    const SeedState st = a.st[inst];
    if (st.none || st.eq_count == st.k_rem) return;
    const uint32_t n = min(st.tie_n, (uint32_t)kTieCap);
    const uint32_t *tl = a.ties + (size_t)inst * kTieCap;
    const int g = inst / a.B;
    const size_t set = (size_t)(inst - g * a.B);
    const int32_t r0 = a.row0[g];
    for (uint32_t c = threadIdx.x; c < n; c += blockDim.x) {
        const uint32_t i = tl[c];
        const uint32_t id = a.orig_id ? a.orig_id[r0 + i] : i;
        uint32_t rank = 0;
        for (uint32_t d = 0; d < n; ++d) {
            const uint32_t idd = a.orig_id ? a.orig_id[r0 + tl[d]] : tl[d];
            rank += (idd < id);
        }
        if (rank < st.k_rem) a.e[(size_t)(r0 + i) * a.Bp + set] = (int16_t)(-a.tau_EI);
    }
}

// Row order <-> caller order.
__device__ __forceinline__ bool caller_slot(const GraphRef &gr, const int32_t *rows, const int64_t *goff,
                                            int64_t r, int64_t &slot) {
    const int g = gr.tile_graph ? (int)gr.tile_graph[r / kTile] : 0;
    const int64_t i = r - gr.row0[g];
    if (i >= rows[g]) return false;
    slot = goff[g] + (int64_t)(gr.orig_id ? gr.orig_id[r] : (uint32_t)i);
    return true;
}

template <typename T>
__global__ void k_rows_to_caller(const T *src, T *dst, GraphRef gr, const int32_t *rows, const int64_t *goff,
                                 int64_t n_rows, SetLayout sl) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t slot;
        if (caller_slot(gr, rows, goff, r, slot))
            for (int b = 0; b < sl.B; ++b) dst[(size_t)b * sl.n_total + slot] = src[(size_t)r * sl.Bp + b];
    }
}

template <typename T>
__global__ void k_caller_to_rows(const T *src, T *dst, GraphRef gr, const int32_t *rows, const int64_t *goff,
                                 int64_t n_rows, SetLayout sl) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t slot;
        if (caller_slot(gr, rows, goff, r, slot))
            for (int b = 0; b < sl.B; ++b) dst[(size_t)r * sl.Bp + b] = src[(size_t)b * sl.n_total + slot];
    }
}

// D_t = m_t * newRM(t) in FP64 (Aggregate, Sec. 3.1), or the counted M entries when m is
// NULL (sampled R/M split); copies counts out.
__global__ void k_fwd_finalize(const int32_t *newRM, const int32_t *counts, const float *m, int ldP,
                               int t0, int T, int I, double *D_ctx, double *D_out, int32_t *counts_out) {
    const int total = I * T;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int inst = idx / T, t = idx - inst * T;
        if (t < t0) continue;
        const size_t src = (size_t)inst * ldP + t;
        const double d = m ? (double)m[src] * (double)newRM[src] : (double)newRM[src];
        D_ctx[src] = d;
        if (D_out) D_out[idx] = d;
        if (counts_out)
            for (int s = 0; s < 4; ++s) counts_out[(size_t)idx * 4 + s] = counts[src * 4 + s];
    }
}

// MSE on daily deaths (Sec. 3.2, Stage 3); one block per instance, fixed-order FP64 sums.
__global__ void __launch_bounds__(256) k_mse(const double *D, int ldP, const double *y, int T,
                                             double *loss, double *gD_ctx, double *gD_out) {
    __shared__ double s_acc[256];
    const int inst = blockIdx.x;
    double acc = 0.0;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const double d = D[(size_t)inst * ldP + t] - y[(size_t)inst * T + t];
        const double g = 2.0 * d / (double)T;
        gD_ctx[(size_t)inst * ldP + t] = g;
        if (gD_out) gD_out[(size_t)inst * T + t] = g;
        acc += d * d;
    }
    s_acc[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) s_acc[threadIdx.x] += s_acc[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) loss[inst] = s_acc[0] / (double)T;
}

// lambda_i(t) = R_t S[a_i] Lam_i(t) for agents susceptible on day t, else 0.
__global__ void k_get_lambda(const float *lam_t, const int16_t *e, const uint8_t *age, GraphRef gr,
                             const float *R, const float *S, int ldP, int t, int64_t n_rows, int B, int Bp,
                             float *out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int g = gr.tile_graph ? (int)gr.tile_graph[r / kTile] : 0;
        for (int b = 0; b < Bp; ++b) {
            const size_t x = (size_t)r * Bp + b;
            const int ei = e[x];
            const bool wasS = (ei == kNever) || (ei >= t);
            float v = 0.f;
            if (ei != kPad && wasS) {
                const int inst = g * B + b;
                v = (R[(size_t)inst * ldP + t] * S[inst * kAges + age[r]]) * lam_t[x];
            }
            out[x] = v;
        }
    }
}

__global__ void k_philox(uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
        philox4x32_10(x, (uint32_t)seed, (uint32_t)(seed >> 32));
        for (int k = 0; k < 4; ++k) out[4 * i + k] = x[k];
    }
}

}  // namespace

cudaError_t launch_infectious_bits(const int16_t *e, int t0, int ndays, int L, int ntiles, uint32_t *bits,
                                   size_t day_stride, cudaStream_t s) {
    int grid = (ntiles + 7) / 8;
    if (grid > 65535) grid = 65535;
    k_infectious_bits<<<grid > 0 ? grid : 1, 256, 0, s>>>(e, t0, ndays, L, ntiles, bits, day_stride);
    return cudaGetLastError();
}

cudaError_t launch_infectious_bits_dur(const int16_t *e, GraphRef gr, const DurRef &d, int t, int ntiles,
                                       uint32_t *bits, cudaStream_t s) {
    int grid = (ntiles + 7) / 8;
    if (grid > 65535) grid = 65535;
    k_infectious_bits_dur<<<grid > 0 ? grid : 1, 256, 0, s>>>(e, gr, d, t, ntiles, bits);
    return cudaGetLastError();
}

cudaError_t launch_infectious_bits_fate(const int16_t *e, GraphRef gr, FateRef f, int t, int ntiles, uint32_t *bits,
                                        cudaStream_t s) {
    int grid = (ntiles + 7) / 8;
    if (grid > 65535) grid = 65535;
    k_infectious_bits_fate<<<grid > 0 ? grid : 1, 256, 0, s>>>(e, gr, f, t, ntiles, bits);
    return cudaGetLastError();
}

cudaError_t launch_init_state(int16_t *e, const int32_t *row0, const int32_t *rows, int G,
                              int64_t n_rows, int B, int Bp, int grid, cudaStream_t s) {
    k_init_state<<<grid, 256, 0, s>>>(e, row0, rows, G, n_rows, B, Bp);
    return cudaGetLastError();
}

cudaError_t launch_seed_reset(SeedState *st, const int32_t *n_seed, int I, cudaStream_t s) {
    k_seed_reset<<<(I + 127) / 128, 128, 0, s>>>(st, n_seed, I);
    return cudaGetLastError();
}

cudaError_t launch_seed_hist(const SeedArgs &a, int I, int grid_x, cudaStream_t s) {
    k_seed_hist<<<dim3(grid_x, I), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_seed_scan(const SeedArgs &a, int I, cudaStream_t s) {
    k_seed_scan<<<I, 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_seed_mark(const SeedArgs &a, int I, int grid_x, cudaStream_t s) {
    k_seed_mark<<<dim3(grid_x, I), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_seed_ties(const SeedArgs &a, int I, cudaStream_t s) {
    k_seed_ties<<<I, 256, 0, s>>>(a);
    return cudaGetLastError();
}

constexpr int kBitsBlock = 768;   // one block of 24 warps per SM when the bitmap lives in shared memory

__global__ void k_flags_from_bits(const uint32_t *bits_t, Sell m_out, int ntiles, uint8_t *flags) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile < ntiles; tile += warps)
        push_flags(m_out, tile, lane, (bits_t[tile] >> lane) & 1u, flags);
}

cudaError_t launch_flags_from_bits(const uint32_t *bits_t, Sell m_out, int ntiles, uint8_t *flags, cudaStream_t s) {
    int grid = (ntiles + 7) / 8;
    if (grid > 65535) grid = 65535;
    k_flags_from_bits<<<grid > 0 ? grid : 1, 256, 0, s>>>(bits_t, m_out, ntiles, flags);
    return cudaGetLastError();
}

cudaError_t launch_fwd_day(const FwdDayArgs &a, int grid, bool smem_bits, cudaStream_t s) {
    if (a.fate.L_M > 0) {
        k_fwd_day<false, kBlock, GABM_MINBLOCKS, false, kExitFate><<<grid, kBlock, 0, s>>>(a);
    } else if (a.dur.n > 0) {
        k_fwd_day<false, kBlock, GABM_MINBLOCKS, false, kExitDur><<<grid, kBlock, 0, s>>>(a);
    } else if (smem_bits && !a.pull) {
        const size_t bytes = (size_t)a.ntiles * sizeof(uint32_t);
        k_fwd_day<true, kBitsBlock, 1><<<grid, kBitsBlock, bytes, s>>>(a);
    } else if (a.pull) {
        k_fwd_day<false, kBlock, GABM_MINBLOCKS, true><<<grid, kBlock, 0, s>>>(a);
    } else {
        k_fwd_day<false, kBlock, GABM_MINBLOCKS><<<grid, kBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// Blocks per SM of the forward day kernel (global bitmap), or, for the
// shared-memory bitmap of `ntiles` words, 0 if it does not fit.
int occupancy_fwd(int ntiles, bool smem_bits) {
    int blocks = 0;
    if (smem_bits) {
        const size_t bytes = (size_t)ntiles * sizeof(uint32_t);
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (bytes + 4096 > (size_t)optin) return 0;
        cudaFuncSetAttribute(k_fwd_day<true, kBitsBlock, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_fwd_day<true, kBitsBlock, 1>, kBitsBlock, bytes);
        return blocks;
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_fwd_day<false, kBlock, GABM_MINBLOCKS>, kBlock, 0);
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_soft_init(const int16_t *e, int64_t n_rows, int L, const float *c, float *s, float *nh,
                             float *x_cur, cudaStream_t st) {
    int64_t grid = (n_rows + 255) / 256;
    if (grid > 65535) grid = 65535;
    k_soft_init<<<(int)(grid > 0 ? grid : 1), 256, 0, st>>>(e, n_rows, L, c, s, nh, x_cur);
    return cudaGetLastError();
}

cudaError_t launch_fwd_day_soft(const SoftDayArgs &a, int grid, cudaStream_t s) {
    k_fwd_day_soft<<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int occupancy_fwd_soft() {
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_fwd_day_soft, kBlock, 0);
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_soft_finalize(const double *P_nrm, int ntiles, const int32_t *graph_tile0,
                                 const int32_t *graph_ntiles, const float *m, int ldP, int T, int G,
                                 double *newRM_real, double *D_ctx, double *D_out, cudaStream_t s) {
    k_soft_finalize<<<dim3(T, G), 256, 0, s>>>(P_nrm, ntiles, graph_tile0, graph_ntiles, m, ldP, T, newRM_real,
                                               D_ctx, D_out);
    return cudaGetLastError();
}

cudaError_t launch_fwd_finalize(const int32_t *newRM, const int32_t *counts, const float *m, int ldP,
                                int t0, int T, int I, double *D_ctx, double *D_out,
                                int32_t *counts_out, cudaStream_t s) {
    const int total = I * T;
    const int grid = (total + 255) / 256;
    k_fwd_finalize<<<grid > 0 ? grid : 1, 256, 0, s>>>(newRM, counts, m, ldP, t0, T, I, D_ctx, D_out, counts_out);
    return cudaGetLastError();
}

cudaError_t launch_mse(const double *D, int ldP, const double *y, int T, int I, double *loss,
                       double *gD_ctx, double *gD_out, cudaStream_t s) {
    k_mse<<<I, 256, 0, s>>>(D, ldP, y, T, loss, gD_ctx, gD_out);
    return cudaGetLastError();
}

cudaError_t launch_get_lambda(const float *lam_t, const int16_t *e, const uint8_t *age, GraphRef gr,
                              const float *R, const float *S, int ldP, int t, int64_t n_rows, int B, int Bp,
                              float *out_rows, cudaStream_t s) {
    int grid = (int)((n_rows + 255) / 256);
    if (grid > 65535) grid = 65535;
    k_get_lambda<<<grid > 0 ? grid : 1, 256, 0, s>>>(lam_t, e, age, gr, R, S, ldP, t, n_rows, B, Bp, out_rows);
    return cudaGetLastError();
}

static int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 65535) g = 65535;
    return (int)(g > 0 ? g : 1);
}

cudaError_t launch_rows_to_caller_i16(const int16_t *src, int16_t *dst, GraphRef gr, const int32_t *rows,
                                      const int64_t *goff, int64_t n_rows, SetLayout sl, cudaStream_t s) {
    k_rows_to_caller<int16_t><<<grid_for(n_rows), 256, 0, s>>>(src, dst, gr, rows, goff, n_rows, sl);
    return cudaGetLastError();
}

cudaError_t launch_rows_to_caller_f32(const float *src, float *dst, GraphRef gr, const int32_t *rows,
                                      const int64_t *goff, int64_t n_rows, SetLayout sl, cudaStream_t s) {
    k_rows_to_caller<float><<<grid_for(n_rows), 256, 0, s>>>(src, dst, gr, rows, goff, n_rows, sl);
    return cudaGetLastError();
}

cudaError_t launch_caller_to_rows_i16(const int16_t *src, int16_t *dst, GraphRef gr, const int32_t *rows,
                                      const int64_t *goff, int64_t n_rows, SetLayout sl, cudaStream_t s) {
    k_caller_to_rows<int16_t><<<grid_for(n_rows), 256, 0, s>>>(src, dst, gr, rows, goff, n_rows, sl);
    return cudaGetLastError();
}

cudaError_t launch_philox(uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t count, cudaStream_t s) {
    int64_t grid = (count + 255) / 256;
    if (grid > 65535) grid = 65535;
    k_philox<<<(int)(grid > 0 ? grid : 1), 256, 0, s>>>(seed, ctr, out, count);
    return cudaGetLastError();
}

}  // namespace gabm
