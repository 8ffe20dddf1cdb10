// sirs.cu -- forward and reverse day kernels of SIRS reinfection (see sirs.cuh).
//
// Each warp holds one 32-row tile at a time.  The sums
// are those of the base model's kernels -- the same row_sums over the same SELL entries,
// the same fused multiply-adds in the same order for G -- so with nobody returning
// within the horizon the results are bitwise the base model's.
#include "sirs.cuh"
#include "rowsum.cuh"

namespace gabm {

namespace {

__device__ __forceinline__ void flush_counts(int32_t *counts, int32_t *newRM, int ldP, int g, int t, int cS, int cE,
                                             int cI, int cR, int cN, int lane) {
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

// The history of every row starts with its state after seeding (a seed's exposure day).
__global__ void k_sirs_hist_init(const int16_t *e, int64_t n_rows, int H, int16_t *hist, uint16_t *cnt) {
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n_rows;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int ei = e[row];
        const bool exposed = ei != kNever && ei != kPad;
        cnt[row] = exposed ? 1 : 0;
        if (exposed) hist[row * H] = (int16_t)ei;
    }
}

// Day t: rows susceptible on day t (never exposed, or at least `cycle` days past their
// last exposure) draw; an exposure is appended to the row's history.  Each block takes a
// contiguous range of tiles (neighbours stay in its SM's L1), each warp's next tile is
// read one tile ahead, and a susceptible row with no infectious in-neighbour (flag_cur)
// reads no entries: its lambda is 0 exactly.
__global__ void __launch_bounds__(kBlock, 3) k_fwd_day_sirs(const SirsFwdArgs a) {
    __shared__ float c_s[kMaxL];
    if (threadIdx.x < kMaxL) c_s[threadIdx.x] = a.c[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int t = a.t, L = a.L, ntiles = a.ntiles;
    const uint32_t *bits = a.bits_cur;
    const int16_t *e = a.e;
    // neighbours marked infectious today (never written by this launch) contribute
    auto contrib = [&](uint32_t j, float w, bool valid, float (&out)[1], bool (&take)[1]) {
        const bool mk = valid && marked(bits, j);
        const int ej = ld_if(e + j, mk, kNever);
        out[0] = mk ? w * infectiousness(ej, c_s, t, L) : 0.f;
        take[0] = mk;
    };
    const bool want[1] = {true};
    int cur_g = -1, cS = 0, cE = 0, cI = 0, cR = 0, cN = 0;
    BlockTiles disp;
    disp.init(ntiles, lane);
    TileRows cur, nxt;
    load_tile_rows(a.m, e, a.gr.tile_graph, ntiles, disp.get(), lane, cur, a.flag_cur);
    load_tile_rows(a.m, e, a.gr.tile_graph, ntiles, disp.get(), lane, nxt, a.flag_cur);
    while (cur.tile < ntiles) {
        TileRows nn;
        load_tile_rows(a.m, e, a.gr.tile_graph, ntiles, disp.get(), lane, nn, a.flag_cur);
        const int g = cur.g, tile = cur.tile;
        if (g != cur_g) {
            if (cur_g >= 0) flush_counts(a.counts, a.newRM, a.ldP, cur_g, t, cS, cE, cI, cR, cN, lane);
            cur_g = g;
            cS = cE = cI = cR = cN = 0;
        }
        const int row = tile * kTile + lane;
        const int ei = cur.e;
        const bool agent = ei != kPad;
        const int k = t - ei;
        const bool isS = agent && (ei == kNever || k >= a.cycle);
        if (agent && !isS) {
            if (k < a.tau_EI) ++cE; else if (k < L) ++cI; else ++cR;
            cN += (k == L);
        }
        cS += isS;
        const bool act = isS && cur.flag;
        float sum[1];
        const unsigned amask = __ballot_sync(0xffffffffu, act);
        if (a.flag_cur && __popc(amask) <= GABM_COOP_ROWS) {   // few summing rows: warp-wide, together
            float cs = 0.f;
            sum[0] = 0.f;
            if (amask) few_row_sums(a.m, cur.p0, cur.len, amask, lane, contrib, sum[0], cs);
        } else {
            row_sums<1>(a.m, cur.p0, cur.len, act, lane, contrib, want, sum);
        }
        int e_next = ei;
        if (act) {
            const float Lam = sum[0] * a.gr.inv_Dbar[g];
            const float lam = (a.R[(size_t)g * a.ldP + t] * a.S[g * kAges + a.age[row]]) * Lam;
            const float p = -expm1f(-lam);
            const uint32_t id = caller_id(a.gr, row, g);
            const float u = uniform_from_word(philox_word(a.seed, id, (uint32_t)t, (uint32_t)g, 0u));
            if (u < p) {
                a.e[row] = (int16_t)t;
                e_next = t;
                // H covers the horizon (exposures are at least `cycle` days apart), so ci < H;
                // the count stops at H all the same, keeping every history access in bounds
                const int ci = a.cnt[row];
                if (ci < a.H) {
                    a.hist[(size_t)row * a.H + ci] = (int16_t)t;
                    a.cnt[row] = (uint16_t)(ci + 1);
                }
            }
            a.lam_out[row] = Lam;
        } else if (isS) {
            a.lam_out[row] = 0.f;
        }
        const int kn = t + 1 - e_next;
        const bool inf = (unsigned)(kn - 1) < (unsigned)(L - 1);
        const unsigned inf_next = __ballot_sync(0xffffffffu, inf);
        if (lane == 0) a.bits_next[tile] = inf_next;
        if (a.flag_cur) {   // tomorrow's flags: the out-neighbours of tomorrow's infectious rows
            push_flags(a.m_out, tile, lane, inf, a.flag_next);
            a.flag_clear[row] = 0;
        }
        cur = nxt;
        nxt = nn;
    }
    if (cur_g >= 0) flush_counts(a.counts, a.newRM, a.ldP, cur_g, t, cS, cE, cI, cR, cN, lane);
}

// The next tile's row data for the reverse sweep (one tile ahead of use).
__device__ __forceinline__ TileRows nn_next(const SirsBwdArgs &a, BlockTiles &disp, int lane) {
    TileRows nn;
    load_tile_rows(a.m, a.E, a.gr.tile_graph, a.ntiles, disp.get(), lane, nn);
    return nn;
}

// Reverse day t: gx(t+1) of every agent into the ring, then for rows susceptible on
// day t the adjoint of the draw, with the return terms B(t+1) and B(t+cycle) read from
// the G stored at the row's later exposures.
__global__ void __launch_bounds__(kBlock, 3) k_bwd_day_sirs(const SirsBwdArgs a) {
    __shared__ float c_s[kMaxL];
    __shared__ int slot_k[kMaxL];
    if (threadIdx.x < kMaxL) {
        c_s[threadIdx.x] = a.c[threadIdx.x];
        slot_k[threadIdx.x] = a.ring_slot[threadIdx.x];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int t = a.t, T = a.T, L = a.L, C = a.cycle, H = a.H;
    const bool has_next = t + 1 < T;
    const float *__restrict__ r_next = a.r_next;
    auto contrib = [&](uint32_t j, float w, bool valid, float (&out)[1], bool (&take)[1]) {
        out[0] = w * ld_if(r_next + j, valid);
        take[0] = valid;
    };
    const bool want[1] = {true};
    int cur_g = -1, cN = 0;
    unsigned emax_w = 0u;
    BlockTiles disp;
    disp.init(a.ntiles, lane);
    TileRows cur, nxt;
    load_tile_rows(a.m, a.E, a.gr.tile_graph, a.ntiles, disp.get(), lane, cur);
    load_tile_rows(a.m, a.E, a.gr.tile_graph, a.ntiles, disp.get(), lane, nxt);
    for (; cur.tile < a.ntiles; cur = nxt, nxt = nn_next(a, disp, lane)) {
        const int tile = cur.tile;
        const int g = cur.g;
        if (g != cur_g) {
            if (cur_g >= 0) {
                const int sN = __reduce_add_sync(0xffffffffu, cN);
                if (lane == 0 && sN) atomicAdd(a.newRM + (size_t)cur_g * a.ldP + t, sN);
                flush_emax(a.emax + (size_t)cur_g * a.ld_sig + t, emax_w);
                emax_w = 0u;
            }
            cur_g = g;
            cN = 0;
        }
        const int32_t *sg = a.sig + (size_t)g * a.ld_sig;
        const int sig_t = next_sigma(sg[t + 1], a.emax[(size_t)g * a.ld_sig + t + 1]);
        if (lane == 0 && tile * kTile == a.gr.row0[g]) a.sig[(size_t)g * a.ld_sig + t] = sig_t;

        const int row = tile * kTile + lane;
        const bool agent = cur.e != kPad;
        const int n_e = min((int)a.cnt[row], H);
        const int16_t *hr = a.hist + (size_t)row * H;
        int j_t = 0;   // exposures before day t
        while (j_t < n_e && hr[j_t] < t) ++j_t;
        const bool y = j_t < n_e && hr[j_t] == t;
        const int e_t = j_t > 0 ? hr[j_t - 1] : kNever;
        const bool isS = agent && (e_t == kNever || t - e_t >= C);
        cN += (agent && e_t != kNever && t - e_t == L);

        // gx(t+1) is used by the G of the row's susceptible days in [t + 2 - L, t]; a row
        // with none lies, the whole window, inside one exposure's stretch (e, e + C) of not
        // being susceptible, e in [t - C + 1, lo - 1], and skips the gather
        const int lo = max(0, t + 2 - L);
        bool covered = false;
        for (int j = 0; j < j_t; ++j) covered |= (hr[j] >= t - C + 1 && hr[j] <= lo - 1);
        const bool act = has_next && agent && !covered;
        float sum[1];
        row_sums<1>(a.m, cur.p0, cur.len, act, lane, contrib, want, sum,
                    [&](uint32_t j, float w) { return w * r_next[j]; });
        const float gx1 = sum[0];
        if (act) a.ring[(size_t)slot_k[1] * a.ring_stride + row] = gx1;

        float v = 0.f, rc = 0.f;
        int ai = 0;
        if (isS) {
            ai = a.age[row];
            // B(t'): G at the row's first exposure on or after day t' (0 if none), at day t's scale
            auto B_at = [&](int tp) -> float {
                int j = j_t;
                while (j < n_e && hr[j] < tp) ++j;
                return j < n_e ? a.Gh[(size_t)row * H + j] * exp2i(sg[hr[j]] - sig_t) : 0.f;
            };
            const size_t pg = (size_t)g * a.ldP;
            // the day's own terms: the death term and the infectiousness it would cause
            float loc = (t + L < T) ? a.m_t[pg + t + L] * (float)a.gD[pg + t + L] * exp2i(-sig_t) : 0.f;
            if (has_next) loc = __fmaf_rn(c_s[1], gx1 * exp2i(sg[t + 1] - sig_t), loc);
            for (int k = 2; k < L; ++k)
                if (t + k < T) loc = __fmaf_rn(c_s[k], a.ring[(size_t)slot_k[k] * a.ring_stride + row] * exp2i(sg[t + k] - sig_t), loc);
            const float G = loc + B_at(t + C);
            // dL/dy = G - B(t+1).  With t' the row's first exposure after t, B(t+1) = G(t'),
            // and B(t+C) = B(t'+C) when t' < t+C (the next exposure after t' is at least
            // t'+C), while B(t+C) = G(t') when t' >= t+C: so dL/dy = loc - loc(t') or loc.
            // Formed this way the return terms cancel exactly instead of in fp32, where on
            // short cycles they dwarf the difference.
            const int jn = y ? j_t + 1 : j_t;
            float dy = loc;
            if (jn < n_e && hr[jn] < t + C) dy = loc - a.Lh[(size_t)row * H + jn] * exp2i(sg[hr[jn]] - sig_t);
            if (y) {
                a.Gh[(size_t)row * H + j_t] = G;
                a.Lh[(size_t)row * H + j_t] = loc;
            }
            float stored = fmaxf(fabsf(G), fabsf(loc));
            const float Lam = a.lam_t[row];
            const float RS = a.R[pg + t] * a.S[g * kAges + ai];
            const float lam = RS * Lam;
            const float q = expf(-lam);
            const float p = -expm1f(-lam);
            const uint32_t id = caller_id(a.gr, row, g);
            const float u = uniform_from_word(philox_word(a.seed, id, (uint32_t)t, (uint32_t)g, 0u));
            const float den = __fmaf_rn(p, 1.f - u, q * u);
            const float dydl = (u * (1.f - u)) * q / (den * den);
            const float glam = dy * dydl;
            rc = RS * glam * a.gr.inv_Dbar[g];
            v = glam * Lam;
            stored = fmaxf(stored, fabsf(rc));
            emax_w = max(emax_w, (unsigned)(float_exponent(stored) + 128));
        }
        a.r_cur[row] = rc;   // 0 for rows not susceptible today (r of a later day may sit there)

        const unsigned smask = __ballot_sync(0xffffffffu, isS);
        float mine = 0.f;   // lanes 2b, 2b + 1: bin b (the base kernel's tree)
        if (smask) mine = warp_bin_sums16(isS ? v : 0.f, ai, lane);
        if (!(lane & 1) && (lane >> 1) < kAges) a.P_t[(size_t)tile * kAges + (lane >> 1)] = (double)mine;
    }
    if (cur_g >= 0) {
        const int sN = __reduce_add_sync(0xffffffffu, cN);
        if (lane == 0 && sN) atomicAdd(a.newRM + (size_t)cur_g * a.ldP + t, sN);
        flush_emax(a.emax + (size_t)cur_g * a.ld_sig + t, emax_w);
    }
}

}  // namespace

cudaError_t launch_sirs_hist_init(const int16_t *e, int64_t n_rows, int H, int16_t *hist, uint16_t *cnt,
                                  cudaStream_t s) {
    const int grid = (int)std::min<int64_t>((n_rows + 255) / 256, 65535);
    k_sirs_hist_init<<<grid > 0 ? grid : 1, 256, 0, s>>>(e, n_rows, H, hist, cnt);
    return cudaGetLastError();
}

cudaError_t launch_fwd_day_sirs(const SirsFwdArgs &a, int grid, cudaStream_t s) {
    k_fwd_day_sirs<<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bwd_day_sirs(const SirsBwdArgs &a, int grid, cudaStream_t s) {
    k_bwd_day_sirs<<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int occupancy_sirs(bool backward) {
    int blocks = 0;
    if (backward) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day_sirs, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_fwd_day_sirs, kBlock, 0);
    return blocks > 0 ? blocks : 1;
}

}  // namespace gabm
