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
// lambda_i(t) comes from the forward's store or is recomputed in the same pass
// from the final exposure days E (no reinfection, A3/A4 of App. A, so E
// determines every day's state and no checkpoints are needed).
#include "gabm_internal.cuh"
#include "rowsum.cuh"

namespace gabm {

namespace {

template <int GL, int MODE>
__global__ void __launch_bounds__(kBlock) k_bwd_day(const BwdDayArgs a) {
    __shared__ float c_s[kMaxL];
    __shared__ int slot_k[kMaxL];
    __shared__ uint8_t slot_s[kBlock / 32][32];
    __shared__ int32_t red_s[kBlock / 32][2];
    if (threadIdx.x < kMaxL) {
        c_s[threadIdx.x] = a.c[threadIdx.x];
        slot_k[threadIdx.x] = a.ring_slot[threadIdx.x];
    }
    __syncthreads();

    constexpr int RPP = 32 / GL;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int sub = lane / GL, gl = lane % GL;
    const int t = a.t, T = a.T, L = a.L;
    const bool has_next = (t + 1 < T);
    const int nwarps = gridDim.x * (kBlock / 32);

    int cur_g = -1, cN = 0;
    for (int tile = blockIdx.x * (kBlock / 32) + wib; tile < a.ntiles; tile += nwarps) {
        const int g = a.gr.tile_graph ? (int)a.gr.tile_graph[tile] : 0;
        if (g != cur_g) {
            if (cur_g >= 0) {
                const int s = __reduce_add_sync(0xffffffffu, cN);
                if (lane == 0 && s) atomicAdd(a.newRM + (size_t)cur_g * a.ldP + t, s);
            }
            cur_g = g;
            cN = 0;
        }
        const int row = tile * kTile + lane;
        const int Ei = a.E[row];
        const bool agent = (Ei != kPad);
        const bool never = (Ei == kNever);
        const bool live = agent && (never || Ei >= 0);           // seeds are constants
        const bool isS = live && (never || Ei >= t);
        const bool needA = has_next && live && (never || Ei >= t + 2 - L);
        cN += (agent && !never && t - Ei == L);
        const bool act = needA || isS;
        const unsigned amask = __ballot_sync(0xffffffffu, act);

        float gx_mine = 0.f, lam_mine = 0.f;
        if (amask) {
            uint32_t rs = 0, re = 0, irs = 0, ire = 0;
            if (act) { rs = a.rowptr[row]; re = a.rowptr[row + 1]; }
            if (MODE == kBwdSplit && isS) { irs = a.in_rowptr[row]; ire = a.in_rowptr[row + 1]; }
            const int rank = __popc(amask & lt_mask);
            if (act) slot_s[wib][rank] = (uint8_t)lane;
            __syncwarp();
            const int nA = __popc(amask);
            for (int base = 0; base < nA; base += RPP) {
                const int j = base + sub;
                const int src = (j < nA) ? slot_s[wib][j] : 0;
                const uint32_t rsj = __shfl_sync(0xffffffffu, rs, src);
                const uint32_t rej = __shfl_sync(0xffffffffu, re, src);
                const bool nAj = __shfl_sync(0xffffffffu, needA, src);
                const bool Sj = __shfl_sync(0xffffffffu, isS, src);
                float gxp = 0.f, lmp = 0.f;
                if (j < nA) {
                    if (MODE == kBwdFused) {
                        lane_adjoint_sums<GL, true>(a.col4, a.w4, a.E, a.r_next, c_s, rsj, rej, gl, t, L,
                                                    nAj, Sj, gxp, lmp);
                    } else {
                        if (nAj)
                            lane_adjoint_sums<GL, false>(a.col4, a.w4, a.E, a.r_next, c_s, rsj, rej, gl, t,
                                                         L, true, false, gxp, lmp);
                    }
                }
                if (MODE == kBwdSplit) {
                    const uint32_t irsj = __shfl_sync(0xffffffffu, irs, src);
                    const uint32_t irej = __shfl_sync(0xffffffffu, ire, src);
                    if (j < nA && Sj)
                        lmp = lane_infectious_sum<GL>(a.in_col4, a.in_w4, a.E, c_s, irsj, irej, gl, t, L);
                }
#pragma unroll
                for (int o = GL / 2; o > 0; o >>= 1) {
                    gxp += __shfl_xor_sync(0xffffffffu, gxp, o);
                    if (MODE != kBwdStore) lmp += __shfl_xor_sync(0xffffffffu, lmp, o);
                }
                const int myj = rank - base;
                const int from = (myj & (RPP - 1)) * GL;
                const float g1 = __shfl_sync(0xffffffffu, gxp, from);
                const float g2 = __shfl_sync(0xffffffffu, lmp, from);
                if (act && myj >= 0 && myj < RPP) { gx_mine = g1; lam_mine = g2; }
            }
            __syncwarp();
        }

        if (needA) a.ring[(size_t)slot_k[1] * a.ring_stride + row] = gx_mine;

        float v = 0.f;
        int ai = 0;
        if (isS) {
            ai = a.age[row];
            const int inst = g;
            const size_t pi = (size_t)inst * a.ldP;
            float G = 0.f;
            if (t + L < T) G = a.m[pi + t + L] * (float)a.gD[pi + t + L];
            if (has_next) G = __fmaf_rn(c_s[1], gx_mine, G);
            for (int k = 2; k < L; ++k)
                if (t + k < T) G = __fmaf_rn(c_s[k], a.ring[(size_t)slot_k[k] * a.ring_stride + row], G);
            float dy;
            if (Ei == t) { a.A[row] = G; dy = G; }
            else if (never) dy = G;
            else dy = G - a.A[row];
            const float Lam = (MODE == kBwdStore) ? a.lam_t[row] : lam_mine * a.gr.inv_Dbar[g];
            const float RS = a.R[pi + t] * a.S[inst * kAges + ai];
            const float lam = RS * Lam;
            const float q = expf(-lam);
            const float p = -expm1f(-lam);
            const uint32_t id = (uint32_t)(row - a.gr.row0[g]);
            const float u = uniform_from_word(philox_word(a.seed, id, (uint32_t)t, (uint32_t)inst, 0u));
            const float den = __fmaf_rn(p, 1.f - u, q * u);
            const float dydl = (u * (1.f - u)) * q / (den * den);
            const float glam = dy * dydl;
            a.r_cur[row] = RS * glam * a.gr.inv_Dbar[g];
            v = glam * Lam;
        }

        // per-tile sums of gl * Lam by age bin (fp32 over 32 rows, FP64 from here on)
        const unsigned smask = __ballot_sync(0xffffffffu, isS);
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

    const int s = __reduce_add_sync(0xffffffffu, cN);
    if (lane == 0) { red_s[wib][0] = cur_g; red_s[wib][1] = s; }
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

// Q[inst][t][a] = sum over the graph's tiles of P[t][tile][a], fixed order, FP64.
__global__ void __launch_bounds__(256) k_bwd_reduce(const double *P, int ntiles, const int32_t *graph_tile0,
                                                    const int32_t *graph_ntiles, int T, double *Q) {
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
    if (threadIdx.x < kAges) Q[((size_t)inst * T + t) * kAges + threadIdx.x] = s[0][threadIdx.x];
}

// dR_t = sum_a S_a Q[t][a];  dS_a = sum_t R_t Q[t][a];  dm_t = gD_t newRM(t).
__global__ void __launch_bounds__(256) k_bwd_finalize(const double *Q, const float *R, const float *S,
                                                      const double *gD, const int32_t *newRM, int ldP,
                                                      int T, double *dR, double *dm, double *dS) {
    const int inst = blockIdx.x;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const double *q = Q + ((size_t)inst * T + t) * kAges;
        double acc = 0.0;
        for (int b = 0; b < kAges; ++b) acc += (double)S[inst * kAges + b] * q[b];
        dR[(size_t)inst * T + t] = acc;
        dm[(size_t)inst * T + t] = gD[(size_t)inst * ldP + t] * (double)newRM[(size_t)inst * ldP + t];
    }
    if (threadIdx.x < kAges) {
        const int b = threadIdx.x;
        double acc = 0.0;
        for (int t = 0; t < T; ++t) acc += (double)R[(size_t)inst * ldP + t] * Q[((size_t)inst * T + t) * kAges + b];
        dS[inst * kAges + b] = acc;
    }
}

template <int MODE>
cudaError_t launch_bwd_mode(const BwdDayArgs &a, int lanes_per_row, int grid, cudaStream_t s) {
    switch (lanes_per_row) {
        case 4: k_bwd_day<4, MODE><<<grid, kBlock, 0, s>>>(a); break;
        case 8: k_bwd_day<8, MODE><<<grid, kBlock, 0, s>>>(a); break;
        case 16: k_bwd_day<16, MODE><<<grid, kBlock, 0, s>>>(a); break;
        case 32: k_bwd_day<32, MODE><<<grid, kBlock, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int MODE>
int occupancy_mode(int lanes_per_row) {
    int blocks = 0;
    switch (lanes_per_row) {
        case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day<4, MODE>, kBlock, 0); break;
        case 8: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day<8, MODE>, kBlock, 0); break;
        case 16: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day<16, MODE>, kBlock, 0); break;
        case 32: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_bwd_day<32, MODE>, kBlock, 0); break;
        default: break;
    }
    return blocks > 0 ? blocks : 1;
}

}  // namespace

cudaError_t launch_bwd_day(const BwdDayArgs &a, int lanes_per_row, int grid, cudaStream_t s) {
    switch (a.mode) {
        case kBwdStore: return launch_bwd_mode<kBwdStore>(a, lanes_per_row, grid, s);
        case kBwdFused: return launch_bwd_mode<kBwdFused>(a, lanes_per_row, grid, s);
        case kBwdSplit: return launch_bwd_mode<kBwdSplit>(a, lanes_per_row, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int occupancy_bwd(int lanes_per_row, int mode) {
    switch (mode) {
        case kBwdStore: return occupancy_mode<kBwdStore>(lanes_per_row);
        case kBwdFused: return occupancy_mode<kBwdFused>(lanes_per_row);
        default: return occupancy_mode<kBwdSplit>(lanes_per_row);
    }
}

cudaError_t launch_bwd_reduce(const double *P, int ntiles, int ldP, const int32_t *graph_tile0,
                              const int32_t *graph_ntiles, int T, int I, double *Q, cudaStream_t s) {
    (void)ldP;
    k_bwd_reduce<<<dim3(T, I), 256, 0, s>>>(P, ntiles, graph_tile0, graph_ntiles, T, Q);
    return cudaGetLastError();
}

cudaError_t launch_bwd_finalize(const double *Q, const float *R, const float *S, const double *gD,
                                const int32_t *newRM, int ldP, int T, int I, double *dR, double *dm,
                                double *dS, cudaStream_t s) {
    k_bwd_finalize<<<I, 256, 0, s>>>(Q, R, S, gD, newRM, ldP, T, dR, dm, dS);
    return cudaGetLastError();
}

}  // namespace gabm
