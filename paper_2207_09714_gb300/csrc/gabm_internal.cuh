// gabm_internal.cuh -- internal declarations of the GB300 GradABM library.
//
// Layout in device memory (one ctx):
//   graphs are concatenated block-diagonally, each padded to a multiple of 32
//   rows so that a 32-row tile never straddles two graphs; padding rows have
//   no edges and exposure day kPad.
//   SELL-32 in-edges (row i lists its in-neighbours j with w_ji), one slice of
//   max_len x 32 entries per 32-row tile, column-major:
//   slice_ptr u32 [ntiles+1], row_len u32 [n_rows], col u32 / w f32 [entries]
//   (the out-edges in the same layout when the weights are not symmetric)
//   age     u8  [n_rows]
//   e       i16 [n_rows]          exposure day (kNever = susceptible)
//   lam     f32 [Tcap][n_rows]    normalised neighbour sums (store policy)
//   ring    f32 [L-1][n_rows]     adjoint of infectiousness, last L-1 days
//   r       f32 [2][n_rows]       per-day transpose-gather coefficients
//   P       f64 [Tcap][ntiles][9] per-tile, per-age partial gradient sums
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gabm.h"

namespace gabm {

constexpr int kNever = GABM_NEVER;
constexpr int kPad = -32768;       // exposure day of a padding row (not an agent)
constexpr int kAges = GABM_NUM_AGES;
constexpr int kMaxL = GABM_MAX_L;
constexpr int kTile = 32;          // rows per warp tile
constexpr int kBlock = 256;        // threads per block of the day kernels
constexpr int kHistBins = 2048;    // radix-select digit bins (11 bits)
// Agents sharing the threshold hash (seeding).  A tie needs equal 32-bit Philox words;
// among n < 2^31 agents the count of any one word is Binomial(n, 2^-32), mean < 0.5, so
// more than kTieCap agents on one word has probability below 2^32 * 0.5^4097 / 4097!,
// far below 1e-10000.  k_seed_mark still flags that case (SeedState::overflow) rather than
// write past the list.
constexpr int kTieCap = 4096;
constexpr int kMaxSets = 64;       // parameter sets per graph (batched kernels: two per lane)
// Batched sums use plain fused multiply-adds when no row has more entries than this:
// a sum of k non-negative terms then carries a relative error below (k + 3) 2^-24 < 1e-5.
constexpr int kPlainSumMaxDegree = 64;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its
// published definition: ten rounds, each multiplying counter words 0 and 2 by
// the two round multipliers (32x32 -> 64 bits), swapping/xoring the halves
// with counter words 1 and 3 and the key; the key is advanced by the two Weyl
// constants between rounds.  Only the first output word is used.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ void philox4x32_10(uint32_t x[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = mulhi32(m0, x[0]), lo0 = m0 * x[0];
        uint32_t hi1 = mulhi32(m1, x[2]), lo1 = m1 * x[2];
        uint32_t y0 = hi1 ^ x[1] ^ k0;
        uint32_t y2 = hi0 ^ x[3] ^ k1;
        x[0] = y0; x[1] = lo1; x[2] = y2; x[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ uint32_t philox_word(uint64_t seed, uint32_t id, uint32_t day,
                                                uint32_t inst, uint32_t stream) {
    uint32_t x[4] = {id, day, inst, stream};
    philox4x32_10(x, (uint32_t)seed, (uint32_t)(seed >> 32));
    return x[0];
}

// u = ((x0 >> 9) + 0.5) * 2^-23 = (2 (x0 >> 9) + 1) * 2^-24: an odd integer below
// 2^24 times a power of two, so exact in fp32.
__device__ __forceinline__ float uniform_from_word(uint32_t x0) {
    return __uint2float_rn(((x0 >> 9) << 1) | 1u) * 5.9604644775390625e-8f;
}

// ---------------------------------------------------------------------------
// Kernel arguments
// ---------------------------------------------------------------------------
struct GraphRef {                 // where each graph sits in the concatenated arrays
    const int32_t *row0;          // [G] first row of each graph
    const uint16_t *tile_graph;   // [ntiles] graph of each tile (nullptr when G == 1)
    const float *inv_Dbar;        // [G] 1 / mean weighted degree (0 for an edgeless graph)
    const uint32_t *orig_id;      // [n_rows] caller's id of each row (nullptr: row - row0)
};

__device__ __forceinline__ uint32_t caller_id(const GraphRef &gr, int row, int g) {
    return gr.orig_id ? gr.orig_id[row] : (uint32_t)(row - gr.row0[g]);
}

// Sampled R/M split (Sec. 3.1 names a mortality stage M with its own I->M time tau_IM):
// an agent exposed on day d draws its fate on its I-entry day t_I = d + tau_EI (day 0 for
// exposures before -tau_EI) -- M with probability m_{t_I}, else R -- and leaves I at
// L_M = tau_EI + tau_IM or L_R = tau_EI + tau_IR days after exposure.  Deaths are the
// M entries.  L_M = 0 selects the base model's single RM exit.
struct FateRef {
    const float *mort;   // mortality m [I][ldP]
    int ldP, tau_EI, L_R, L_M;
    uint64_t seed;
};

// The fate's uniform v: Philox stream 1 of the agent's caller id on day t_I (stream 0 is
// the infection draw); M iff v < m_{t_I}.
__device__ __forceinline__ float fate_uniform(const FateRef &f, uint32_t id, int tI, int inst) {
    return uniform_from_word(philox_word(f.seed, id, (uint32_t)tI, (uint32_t)inst, 1u));
}

// Whether agent `id`'s exposure on day d is M-fated; draws on or after day T are not made.
__device__ __forceinline__ bool fate_M(const FateRef &f, uint32_t id, int d, int inst, int T) {
    const int tI = max(d + f.tau_EI, 0);
    if (tI >= T) return false;
    return fate_uniform(f, id, tI, inst) < f.mort[(size_t)inst * f.ldP + tI];
}

// Stochastic I-stage durations (Sec. 6 names stochastic progression): an exposure of
// day d stays in I for j days, j the first with u < F[j-1] (F: the pmf's running sums in
// FP64, tau_IR if none), u the Philox uniform of (caller id, max(d, 0), instance, stream 2);
// it leaves I at L_i = tau_EI + j days after exposure.  n = 0: every agent stays tau_IR days.
struct DurRef {
    int n;               // pmf entries (tau_IR) or 0
    int tau_EI;
    uint64_t seed;
    double F[kMaxL];     // running sums of the pmf
};

// Exit offset L_i of agent `id`'s exposure on day d (F_s: the running sums, e.g. in shared memory).
__device__ __forceinline__ int dur_exit(const DurRef &dr, const double *F_s, uint32_t id, int d, int inst) {
    const double u = (double)uniform_from_word(philox_word(dr.seed, id, (uint32_t)max(d, 0), (uint32_t)inst, 2u));
    int j = 1;
    while (j < dr.n && !(u < F_s[j - 1])) ++j;
    return dr.tau_EI + j;
}

enum { kExitBase = 0, kExitFate = 1, kExitDur = 2 };

// Edges of one orientation in SELL-32 layout (one slice per 32-row tile).
struct Sell {
    const uint32_t *slice_ptr;  // [ntiles+1] first entry of each slice
    const uint32_t *row_len;    // [n_rows] entries of each row
    const uint32_t *col;        // [entries] column (neighbour row) of each entry
    const float *w;             // [entries] weight of each entry (0 in padding)
};

struct FwdDayArgs {
    Sell m;               // in-edges: row i lists j with w_ji
    const uint8_t *age;
    GraphRef gr;
    int16_t *e;
    float *lam_out;       // day-t slice of the lambda store, or nullptr
    const float *R;       // [I][ldP]
    const float *S;       // [I][9]
    int ldP;              // per-instance stride of R (and m)
    int32_t *counts;      // [I][ldP][4]
    int32_t *newRM;       // [I][ldP]
    const uint32_t *bits_cur;   // [ntiles] bit i of word r/32: row r infectious on day t
    uint32_t *bits_next;        // [ntiles] the same for day t + 1 (written by this launch)
    const float *pull;          // agent-location graphs: location pressures P [locations] (m lists
                                // each agent's locations), gathered in place of marked neighbours
    // Rows with an infectious in-neighbour (one byte per row), or nullptr (every
    // susceptible row sums): flag_cur for day t; the launch sets flag_next (day t + 1)
    // for the out-neighbours of the rows infectious tomorrow, and clears its rows of
    // flag_clear (the buffer day t + 1 will fill for day t + 2).
    const uint8_t *flag_cur;
    uint8_t *flag_next, *flag_clear;
    Sell m_out;                 // out-edges (the in-edges when the weights are symmetric)
    int t_first;                // first day of this forward (counts of earlier days are not its own)
    int ntiles, t, tau_EI, L;   // L: the longest infectious window (the table's length)
    uint64_t seed;
    FateRef fate;               // sampled R/M split (fate.L_M > 0) or the single RM exit
    DurRef dur;                 // stochastic I-stage durations (dur.n > 0)
    float c[kMaxL];
};

// Fixed-noise soft relaxation (every draw uses y = sigmoid(logit p - logit u)):
// the state is the susceptible mass s_i and the newly exposed mass n_i(d) of
// the last L days; x_i(t) = sum_{k=1}^{L-1} c[k] n_i(t-k) is what neighbours pull.
struct SoftDayArgs {
    Sell m;                  // in-edges
    const uint8_t *age;
    GraphRef gr;
    const int16_t *e;        // exposure days after seeding (padding rows: kPad)
    const float *x_cur;      // [n_rows] x_i(t)
    float *x_next;           // [n_rows] x_i(t+1)
    float *s;                // [n_rows] susceptible mass
    float *nh;               // [L][n_rows] n_i(d) in slot d mod L
    float *s_hist_t, *y_hist_t, *lam_t;   // day-t histories [n_rows]: s_i(t), y_i(t), Lam_i(t)
    const float *R, *S;
    int ldP;
    double *P_nrm_t;         // [ntiles] per-tile sums of n_i(t - L) (newRM of day t)
    int ntiles, t, L;
    uint64_t seed;
    float c[kMaxL];
};

struct BwdDayArgs {
    Sell m;                    // out-edges (the in-edges themselves when the weights are symmetric)
    const uint8_t *age;
    GraphRef gr;
    const int16_t *E;          // final exposure days
    const uint32_t *bits_t;    // [ntiles] rows infectious on day t (recompute policy) or nullptr
    const float *lam_t;        // stored normalised sums for day t (store policy) or nullptr
    const float *r_next;       // coefficients of day t+1 [n_rows]
    float *r_cur;              // coefficients of day t   [n_rows]
    float *ring;               // [L-1][n_rows]
    size_t ring_stride;
    float *A;                  // [n_rows] adjoint of s carried back from the infection day (soft: dL/ds(t+1))
    const float *s_hist_t, *y_hist_t;   // soft mode: s_i(t), y_i(t)
    const float *s_hist, *y_hist;       // soft mode, table adjoint: all days [T][hist_stride]
    size_t hist_stride;
    const float *R, *m_t, *S;  // R and mortality [I][ldP], susceptibility [I][9]
    const double *gD;          // [I][ldP]
    int ldP;
    double *P_t;               // [ntiles][9] partial sums of gl * Lam for day t
    int32_t *newRM;            // [I][ldP]
    int ntiles, t, T, tau_EI, L;
    int mode;                  // kBwdStore, kBwdFused or kBwdSplit
    uint64_t seed;
    float c[kMaxL];
    int ring_slot[kMaxL];      // ring slot holding day t + k, k = 1..L-1
    int32_t *sig, *emax;       // [G][ld_sig] scale exponent and largest stored exponent per day
    int ld_sig;
    double *dc_tile;           // [ntiles][kMaxL] per-tile sums of the table adjoint over days, or nullptr
    // agent-location graphs: r_next is the location adjoint gP; the agent's own share of its
    // locations, self_q[i] * self_r[i] with self_q = sum_l w_il^2 and self_r = r(t+1), is
    // removed from the gather (the pair weights have no self term)
    const float *self_r, *self_q;
    // sampled R/M split (fate.L_M > 0): Pm_t [ntiles] receives, per tile, the fate-draw share
    // of dL/dm on day t + tau_EI of the agents exposed on day t
    FateRef fate;
    double *Pm_t;
    DurRef dur;                // stochastic I-stage durations (dur.n > 0)
};

enum { kBwdStore = 0, kBwdFused = 1, kBwdSplit = 2, kBwdSoft = 3 };

struct SeedState {
    uint32_t prefix;    // high bits of the threshold hash found so far
    uint32_t k_rem;     // seeds still to choose among keys matching the prefix
    uint32_t eq_count;  // keys equal to the final threshold hash
    uint32_t tie_n;     // candidates appended to the tie list
    int32_t none;       // 1 when no seed is to be chosen
    int32_t overflow;   // tie list overflowed
};

struct SeedArgs {
    const int32_t *row0;  // [G]
    const int32_t *rows;  // [G] real rows per graph
    const uint32_t *orig_id;  // [n_rows] or nullptr
    int16_t *e;           // [n_rows][Bp]: instance i = graph i / B, set i % B
    int B, Bp;            // parameter sets per graph and the row stride of e
    SeedState *st;        // [I]
    uint32_t *hist;       // [I][kHistBins]
    uint32_t *ties;       // [I][kTieCap]
    uint64_t seed;
    int tau_EI;
    int pass;             // 0, 1, 2
};

// ---------------------------------------------------------------------------
// Batched instances: B parameter sets on each graph (batched.cu).  Per-agent
// arrays are agent-major, [n_rows][Bp] with Bp = B rounded up to a power of two
// (2..64); sets B..Bp-1 are padding (exposure day kPad).  One warp handles a
// row with Bp/2 lanes, two sets per lane, so one neighbour's exposure days for
// all sets are one contiguous Bp*2-byte gather.
// ---------------------------------------------------------------------------
struct Csr {                     // one orientation of the edges, row-compressed
    const uint32_t *rowptr;      // [n_rows+1]
    const uint32_t *col;         // [nnz]
    const float *w;              // [nnz]
};

struct FwdBatchArgs {
    Csr m;                       // in-edges
    const uint8_t *age;
    GraphRef gr;
    int16_t *e;                  // [n_rows][Bp]
    float *lam_out;              // day-t slice [n_rows][Bp] of the lambda store, or nullptr
    const float *R, *S;          // [I][ldP], [I][9]
    int ldP;
    uint8_t *tile_new;           // [ntiles][Bp] agents exposed on day t, by tile and set
    int *tile_ctr;
    const uint32_t *bits_cur;    // [ntiles] rows infectious on day t in any set
    uint32_t *bits_next;         // the same for day t + 1
    int ntiles, t, tau_EI, L, B;
    uint64_t seed;
    float c[kMaxL];
};

struct BwdBatchArgs {
    Csr m;                       // out-edges (the in-edges when the weights are symmetric)
    const uint8_t *age;
    GraphRef gr;
    const int16_t *E;            // [n_rows][Bp] final exposure days
    const float *lam_t;          // [n_rows][Bp] stored normalised sums of day t
    const float *r_next;         // [n_rows][Bp] coefficients of day t+1
    float *r_cur;                // [n_rows][Bp] coefficients of day t
    const uint32_t *rbits_next;  // [ntiles] rows susceptible on day t+1 in some set
    uint32_t *rbits_cur;         // the same for day t
    float *ring;                 // [L-1][n_rows][Bp]
    size_t ring_stride;
    float *A;                    // [n_rows][Bp]
    const float *R, *m_t, *S;
    const double *gD;
    int ldP;
    double *P_t;                 // [ntiles][9][Bp] per-tile partial sums of gl * Lam
    int *tile_ctr;
    int ntiles, t, T, tau_EI, L, B;
    uint64_t seed;
    float c[kMaxL];
    int ring_slot[kMaxL];
    int32_t *sig, *emax;         // [G][ld_sig] per graph (shared by its sets)
    int ld_sig;
    int Bw, s0;                  // row width of the per-agent arrays; first set of this launch
    double *dc_tile;             // [ntiles][L][Bw] per-tile sums of the table adjoint over days, or nullptr
    const uint32_t *bits_t;      // recompute policy (lam_t == nullptr): [ntiles] rows infectious on day t in any set
};

// Schedules: spl sets per lane (2, 4 or 8; Bp / spl lanes share a row).
bool batch_config_ok(int Bp, int spl);
cudaError_t launch_fwd_day_b(const FwdBatchArgs &a, int Bp, int spl, bool kahan, int grid, cudaStream_t s);
// The backward runs the row's sets in launches of Bc sets (a.s0 .. a.s0 + Bc - 1).
cudaError_t launch_bwd_day_b(const BwdBatchArgs &a, int Bc, int spl, bool kahan, int grid, cudaStream_t s);
int occupancy_fwd_b(int Bp, int spl, bool kahan);
int occupancy_bwd_b(int Bc, int spl, bool kahan);
// rows with 1 <= t0 - e < L in any set
cudaError_t launch_infectious_bits_b(const int16_t *e, int Bp, int t0, int L, int ntiles, uint32_t *bits,
                                     cudaStream_t s);
// H [I][L+2] (zeroed by the caller): exposure days of the state at the start of day t0
cudaError_t launch_exposure_hist_b(const int16_t *e, GraphRef gr, int64_t n_rows, int B, int Bp, int t0, int L,
                                   int32_t *H, cudaStream_t s);
// counts [I][ldP][4] and newRM [I][ldP] of days t0..T-1 from H and the per-tile exposures
// tile_new [T][ntiles][Bp]; newinf [I][ldP] is scratch, zeroed by the caller.
cudaError_t launch_counts_b(const uint8_t *tile_new, int ntiles, const int32_t *d_tile0, const int32_t *d_ntiles,
                            const int32_t *d_rows, int G, int B, int Bp, int max_tiles, int t0, int T, int ldP,
                            int tau_EI, int L, const int32_t *H, int32_t *newinf, int32_t *counts, int32_t *newRM,
                            cudaStream_t s);
// Q[g*B+s][t][a] = sum over graph g's tiles of P[t][tile][a][s], in a fixed order (two levels of
// kReduceChunkTiles tiles); scratch holds T * G * max_chunks * 9 * Bp doubles.
cudaError_t launch_bwd_reduce_b(const double *P, int ntiles, const int32_t *d_tile0, const int32_t *d_ntiles, int G,
                                int B, int Bp, int T, double *scratch, int max_chunks, const int32_t *sig,
                                int ld_sig, double *Q, cudaStream_t s);
constexpr int kReduceChunkTiles = 64;

// ---------------------------------------------------------------------------
// Range of the reverse sweep.  The straight-through factor dy/dlambda = (1-u)/u at
// p -> 0 is heavy-tailed, so the adjoint grows multiplicatively along infection
// chains and can leave the fp32 range over long horizons.  Every value the sweep
// stores for day d of graph g (ring entries, A, r, per-tile partial sums) is kept
// at scale 2^-sigma_g(d): sigma_g(T) = 0 and, going back, sigma_g(t) = sigma_g(t+1)
// + (emax_g(t+1) > kScaleHigh ? emax_g(t+1) - kScaleTarget : 0), where emax_g(d) is
// the largest binary exponent of the values stored on day d (a max, so the same in
// every block and every run).  Terms of different days are combined with exact
// power-of-two factors; the FP64 reductions multiply 2^sigma back in.
// ---------------------------------------------------------------------------
constexpr int kScaleHigh = 64;
constexpr int kScaleTarget = 32;

__device__ __forceinline__ int float_exponent(float x) {   // floor(log2 |x|), -127 for 0
    return (int)((__float_as_uint(x) >> 23) & 0xffu) - 127;
}

__device__ __forceinline__ int next_sigma(int sigma_next, int emax_next) {
    return sigma_next + (emax_next > kScaleHigh ? emax_next - kScaleTarget : 0);
}

// 2^k for k <= 127 (0 below the normal range: such terms are negligible at this day's scale)
__device__ __forceinline__ float exp2i(int k) {
    return k < -126 ? 0.f : __int_as_float((k + 127) << 23);
}

// Record this warp's largest stored exponent (+128, 0 = none) for one day of one graph;
// the atomic is skipped when the stored maximum is already as large.
__device__ __forceinline__ void flush_emax(int32_t *emax_gt, unsigned em_lane) {
    const unsigned em = __reduce_max_sync(0xffffffffu, em_lane);
    if ((threadIdx.x & 31) == 0 && em) {
        const int v = (int)em - 128;
        if (*(volatile int32_t *)emax_gt < v) atomicMax(emax_gt, v);
    }
}

// Launchers (forward.cu / backward.cu)
cudaError_t launch_init_state(int16_t *e, const int32_t *row0, const int32_t *rows, int G,
                              int64_t n_rows, int B, int Bp, int grid, cudaStream_t s);
cudaError_t launch_seed_reset(SeedState *st, const int32_t *n_seed, int I, cudaStream_t s);
cudaError_t launch_seed_hist(const SeedArgs &a, int I, int grid_x, cudaStream_t s);
cudaError_t launch_seed_scan(const SeedArgs &a, int I, cudaStream_t s);
cudaError_t launch_seed_mark(const SeedArgs &a, int I, int grid_x, cudaStream_t s);
cudaError_t launch_seed_ties(const SeedArgs &a, int I, cudaStream_t s);
cudaError_t launch_fwd_day(const FwdDayArgs &a, int grid, bool smem_bits, cudaStream_t s);
// Flags for day t of the rows with an in-neighbour infectious on day t (bits_t): every
// out-neighbour of a marked row gets flag 1.  flags must be zero on entry.
cudaError_t launch_flags_from_bits(const uint32_t *bits_t, Sell m_out, int ntiles, uint8_t *flags, cudaStream_t s);
// bits[d][tile] for days t0 .. t0 + ndays - 1: rows with 1 <= t - e < L (infectious on day t).
cudaError_t launch_infectious_bits_fate(const int16_t *e, GraphRef gr, FateRef f, int t, int ntiles, uint32_t *bits,
                                        cudaStream_t s);
cudaError_t launch_infectious_bits_dur(const int16_t *e, GraphRef gr, const DurRef &d, int t, int ntiles,
                                       uint32_t *bits, cudaStream_t s);
cudaError_t launch_fate_seeds(Sell m_out, const int16_t *E, const float *r0, const float *ring, size_t ring_stride,
                              int Lm1, GraphRef gr, FateRef f, const double *gD, const int32_t *sig, int ld_sig,
                              int ntiles, int T, const float *c, double *Pm, int grid, cudaStream_t s);
cudaError_t launch_fate_dm(const double *Pm, int ntiles, const int32_t *graph_tile0, const int32_t *graph_ntiles,
                           int G, int T, double *dm, cudaStream_t s);
cudaError_t launch_infectious_bits(const int16_t *e, int t0, int ndays, int L, int ntiles, uint32_t *bits,
                                   size_t day_stride, cudaStream_t s);
cudaError_t launch_fwd_finalize(const int32_t *newRM, const int32_t *counts, const float *m, int ldP,
                                int t0, int T, int I, double *D_ctx, double *D_out,
                                int32_t *counts_out, cudaStream_t s);
cudaError_t launch_mse(const double *D, int ldP, const double *y, int T, int I, double *loss,
                       double *gD_ctx, double *gD_out, cudaStream_t s);
cudaError_t launch_bwd_day(const BwdDayArgs &a, int grid, cudaStream_t s);
// Adjoint of the infectiousness table (hard mode, one set per graph): the seeds'
// share through their day-0 infectiousness, then the per-graph sums of dc_tile.
cudaError_t launch_dc_seeds(Sell m_out, const int16_t *E, const float *r0, GraphRef gr, const int32_t *sig,
                            int ld_sig, int ntiles, int L, double *dc_tile, int grid, cudaStream_t s);
cudaError_t launch_dc_reduce(const double *dc_tile, const int32_t *graph_tile0, const int32_t *graph_ntiles, int G,
                             int L, double *dc, cudaStream_t s);
cudaError_t launch_dc_seeds_b(Csr m_out, const int16_t *E, const float *r0, GraphRef gr, const int32_t *sig,
                              int ld_sig, int ntiles, int L, int B, int Bp, double *dc_tile, cudaStream_t s);
cudaError_t launch_dc_reduce_b(const double *dc_tile, const int32_t *graph_tile0, const int32_t *graph_ntiles, int G,
                               int B, int Bp, int L, double *dc, cudaStream_t s);
// Location hop of agent-location graphs (twohop.cu): pressures of day t and adjoints.  Small
// locations are SELL-32 tiles (values at [0, 32 * nloc_tiles)); large ones a CSR of their
// members (values at [base, base + n)).
struct LocCsr {
    const uint32_t *rowptr;   // [n+1]
    const uint32_t *col;      // member rows
    const float *w;           // attendance weights
    int n, base;
};
cudaError_t launch_loc_pressure(Sell ml, int nloc_tiles, LocCsr big, const int16_t *e, const uint32_t *bits, int t,
                                int L, const float *c, float *P, int grid, cudaStream_t s);
cudaError_t launch_loc_adjoint(Sell ml, int nloc_tiles, LocCsr big, const float *r, const float *c, float *gP,
                               int grid, cudaStream_t s);
int occupancy_loc();
cudaError_t launch_lam_day(Sell m, const int16_t *E, const uint32_t *bits, GraphRef gr, int t, int L, int ntiles,
                           const float *c, float *lam_out, int grid, cudaStream_t s);
// Q[g][t][a] = 2^sigma_g(t) x (sum over graph g's tiles of P[t][tile][a]), FP64.
cudaError_t launch_bwd_reduce(const double *P, int ntiles, int ldP, const int32_t *graph_tile0,
                              const int32_t *graph_ntiles, int T, int I, const int32_t *sig, int ld_sig,
                              double *Q, cudaStream_t s);
// newRM_real (soft mode, [I][ldP]) replaces the integer newRM when non-null.
cudaError_t launch_bwd_finalize(const double *Q, const float *R, const float *S, const double *gD,
                                const int32_t *newRM, const double *newRM_real, int ldP, int T, int I, double *dR,
                                double *dm, double *dS, cudaStream_t s);
// Soft relaxation (forward.cu): state from the seeded exposure days, one day, newRM reduction,
// and D = m newRM with copies out.
cudaError_t launch_soft_init(const int16_t *e, int64_t n_rows, int L, const float *c, float *s, float *nh,
                             float *x_cur, cudaStream_t st);
cudaError_t launch_fwd_day_soft(const SoftDayArgs &a, int grid, cudaStream_t s);
int occupancy_fwd_soft();
cudaError_t launch_soft_finalize(const double *P_nrm, int ntiles, const int32_t *graph_tile0,
                                 const int32_t *graph_ntiles, const float *m, int ldP, int T, int G,
                                 double *newRM_real, double *D_ctx, double *D_out, cudaStream_t s);
cudaError_t launch_get_lambda(const float *lam_t, const int16_t *e, const uint8_t *age,
                              GraphRef gr, const float *R, const float *S, int ldP, int t,
                              int64_t n_rows, int B, int Bp, float *out_rows, cudaStream_t s);
cudaError_t launch_philox(uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t count,
                          cudaStream_t s);
// Row order [n_rows][Bp] <-> caller order [B][n_total] (graphs concatenated, caller ids
// within each graph; B = Bp = 1 for one set per graph).
struct SetLayout {
    int B, Bp;
    int64_t n_total;
};
cudaError_t launch_rows_to_caller_i16(const int16_t *src, int16_t *dst, GraphRef gr, const int32_t *rows,
                                      const int64_t *goff, int64_t n_rows, SetLayout sl, cudaStream_t s);
cudaError_t launch_rows_to_caller_f32(const float *src, float *dst, GraphRef gr, const int32_t *rows,
                                      const int64_t *goff, int64_t n_rows, SetLayout sl, cudaStream_t s);
cudaError_t launch_caller_to_rows_i16(const int16_t *src, int16_t *dst, GraphRef gr, const int32_t *rows,
                                      const int64_t *goff, int64_t n_rows, SetLayout sl, cudaStream_t s);
int occupancy_fwd(int ntiles, bool smem_bits);
int occupancy_bwd(int mode, bool dc = false, int exit_mode = kExitBase);

}  // namespace gabm
