// sirs.cuh -- day kernels of SIRS reinfection (one set per graph, hard model, lambda store).
//
// App. A's A4 (no infection from RM) relaxed: an agent exposed on day d is in E for
// k = t - d < tau_EI, in I for k < L, in RM for k < L + tau_RS ("cycle"), and susceptible
// again from k = cycle on.  The state is the last exposure day (Sec. 3.1's e^t).  The
// final state no longer encodes the trajectory, so the forward appends every exposure to
// a per-agent history, which the reverse sweep reads:
//   hist [n_rows][H] int16   exposure days in order (a seed's initial exposure first)
//   cnt  [n_rows]    u16     entries used (H <= GABM_MAX_DAYS / 3 + 2 < 65536)
//   Gh   [n_rows][H] f32     G at each exposure day (that day's scale), written by the sweep
//   Lh   [n_rows][H] f32     G's own-day terms at each exposure (G without the return term)
// Adjoint (straight-through, App. B): with B_i(t) = dL/ds_i(t), which equals G_i at the
// agent's first exposure on or after t (0 if none),
//   G_i(t) = sum_{k=1}^{L-1} c[k] gx_i(t+k) + m_{t+L} gD_{t+L} + B_i(t + cycle)
//   dL/dy_i(t) = G_i(t) - B_i(t+1)  for rows susceptible on day t,
// evaluated as the own-day terms of G_i(t) minus those of the next exposure when that falls
// within `cycle` days (the return terms cancel exactly; see k_bwd_day_sirs).
#pragma once
#include "gabm_internal.cuh"

namespace gabm {

struct SirsFwdArgs {
    Sell m;                     // in-edges
    const uint8_t *age;
    GraphRef gr;
    int16_t *e;                 // last exposure day
    int16_t *hist;
    uint16_t *cnt;
    int H;
    float *lam_out;             // day-t slice of the lambda store
    const float *R, *S;         // [I][ldP], [I][9]
    int ldP;
    int32_t *counts, *newRM;    // [I][ldP][4], [I][ldP]
    const uint32_t *bits_cur;   // rows infectious on day t
    uint32_t *bits_next;        // the same for day t + 1 (written here)
    const uint8_t *flag_cur;    // rows with an infectious in-neighbour on day t (or nullptr: all)
    uint8_t *flag_next, *flag_clear;   // day t + 1's flags (set here), day t + 2's (cleared here)
    Sell m_out;                 // out-edges
    int ntiles, t, tau_EI, L, cycle;
    uint64_t seed;
    float c[kMaxL];
};

struct SirsBwdArgs {
    Sell m;                     // out-edges (the in-edges when the weights are symmetric)
    const uint8_t *age;
    GraphRef gr;
    const int16_t *E;           // final state (kPad marks padding rows)
    const int16_t *hist;
    const uint16_t *cnt;
    int H;
    float *Gh, *Lh;
    const float *lam_t;         // stored normalised sums of day t
    const float *r_next;        // r of day t + 1
    float *r_cur;               // r of day t (0 for rows not susceptible on day t)
    float *ring;                // [L-1][n_rows] gx of the next L-1 days
    size_t ring_stride;
    int ring_slot[kMaxL];       // slot of day t + k
    const float *R, *m_t, *S;
    const double *gD;
    int ldP;
    double *P_t;                // [ntiles][9] per-tile sums of gl * Lam by age
    int32_t *newRM;             // [I][ldP] recounted
    int32_t *sig, *emax;        // [G][ld_sig] per-day scale exponents
    int ld_sig;
    int ntiles, t, T, tau_EI, L, cycle;
    uint64_t seed;
    float c[kMaxL];
};

cudaError_t launch_sirs_hist_init(const int16_t *e, int64_t n_rows, int H, int16_t *hist, uint16_t *cnt,
                                  cudaStream_t s);
cudaError_t launch_fwd_day_sirs(const SirsFwdArgs &a, int grid, cudaStream_t s);
cudaError_t launch_bwd_day_sirs(const SirsBwdArgs &a, int grid, cudaStream_t s);
int occupancy_sirs(bool backward);

}  // namespace gabm
