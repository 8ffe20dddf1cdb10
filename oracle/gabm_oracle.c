/*
 * gabm_oracle.c -- FP64 CPU oracle for the per-day step of GradABM
 * ("Differentiable Agent-based Epidemiology", Sec. 3.1 and App. A-B).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference the CUDA
 * path is checked against.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may build, load or run it; the product path
 * never calls it.  It shares no code, header, table or constant with the CUDA
 * library (it has its own Philox, its own seed selection, its own sums).
 *
 * Everything is computed in FP64 from the fp32-valued inputs, in the order the
 * paper's update states it:
 *   state of agent j at day t: (age a_j, stage d_j^t, exposure day e_j^t)  Sec. 3.1
 *   Update: Transmit if d = S, Progress if d in {E, I}                    Sec. 3.1, Eq. 2
 *   q = 1 - exp(-lambda_A), lambda_A = sum_j lambda(R^t, S_i, T_j, e_j)   Sec. 3.1, Eq. 3
 *   Bernoulli(q) draw, relaxed by Gumbel-softmax for gradients            Sec. 3.1, App. B
 *   Aggregate: deaths = m x #{R, M}                                       Sec. 3.1
 *   assumptions A1-A6 (1-day step, no same-day onward infection,
 *   no reinfection, additive transmission, no carry-over)                 App. A
 *   MSE loss on deaths                                                    Sec. 3.2, Stage 3
 *   backpropagation through the unrolled day loop                         App. B
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *   lambda_i(t) = R_t * S[a_i] * (1/Dbar) * sum_{j in N_in(i)} w_ji * c[t - e_j],
 *     with Dbar = (sum of all weights)/n and c[k] the per-day infectiousness
 *     (c[0] = 0 by A2, c[k] = 0 for k >= L = tau_EI + tau_IR and for S agents);
 *   stage from k = t - e: E if k < tau_EI, I if k < L, RM otherwise;
 *   e = NEVER (32767) marks a susceptible agent; seeds start at e = -tau_EI;
 *   daily new deaths D_t = m_t * #{i : t - e_i = L};
 *   the draw uses u = Philox4x32-10(key = seed; ctr = (id, day, instance, 0)),
 *     u = ((x0 >> 9) + 0.5) * 2^-23, infected iff u < p;
 *   the relaxed sample is y = sigmoid((logit p - logit u) / tau_g), tau_g = 1,
 *     used straight-through (hard value forward, d y_soft / d lambda backward).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NEVER 32767
#define ORC_NUM_AGES 9

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw, */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two  */
/* 32x32->64 multiplies on the counter words, key bumped by the Weyl         */
/* constants before every round after the first.                            */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* First output word of Philox at counter (id, day, inst, stream), key = seed. */
uint32_t orc_hash(uint64_t seed, uint32_t id, uint32_t day, uint32_t inst, uint32_t stream)
{
    uint32_t ctr[4] = {id, day, inst, stream};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[0];
}

/* The uniform of the relaxed Bernoulli draw: midpoint of one of 2^23 equal bins. */
double orc_uniform(uint64_t seed, uint32_t id, uint32_t day, uint32_t inst, uint32_t stream)
{
    uint32_t x0 = orc_hash(seed, id, day, inst, stream);
    return ((double)(x0 >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* ------------------------------------------------------------------------ */
/* Initial infections i^0 (Sec. 3.1 lists i^0 among theta_T): the n_seed    */
/* agents whose 64-bit key (Philox word at (id, 0, inst, 1) << 32 | id) is   */
/* smallest.  Keys are unique, so the set is well defined.                  */
/* ------------------------------------------------------------------------ */
static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

int orc_select_seeds(int64_t n, const uint32_t *orig_id, uint64_t seed, uint32_t inst,
                     int64_t n_seed, int64_t *out_rows)
{
    if (n_seed < 0 || n_seed > n) return 1;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *row_of = NULL;
    if (!keys) return 2;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t id = orig_id ? orig_id[i] : (uint32_t)i;
        keys[i] = ((uint64_t)orc_hash(seed, id, 0, inst, 1) << 32) | (uint64_t)id;
    }
    qsort(keys, (size_t)n, sizeof(uint64_t), cmp_u64);
    if (orig_id) {
        /* map original ids back to rows */
        uint32_t maxid = 0;
        for (int64_t i = 0; i < n; ++i) if (orig_id[i] > maxid) maxid = orig_id[i];
        row_of = (int64_t *)malloc(sizeof(int64_t) * ((size_t)maxid + 1));
        if (!row_of) { free(keys); return 2; }
        for (int64_t i = 0; i < n; ++i) row_of[orig_id[i]] = i;
    }
    for (int64_t s = 0; s < n_seed; ++s) {
        uint32_t id = (uint32_t)(keys[s] & 0xffffffffu);
        out_rows[s] = row_of ? row_of[id] : (int64_t)id;
    }
    free(row_of);
    free(keys);
    return 0;
}

/* Mean weighted in-degree: Dbar = (sum_p w[p]) / n, in FP64. */
double orc_mean_weighted_degree(int64_t n, const uint64_t *rowptr, const float *w)
{
    double s = 0.0;
    for (uint64_t p = 0; p < rowptr[n]; ++p) s += (double)w[p];
    return n > 0 ? s / (double)n : 0.0;
}

/* Infectiousness of an agent exposed on day e, seen on day t (0 for S agents). */
static double infectiousness(const float *c, int L, int t, int e)
{
    if (e == ORC_NEVER) return 0.0;
    int k = t - e;
    if (k < 1 || k >= L) return 0.0;
    return (double)c[k];
}

/* Progress (Sec. 3.1): stage index from days since exposure. 0=S 1=E 2=I 3=RM */
static int stage_of(int tau_EI, int L, int t, int e)
{
    if (e == ORC_NEVER) return 0;
    int k = t - e;
    if (k < tau_EI) return 1;
    if (k < L) return 2;
    return 3;
}

typedef struct {
    int64_t n;
    const uint64_t *rowptr;
    const uint32_t *col;
    const float *w;
    const uint8_t *age;
    const uint32_t *orig_id; /* NULL = identity */
} orc_graph;

typedef struct {
    int tau_EI, tau_IR;
    const float *c; /* [L] */
    uint64_t seed;
    uint32_t inst;
} orc_model;

/* Normalised neighbour sum Lam_i(t) = (1/Dbar) sum_j w_ji c[t - e_j]  (Sec. 3.1, Eq. 3). */
static double neighbour_sum(const orc_graph *g, const float *c, int L, double Dbar, int t,
                            const int16_t *e, int64_t i)
{
    double acc = 0.0;
    for (uint64_t p = g->rowptr[i]; p < g->rowptr[i + 1]; ++p)
        acc += (double)g->w[p] * infectiousness(c, L, t, e[g->col[p]]);
    return Dbar > 0.0 ? acc / Dbar : 0.0;   /* no interactions at all: no force of infection */
}

/*
 * One synchronous day t of the hard model from state e_in (Sec. 3.1, Eq. 1-3):
 * counts and new RM entries at the start of the day, then Transmit for every S
 * agent, all from the start-of-day state (A2: nobody infects on the day of
 * exposure), then newly infected agents get e = t.
 * Per S agent: Lam (normalised neighbour sum), p = 1 - exp(-lambda), u.
 * Non-S agents get Lam = p = 0 and u = -1.  *margin = min |u - p| over draws.
 */
int orc_day_hard(int64_t n, const uint64_t *rowptr, const uint32_t *col, const float *w,
                 const uint8_t *age, const uint32_t *orig_id, int tau_EI, int tau_IR,
                 const float *c, uint64_t seed, uint32_t inst, double Dbar, int t, double R_t,
                 const float *S_age, const int16_t *e_in, int16_t *e_out, double *Lam_out,
                 double *p_out, double *u_out, int64_t *newRM, int64_t counts[4], double *margin)
{
    orc_graph g = {n, rowptr, col, w, age, orig_id};
    const int L = tau_EI + tau_IR;
    int64_t cnt[4] = {0, 0, 0, 0}, nrm = 0;
    for (int64_t i = 0; i < n; ++i) {
        cnt[stage_of(tau_EI, L, t, e_in[i])] += 1;
        if (e_in[i] != ORC_NEVER && t - e_in[i] == L) nrm += 1;
    }
    double mg = INFINITY;
#pragma omp parallel for schedule(dynamic, 4096) reduction(min : mg)
    for (int64_t i = 0; i < n; ++i) {
        e_out[i] = e_in[i];
        double Lam = 0.0, p = 0.0, u = -1.0;
        if (e_in[i] == ORC_NEVER) {
            Lam = neighbour_sum(&g, c, L, Dbar, t, e_in, i);
            double lam = (double)R_t * (double)S_age[age[i]] * Lam;
            p = -expm1(-lam);
            uint32_t id = orig_id ? orig_id[i] : (uint32_t)i;
            u = orc_uniform(seed, id, (uint32_t)t, inst, 0);
            if (u < p) e_out[i] = (int16_t)t;
            double d = fabs(u - p);
            if (d < mg) mg = d;
        }
        if (Lam_out) Lam_out[i] = Lam;
        if (p_out) p_out[i] = p;
        if (u_out) u_out[i] = u;
    }
    if (newRM) *newRM = nrm;
    if (counts) for (int s = 0; s < 4; ++s) counts[s] = cnt[s];
    if (margin) *margin = mg;
    return 0;
}

/* Initial state: e0 given, or NEVER everywhere with the selected seeds at -tau_EI. */
static int initial_state(const orc_graph *g, const orc_model *md, int64_t n_seed,
                         const int16_t *e0, int16_t *e)
{
    if (e0) {
        memcpy(e, e0, sizeof(int16_t) * (size_t)g->n);
        return 0;
    }
    for (int64_t i = 0; i < g->n; ++i) e[i] = ORC_NEVER;
    int64_t *rows = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_seed > 0 ? n_seed : 1));
    if (!rows) return 2;
    int rc = orc_select_seeds(g->n, g->orig_id, md->seed, md->inst, n_seed, rows);
    if (rc == 0)
        for (int64_t s = 0; s < n_seed; ++s) e[rows[s]] = (int16_t)(-md->tau_EI);
    free(rows);
    return rc;
}

/*
 * Hard forward over days t0..T-1 (t0 = 0 unless e0 is a mid-horizon state).
 * Outputs: e_final [n]; D [T] = m_t * newRM(t); counts [T][4] (S,E,I,RM at the
 * start of each day); newRM [T]; optional e_hist [(T+1)][n] (state at the start
 * of each day, row T = final) and Lam_hist [T][n]; *margin = min |u - p|.
 * Days before t0 are left untouched in every per-day output.
 */
int orc_forward_hard(int64_t n, const uint64_t *rowptr, const uint32_t *col, const float *w,
                     const uint8_t *age, const uint32_t *orig_id, int tau_EI, int tau_IR,
                     const float *c, uint64_t seed, uint32_t inst, int T, int t0, const float *R,
                     const float *m, const float *S_age, int64_t n_seed, const int16_t *e0,
                     int16_t *e_final, double *D, int64_t *counts, int64_t *newRM,
                     int16_t *e_hist, double *Lam_hist, double *margin)
{
    orc_graph g = {n, rowptr, col, w, age, orig_id};
    orc_model md = {tau_EI, tau_IR, c, seed, inst};
    double Dbar = orc_mean_weighted_degree(n, rowptr, w);
    int16_t *cur = (int16_t *)malloc(sizeof(int16_t) * (size_t)(n > 0 ? n : 1));
    int16_t *nxt = (int16_t *)malloc(sizeof(int16_t) * (size_t)(n > 0 ? n : 1));
    if (!cur || !nxt) { free(cur); free(nxt); return 2; }
    int rc = initial_state(&g, &md, n_seed, e0, cur);
    if (rc) { free(cur); free(nxt); return rc; }
    double mg = INFINITY;
    for (int t = t0; t < T; ++t) {
        if (e_hist) memcpy(e_hist + (size_t)t * n, cur, sizeof(int16_t) * (size_t)n);
        int64_t nrm, cnt[4];
        double dmg;
        orc_day_hard(n, rowptr, col, w, age, orig_id, tau_EI, tau_IR, c, seed, inst, Dbar, t,
                     (double)R[t], S_age, cur, nxt, Lam_hist ? Lam_hist + (size_t)t * n : NULL,
                     NULL, NULL, &nrm, cnt, &dmg);
        if (dmg < mg) mg = dmg;
        if (D) D[t] = (double)m[t] * (double)nrm;
        if (newRM) newRM[t] = nrm;
        if (counts) for (int s = 0; s < 4; ++s) counts[(size_t)t * 4 + s] = cnt[s];
        int16_t *tmp = cur; cur = nxt; nxt = tmp;
    }
    if (e_hist) memcpy(e_hist + (size_t)T * n, cur, sizeof(int16_t) * (size_t)n);
    if (e_final) memcpy(e_final, cur, sizeof(int16_t) * (size_t)n);
    if (margin) *margin = mg;
    free(cur);
    free(nxt);
    return 0;
}

/* MSE on daily deaths (Sec. 3.2, Stage 3): loss = (1/T) sum (D_t - y_t)^2, gD = dloss/dD. */
void orc_mse(int T, const double *D, const double *y, double *loss, double *gD)
{
    double s = 0.0;
    for (int t = 0; t < T; ++t) {
        double d = D[t] - y[t];
        s += d * d;
        if (gD) gD[t] = 2.0 * d / (double)T;
    }
    if (loss) *loss = T > 0 ? s / (double)T : 0.0;
}

/*
 * Derivative of the relaxed sample y = sigmoid(logit p - logit u) (tau_g = 1)
 * with respect to lambda, where p = 1 - exp(-lambda) (App. B: Gumbel-softmax
 * reparametrisation).  d y/d p = y (1 - y) / (p (1 - p)), d p / d lambda = 1 - p,
 * which simplifies to u (1-u) (1-p) / (p (1-u) + (1-p) u)^2, finite at p = 0.
 */
double orc_dy_dlambda(double lam, double u)
{
    double q = exp(-lam);   /* 1 - p */
    double p = -expm1(-lam);
    double den = p * (1.0 - u) + q * u;
    return u * (1.0 - u) * q / (den * den);
}

/* Relaxed sample itself, y = p (1-u) / (p (1-u) + (1-p) u)  (tau_g = 1). */
double orc_y_soft(double lam, double u)
{
    double q = exp(-lam);
    double p = -expm1(-lam);
    return p * (1.0 - u) / (p * (1.0 - u) + q * u);
}

/*
 * Hard / straight-through adjoint (App. B: backpropagation through the
 * unrolled loop; Gumbel-softmax gradient of the draw used straight-through).
 * E[n] is the final exposure-day vector of a hard run, which determines the
 * whole trajectory (A3/A4: no reinfection): agent i is S on day t iff
 * E_i = NEVER or E_i >= t, and was newly infected on day E_i.
 *
 * Mass-flow view: n_i(t) = s_i(t) y_i(t), s_i(t+1) = s_i(t) - n_i(t),
 * x_i(t) = sum_k c[k] n_i(t - k), newRM(t) = sum_i n_i(t - L), D_t = m_t newRM(t).
 *   G_i(t)   = m_{t+L} gD_{t+L} [t+L<T] + sum_{k=1}^{L-1} c[k] gx_i(t+k) [t+k<T]
 *   dL/dy_i(t) = G_i(t) - A_i for t < E_i, G_i(t) at t = E_i or when E_i = NEVER,
 *     with A_i = G_i(E_i) the adjoint of s carried back through the y = 0 days;
 *   gl_i(t)  = dL/dy_i(t) * dy/dlambda(lambda_i(t), u_i(t))
 *   gx_i(t)  = (R_t / Dbar) sum_{j : i in N_in(j)} w_ij S[a_j] gl_j(t)   (transpose)
 *   dR_t     = sum_i gl_i(t) S[a_i] Lam_i(t);  dS_a = sum_t sum_{a_i=a} gl_i(t) R_t Lam_i(t)
 *   dm_t     = gD_t newRM(t)
 * gl_hist [T][n] (optional) receives gl_i(t) (0 for non-S agents).
 */
int orc_backward_hard(int64_t n, const uint64_t *rowptr, const uint32_t *col, const float *w,
                      const uint8_t *age, const uint32_t *orig_id, int tau_EI, int tau_IR,
                      const float *c, uint64_t seed, uint32_t inst, int T, const float *R,
                      const float *m, const float *S_age, const int16_t *E, const double *gD,
                      double *dR, double *dm, double *dS, double *gl_hist, double *dc)
{
    orc_graph g = {n, rowptr, col, w, age, orig_id};
    const int L = tau_EI + tau_IR;
    double Dbar = orc_mean_weighted_degree(n, rowptr, w);
    size_t N = (size_t)(n > 0 ? n : 1);
    double *gx = (double *)calloc((size_t)(T > 0 ? T : 1) * N, sizeof(double)); /* gx[t][i] */
    double *A = (double *)calloc(N, sizeof(double));
    double *gl = (double *)calloc(N, sizeof(double));
    double *Lam = (double *)calloc(N, sizeof(double));
    if (!gx || !A || !gl || !Lam) { free(gx); free(A); free(gl); free(Lam); return 2; }
    for (int a = 0; a < ORC_NUM_AGES; ++a) dS[a] = 0.0;

    for (int t = T - 1; t >= 0; --t) {
        double Rt = (double)R[t];
        double dRt = 0.0;
        double dSt[ORC_NUM_AGES] = {0};
#pragma omp parallel for schedule(dynamic, 4096)
        for (int64_t i = 0; i < n; ++i) {
            gl[i] = 0.0;
            Lam[i] = 0.0;
            int Ei = E[i];
            int is_S = (Ei == ORC_NEVER) || (Ei >= t);
            if (!is_S) continue;
            double G = 0.0;
            if (t + L < T) G += (double)m[t + L] * gD[t + L];
            for (int k = 1; k <= L - 1; ++k)
                if (t + k < T) G += (double)c[k] * gx[(size_t)(t + k) * N + (size_t)i];
            double dLdy;
            if (Ei == t) { A[i] = G; dLdy = G; }
            else if (Ei == ORC_NEVER) dLdy = G;
            else dLdy = G - A[i];
            Lam[i] = neighbour_sum(&g, c, L, Dbar, t, E, i);
            double lam = Rt * (double)S_age[age[i]] * Lam[i];
            uint32_t id = orig_id ? orig_id[i] : (uint32_t)i;
            double u = orc_uniform(seed, id, (uint32_t)t, inst, 0);
            gl[i] = dLdy * orc_dy_dlambda(lam, u);
        }
        for (int64_t i = 0; i < n; ++i) {
            if (gl[i] == 0.0) continue;
            dRt += gl[i] * (double)S_age[age[i]] * Lam[i];
            dSt[age[i]] += gl[i] * Rt * Lam[i];
        }
        /* transpose of the pull sum: row j's in-neighbour i receives w_ij S[a_j] gl_j */
        double *gxt = gx + (size_t)t * N;
        for (int64_t j = 0; j < n; ++j) {
            if (gl[j] == 0.0) continue;
            double coef = Rt * (double)S_age[age[j]] * gl[j] / Dbar;
            for (uint64_t p = rowptr[j]; p < rowptr[j + 1]; ++p)
                gxt[col[p]] += (double)w[p] * coef;
        }
        dR[t] = dRt;
        for (int a = 0; a < ORC_NUM_AGES; ++a) dS[a] += dSt[a];
        int64_t nrm = 0;
        for (int64_t i = 0; i < n; ++i)
            if (E[i] != ORC_NEVER && t - E[i] == L) nrm += 1;
        dm[t] = gD[t] * (double)nrm;
        if (gl_hist) memcpy(gl_hist + (size_t)t * n, gl, sizeof(double) * (size_t)n);
    }
    /* Adjoint of the infectiousness table: x_i(t) = sum_k c[k] n_i(t - k) with the
     * hard n_i(d) = [E_i = d] (seeds at their negative exposure day), so
     * dL/dc[k] = sum_i gx_i(E_i + k) over 0 <= E_i + k < T.  c[0] is fixed at 0 (A2). */
    if (dc) {
        for (int k = 0; k < L; ++k) dc[k] = 0.0;
        for (int k = 1; k <= L - 1; ++k) {
            double acc = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                if (E[i] == ORC_NEVER) continue;
                int t = (int)E[i] + k;
                if (t >= 0 && t < T) acc += gx[(size_t)t * N + (size_t)i];
            }
            dc[k] = acc;
        }
    }
    free(gx); free(A); free(gl); free(Lam);
    return 0;
}

/*
 * SOFT relaxation with fixed noise: every draw uses the relaxed value
 * y = y_soft(lambda, u) instead of the hard indicator, with the mass-flow
 * state s (S mass) and n (newly exposed mass per day).  Smooth in the
 * parameters, used for finite-difference checks of the adjoint.
 * Initial state from e0 (seed agents at a negative exposure day, s = 0) or
 * from the seed selection.
 * Histories (all [T][n] except s_hist [T+1][n]): s, y, dy/dlambda, Lam.
 * newRM [T] (real-valued) and D [T].
 */
int orc_forward_soft(int64_t n, const uint64_t *rowptr, const uint32_t *col, const float *w,
                     const uint8_t *age, const uint32_t *orig_id, int tau_EI, int tau_IR,
                     const float *c, uint64_t seed, uint32_t inst, int T, const float *R,
                     const float *m, const float *S_age, int64_t n_seed, const int16_t *e0,
                     double *D, double *newRM, double *s_hist, double *y_hist,
                     double *dydl_hist, double *Lam_hist)
{
    orc_graph g = {n, rowptr, col, w, age, orig_id};
    orc_model md = {tau_EI, tau_IR, c, seed, inst};
    const int L = tau_EI + tau_IR;
    size_t N = (size_t)(n > 0 ? n : 1);
    double Dbar = orc_mean_weighted_degree(n, rowptr, w);
    int16_t *e = (int16_t *)malloc(sizeof(int16_t) * N);
    /* nh[(d + L) * N + i] = n_i(d) for d in [-L, T-1] */
    double *nh = (double *)calloc((size_t)(T + L) * N, sizeof(double));
    double *s = (double *)malloc(sizeof(double) * N);
    double *x = (double *)malloc(sizeof(double) * N);
    if (!e || !nh || !s || !x) { free(e); free(nh); free(s); free(x); return 2; }
    int rc = initial_state(&g, &md, n_seed, e0, e);
    if (rc) { free(e); free(nh); free(s); free(x); return rc; }
    for (int64_t i = 0; i < n; ++i) {
        if (e[i] == ORC_NEVER) { s[i] = 1.0; continue; }
        s[i] = 0.0;
        if (e[i] < -L || e[i] >= 0) { free(e); free(nh); free(s); free(x); return 1; }
        nh[(size_t)(e[i] + L) * N + (size_t)i] = 1.0;
    }
    for (int t = 0; t < T; ++t) {
        if (s_hist) memcpy(s_hist + (size_t)t * N, s, sizeof(double) * N);
        double nrm = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double xi = 0.0;
            for (int k = 1; k <= L - 1; ++k)
                xi += (double)c[k] * nh[(size_t)(t - k + L) * N + (size_t)i];
            x[i] = xi;
            nrm += nh[(size_t)(t - L + L) * N + (size_t)i];
        }
        if (newRM) newRM[t] = nrm;
        if (D) D[t] = (double)m[t] * nrm;
        for (int64_t i = 0; i < n; ++i) {
            double acc = 0.0;
            for (uint64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
                acc += (double)w[p] * x[col[p]];
            double Lam = Dbar > 0.0 ? acc / Dbar : 0.0;
            double lam = (double)R[t] * (double)S_age[age[i]] * Lam;
            uint32_t id = orig_id ? orig_id[i] : (uint32_t)i;
            double u = orc_uniform(seed, id, (uint32_t)t, inst, 0);
            double y = orc_y_soft(lam, u);
            double ni = s[i] * y;
            nh[(size_t)(t + L) * N + (size_t)i] = ni;
            if (y_hist) y_hist[(size_t)t * N + (size_t)i] = y;
            if (dydl_hist) dydl_hist[(size_t)t * N + (size_t)i] = orc_dy_dlambda(lam, u);
            if (Lam_hist) Lam_hist[(size_t)t * N + (size_t)i] = Lam;
        }
        for (int64_t i = 0; i < n; ++i) s[i] -= nh[(size_t)(t + L) * N + (size_t)i];
    }
    if (s_hist) memcpy(s_hist + (size_t)T * N, s, sizeof(double) * N);
    free(e); free(nh); free(s); free(x);
    return 0;
}

/*
 * Adjoint of the relaxed model given its per-day histories (s, y, dy/dlambda,
 * Lam).  Reverse-mode of: n = s y, s' = s - n, x(t) = sum_k c[k] n(t-k),
 * lambda = R S Lam, Lam = (1/Dbar) sum_j w_ji x_j, D_t = m_t sum_i n_i(t-L):
 *   dL/dy_i(t) = s_i(t) (G_i(t) - dL/ds_i(t+1))
 *   dL/ds_i(t) = y_i(t) G_i(t) + (1 - y_i(t)) dL/ds_i(t+1),   dL/ds(T) = 0
 * with G, gx, dR, dS, dm as in the hard adjoint.  Evaluated at hard values
 * (s, y in {0,1}, dy/dlambda straight-through) it is the hard/ST adjoint.
 * newRM [T] is the (real-valued) count used for dm.
 */
int orc_backward_soft(int64_t n, const uint64_t *rowptr, const uint32_t *col, const float *w,
                      const uint8_t *age, int tau_EI, int tau_IR, const float *c, int T,
                      const float *R, const float *m, const float *S_age, const double *gD,
                      const double *s_hist, const double *y_hist, const double *dydl_hist,
                      const double *Lam_hist, const double *newRM, double *dR, double *dm,
                      double *dS, const int16_t *e0, double *dc)
{
    const int L = tau_EI + tau_IR;
    size_t N = (size_t)(n > 0 ? n : 1);
    double Dbar = orc_mean_weighted_degree(n, rowptr, w);
    double *gx = (double *)calloc((size_t)(T > 0 ? T : 1) * N, sizeof(double));
    double *ds_next = (double *)calloc(N, sizeof(double));
    double *gl = (double *)calloc(N, sizeof(double));
    if (!gx || !ds_next || !gl) { free(gx); free(ds_next); free(gl); return 2; }
    for (int a = 0; a < ORC_NUM_AGES; ++a) dS[a] = 0.0;
    for (int t = T - 1; t >= 0; --t) {
        double Rt = (double)R[t];
        double dRt = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            size_t ti = (size_t)t * N + (size_t)i;
            double G = 0.0;
            if (t + L < T) G += (double)m[t + L] * gD[t + L];
            for (int k = 1; k <= L - 1; ++k)
                if (t + k < T) G += (double)c[k] * gx[(size_t)(t + k) * N + (size_t)i];
            double si = s_hist[ti], yi = y_hist[ti];
            double dLdy = si * (G - ds_next[i]);
            double ds_now = yi * G + (1.0 - yi) * ds_next[i];
            ds_next[i] = ds_now;
            gl[i] = dLdy * dydl_hist[ti];
            dRt += gl[i] * (double)S_age[age[i]] * Lam_hist[ti];
            dS[age[i]] += gl[i] * Rt * Lam_hist[ti];
        }
        double *gxt = gx + (size_t)t * N;
        for (int64_t j = 0; j < n; ++j) {
            double coef = Rt * (double)S_age[age[j]] * gl[j] / Dbar;
            if (coef == 0.0) continue;
            for (uint64_t p = rowptr[j]; p < rowptr[j + 1]; ++p)
                gxt[col[p]] += (double)w[p] * coef;
        }
        dR[t] = dRt;
        dm[t] = gD[t] * newRM[t];
    }
    /* Adjoint of the infectiousness table: dL/dc[k] = sum_t sum_i n_i(t - k) gx_i(t), with
     * n_i(d) = s_i(d) y_i(d) for d >= 0 and, before day 0, the seeds' unit mass at their
     * exposure day e0_i < 0 (no seeds when e0 is NULL).  c[0] is fixed at 0 (A2). */
    if (dc) {
        for (int k = 0; k < L; ++k) dc[k] = 0.0;
        for (int k = 1; k <= L - 1; ++k) {
            double acc = 0.0;
            for (int t = 0; t < T; ++t) {
                const int d = t - k;
                for (int64_t i = 0; i < n; ++i) {
                    double ni;
                    if (d >= 0) ni = s_hist[(size_t)d * N + (size_t)i] * y_hist[(size_t)d * N + (size_t)i];
                    else ni = (e0 && e0[i] == d) ? 1.0 : 0.0;
                    if (ni != 0.0) acc += ni * gx[(size_t)t * N + (size_t)i];
                }
            }
            dc[k] = acc;
        }
    }
    free(gx); free(ds_next); free(gl);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* u for many agent ids at one (day, instance, stream); test convenience. */
void orc_uniform_array(uint64_t seed, int64_t count, const uint32_t *ids, uint32_t day,
                       uint32_t inst, uint32_t stream, double *out)
{
    for (int64_t i = 0; i < count; ++i) out[i] = orc_uniform(seed, ids[i], day, inst, stream);
}
