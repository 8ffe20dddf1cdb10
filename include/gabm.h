/*
 * gabm.h -- C ABI of the GB300 library for the per-day step of GradABM
 * ("Differentiable Agent-based Epidemiology", arXiv 2207.09714).
 *
 * The library simulates the hard (sampled) epidemic model of Sec. 3.1 over T
 * days on a contact graph and computes the straight-through adjoint of an MSE
 * loss on daily deaths with respect to the per-day transmissibility R_t, the
 * per-day mortality m_t and the per-age susceptibility S_a (Sec. 3.2, App. B).
 *
 * Model (Sec. 3.1, Eq. 1-3; assumptions A1-A6 of App. A):
 *   agent state: age bin a_i in 0..8, exposure day e_i (GABM_NEVER = susceptible);
 *   stage on day t from k = t - e_i: E if k < tau_EI, I if k < L, RM otherwise,
 *     L = tau_EI + tau_IR (Progress is deterministic, Sec. 3.1 and App. B);
 *   Transmit for susceptible i:
 *     lambda_i(t) = R_t * S[a_i] * (1/Dbar) * sum_{j in N_in(i)} w_ji * c[t - e_j],
 *     Dbar = (sum of all weights) / n, c[0] = 0 (A2), c[k] = 0 for k >= L;
 *     p_i = 1 - exp(-lambda_i)  (Eq. 3, one-day step A1);
 *     infected iff u_i < p_i, u_i from Philox4x32-10 keyed (seed; agent, day,
 *     instance, 0), u = ((x0 >> 9) + 0.5) * 2^-23; newly infected get e_i = t;
 *   Aggregate: daily new deaths D_t = m_t * #{i : t - e_i = L};
 *   initial infections: the n_seed agents with the smallest Philox key at
 *     (agent, 0, instance, 1), placed at e = -tau_EI (they start in I on day 0);
 *   backward: Gumbel-softmax relaxation y = sigmoid(logit p - logit u) used
 *     straight-through, adjoint of the unrolled day loop (App. B).
 *
 * Conventions
 *   - Status codes are returned by every call; no exception crosses the ABI.
 *     gabm_last_error() gives a message for the last failing call on a ctx.
 *   - "Instances": num_graphs graphs x sets_per_graph parameter sets; instance
 *     index = graph * sets_per_graph + set.  Per-instance arrays are laid out
 *     [instance][...] row-major.
 *   - Agent ids in and out are the caller's ids within each graph.
 *   - A mem_space argument (GABM_DEVICE / GABM_HOST) says where every array
 *     argument of that call lives.  Device work is enqueued on the ctx stream;
 *     with GABM_DEVICE the call returns without waiting for it, with GABM_HOST
 *     the call copies through ctx-owned device buffers and synchronises the
 *     stream before it returns.
 *   - A ctx owns all of its device memory and is not thread-safe.
 */
#ifndef GABM_H
#define GABM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GABM_OK = 0,
    GABM_EINVAL = 1,       /* invalid argument or input data (nothing was changed) */
    GABM_ENOMEM = 2,       /* device allocation failed (ctx left usable, or not created) */
    GABM_ECUDA = 3,        /* a CUDA runtime call failed */
    GABM_ESTATE = 4,       /* call out of order (e.g. backward without a matching forward) */
    GABM_ETIMEOUT = 5,     /* reserved: a bounded device wait gave up */
    GABM_ECANCELLED = 6,   /* reserved: cancelled between days */
    GABM_EUNSUPPORTED = 7  /* valid request this build does not implement */
} gabm_status;

enum { GABM_DEVICE = 0, GABM_HOST = 1 };
enum { GABM_HARD_ST = 0, GABM_SOFT = 1 };
/* Where the backward gets lambda_i(t): stored by the forward (4 bytes per
 * susceptible agent-day), or recomputed from the final state.  In the hard
 * model the final exposure-day vector determines every day's state (A3/A4: no
 * reinfection), so recomputation needs no intermediate checkpoints. */
enum { GABM_STORE_LAMBDA = 0, GABM_RECOMPUTE = 1 };
/* Device layout of the agents.  GABM_ORDER_BFS relabels the agents of each
 * graph in breadth-first order of the contact graph so that an agent's
 * neighbours sit close together in memory (gathers hit fewer cache lines).
 * GABM_ORDER_COMMUNITY lays out densely connected groups (found by label
 * propagation over the contacts) as consecutive rows, groups in breadth-first
 * order: on contact graphs made of cliques (households, schools, workplaces)
 * with random contacts on top, more of an agent's neighbours sit nearby than in
 * breadth-first order.  It costs a few passes over the edges at creation.
 * Results do not depend on the layout beyond fp32 summation order: the Philox
 * draws and every input and output stay keyed by the caller's agent ids, and
 * the aggregation is permutation invariant (Sec. 2.3, App. A). */
enum { GABM_ORDER_INPUT = 0, GABM_ORDER_BFS = 1, GABM_ORDER_COMMUNITY = 2 };

#define GABM_NEVER 32767     /* exposure day of a susceptible agent */
#define GABM_NUM_AGES 9      /* age bins 0-10, 11-20, ..., 71-80, 80+ (Sec. 3.1) */
#define GABM_MAX_L 32        /* upper bound on tau_EI + tau_IR */
#define GABM_MAX_DAYS 16384  /* upper bound on T (exposure days are int16) */

typedef struct gabm_ctx gabm_ctx;

/* One contact graph in destination-sorted CSR form (Sec. 3.1: interaction
 * network as a sparse adjacency matrix; App. A: sparse, small-world).
 * Row i lists the in-neighbours j of agent i; w[p] is the weight of the
 * interaction from j into i.  Requirements (checked, GABM_EINVAL otherwise):
 * rowptr[0] = 0, non-decreasing, rowptr[n] = nnz; col < n; w finite and >= 0;
 * age <= 8.  Self loops and repeated pairs are allowed and harmless (an agent
 * is never infectious while susceptible; repeated pairs add).  n < 2^31 and
 * nnz < 2^32 per graph.  Arrays are read during gabm_create only. */
typedef struct {
    int64_t n, nnz;
    const uint64_t *rowptr;  /* [n+1] */
    const uint32_t *col;     /* [nnz] */
    const float *w;          /* [nnz] */
    const uint8_t *age;      /* [n]   */
    int mem_space;           /* GABM_HOST or GABM_DEVICE */
} gabm_graph_desc;

/* Model constants fixed for the life of a ctx (Sec. 3.1: theta_P stage times,
 * T_s stage transmissibility folded into c; App. D: infectiousness profile). */
typedef struct {
    int tau_EI, tau_IR;   /* days E->I and I->RM; 1 <= each, L = sum <= GABM_MAX_L */
    const float *c;       /* host [L]: infectiousness by days since exposure, c[0] = 0, c >= 0
                           * (with tau_IM > 0: L = tau_EI + max(tau_IR, tau_IM)) */
    float gumbel_tau;     /* relaxation temperature; this build supports 1.0 */
    int relax_mode;       /* GABM_HARD_ST, or GABM_SOFT (sets_per_graph = 1 and GABM_STORE_LAMBDA):
                           * the fixed-noise soft relaxation -- every agent draws every day
                           * with y = sigmoid(logit p - logit u) and moves mass s y from S to
                           * E; smooth in the parameters (finite-difference checks of the
                           * adjoint).  Its state is masses: gabm_get_state / gabm_set_state
                           * return GABM_EUNSUPPORTED and gabm_forward's counts must be NULL. */
    int lambda_policy;    /* GABM_STORE_LAMBDA or GABM_RECOMPUTE */
    uint64_t seed;        /* Philox key */
    int agent_order;      /* GABM_ORDER_INPUT, _BFS or _COMMUNITY (device layout only) */
    int tau_IM;           /* 0: the single RM exit at L with expected deaths D_t = m_t newRM(t)
                           * (Sec. 3.1 Aggregate).  > 0: the sampled R/M split -- the mortality
                           * stage M with its own I->M time (Sec. 3.1 lists tau_IM in theta_P):
                           * an agent exposed on day d draws its fate on its I-entry day
                           * t_I = d + tau_EI (day 0 for exposures before -tau_EI): M iff v <
                           * m_{t_I}, v the Philox uniform of (caller id, t_I, instance, stream 1).
                           * It is infectious for 1 <= t - d < tau_EI + tau_IR (R) or
                           * tau_EI + tau_IM (M), and D_t counts the M entries
                           * (t - d = tau_EI + tau_IM).  The adjoint relaxes the fate draw like the
                           * infection draw (straight-through, tau = 1), so dm comes from the
                           * fates.  Needs GABM_HARD_ST, sets_per_graph = 1, GABM_STORE_LAMBDA and
                           * a one-hop graph; no table adjoint (GABM_EUNSUPPORTED otherwise). */
    const float *p_IR;    /* NULL: every agent stays tau_IR days in I.  Else host [tau_IR], the pmf
                           * of a per-agent I-stage duration (stochastic progression, Sec. 6):
                           * p_IR[j-1] = P(j days), finite and >= 0 with some mass.  An exposure
                           * on day d stays j days in I, j the first with u < F_j (F_j = p_IR[0] +
                           * ... + p_IR[j-1] summed in order in double; tau_IR if none), u the
                           * Philox uniform of (caller id, max(d, 0), instance, stream 2); it is
                           * infectious for 1 <= t - d < tau_EI + j and enters RM at tau_EI + j,
                           * where the expected deaths m_t newRM(t) count it.  The adjoint takes
                           * each row's drawn window.  Same restrictions as tau_IM > 0, and not
                           * together with it (GABM_EUNSUPPORTED).  Read during gabm_create only. */
    int tau_RS;           /* 0: no reinfection (A4 of App. A).  > 0: SIRS reinfection, A4 relaxed --
                           * an agent returns to S tau_RS days after entering RM (tau_EI + tau_IR +
                           * tau_RS days after its exposure) and can be exposed again; the state is
                           * the last exposure day, and every exposure is recorded for the
                           * backward.  D_t = m_t newRM(t) counts every I -> RM transition.  Needs
                           * GABM_HARD_ST, sets_per_graph = 1, GABM_STORE_LAMBDA, a one-hop graph,
                           * tau_IM = 0 and p_IR = NULL; gabm_set_state and the table adjoint return
                           * GABM_EUNSUPPORTED. */
} gabm_model_desc;

/* Build a ctx: validates and copies the graphs (GABM_EINVAL on bad data, before
 * any CUDA call), builds the device CSR and its transpose (aliased when the
 * weights are symmetric), and allocates the per-agent state.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  num_graphs >= 1 graphs are
 * concatenated block-diagonally (uneven batch); sets_per_graph = B in 1..64
 * parameter sets share each graph (instance i = graph * B + set; B > 1 with
 * GABM_RECOMPUTE needs symmetric weights, else GABM_EUNSUPPORTED).  On success *out
 * owns everything; release with gabm_destroy. */
gabm_status gabm_create(const gabm_graph_desc *graphs, int num_graphs, int sets_per_graph,
                        const gabm_model_desc *model, void *cuda_stream, gabm_ctx **out);

/* An agent-location graph, the heterogeneous contact structure of GradABM-JUNE
 * (Sec. 6): agent i attends location loc[p] with weight w[p] for p in
 * [rowptr[i], rowptr[i+1]).  Two agents interact through every location they
 * share, so the model is that of Sec. 3.1 (Eq. 3) on the agent graph with pair
 * weights W_ij = sum_l w_il w_jl (i != j), and Dbar is W's mean weighted degree.
 * Each day is computed in two hops over the attendance entries -- location
 * pressures P_l(t) = sum_{j at l} w_jl x_j(t), then
 * lambda_i(t) = R_t S[a_i] (1/Dbar) sum_l w_il P_l(t) -- and the adjoint likewise,
 * so W, whose size grows with the square of the location sizes, is never formed.
 * (An agent's own term drops out: x_i = 0 while i is susceptible.)  Host memory. */
typedef struct {
    int64_t n_agents, n_locations, nnz;
    const uint64_t *rowptr;  /* [n_agents+1] */
    const uint32_t *loc;     /* [nnz] location of each attendance, < n_locations */
    const float *w;          /* [nnz] attendance weight, finite and >= 0 (repeats add) */
    const uint8_t *age;      /* [n_agents] age bins 0..8 */
} gabm_bipartite_desc;

/* Build a ctx over num_graphs >= 1 agent-location graphs (copied; GABM_EINVAL on
 * bad data, before any CUDA call).  It then works as a gabm_create ctx of that many
 * graphs and one set per graph (instance g = graph g, with its own Dbar): agents are
 * the rows, in input order within degree windows (agent_order is not used), and no
 * location is shared between graphs.  The model must use GABM_HARD_ST and
 * GABM_STORE_LAMBDA (GABM_EUNSUPPORTED otherwise). */
gabm_status gabm_create_bipartite(const gabm_bipartite_desc *graphs, int num_graphs,
                                  const gabm_model_desc *model, void *cuda_stream, gabm_ctx **out);

/* The device order gabm_create gives one graph's agents, computed on the host (no GPU
 * work for host arrays): order_out[r] (n entries, caller-allocated host memory) is the
 * caller's id of device row r -- the agent order (GABM_ORDER_*), then degree windows of
 * 1024 rows, then, when sets_per_graph == 1, rows of more than 128 entries grouped 32 to
 * a tile.  Always a permutation of 0..n-1.  GABM_EINVAL on a bad graph (gabm_create's
 * checks), an unknown order, sets_per_graph < 1 or a NULL order_out. */
gabm_status gabm_agent_layout(const gabm_graph_desc *graph, int agent_order, int sets_per_graph,
                              uint32_t *order_out);

/* Forward over days t0..T-1 (Sec. 3.1, Eq. 1-3, K = T steps).  t0 = 0 after
 * create (seeding from n_seed), or the day given to the last gabm_set_state.
 *   R      [I][T] float  transmissibility R_t per instance
 *   m      [I][T] float  mortality m_t per instance
 *   S_age  [I][9] float  susceptibility per age bin
 *   n_seed [I]    int32  initial infections per instance (HOST memory always;
 *                        ignored when resuming from gabm_set_state)
 *   D      [I][T] double out: daily new deaths D_t = m_t * newRM(t) (days >= t0)
 *   counts [I][T][4] int32 out or NULL: S, E, I, RM at the start of each day
 * 1 <= T <= GABM_MAX_DAYS.  The first call with a larger T grows the per-day
 * buffers (an allocation). */
gabm_status gabm_forward(gabm_ctx *ctx, int T, const float *R, const float *m, const float *S_age,
                         const int32_t *n_seed, double *D, int32_t *counts, int mem_space);

/* MSE on daily deaths of the last forward (Sec. 3.2, Stage 3):
 *   loss[i] = (1/T) sum_t (D[i][t] - y[i][t])^2,  gD[i][t] = 2 (D[i][t] - y[i][t]) / T.
 *   y [I][T] double in; loss [I] double out; gD [I][T] double out.
 * GABM_ESTATE if no forward has run. */
gabm_status gabm_mse_loss(gabm_ctx *ctx, const double *y, double *loss, double *gD, int mem_space);

/* Replace the infectiousness table c [L] (host floats; c[0] = 0, every entry finite
 * and >= 0, as at creation) for the forwards that follow, e.g. between the steps of a
 * calibration that learns the stage factors or the profile behind c.  Waits for the
 * ctx stream.  The last trajectory used the old table, so gabm_backward returns
 * GABM_ESTATE until the next gabm_forward.  GABM_EINVAL for a NULL or invalid table. */
gabm_status gabm_set_infectiousness(gabm_ctx *ctx, const float *c);

/* Straight-through adjoint of the last forward (App. B): given gD = dL/dD_t
 * [I][T] (double), writes dR [I][T], dm [I][T] and dS_age [I][9] (double).
 * Cross-agent and cross-day sums are FP64 in a fixed order (bitwise
 * reproducible).  GABM_ESTATE without a forward (or set_state) of the same T,
 * with GABM_STORE_LAMBDA when the stored lambdas do not cover days 0..T-1, or with
 * several sets per graph when the last forward did not start at day 0.  Several sets
 * under GABM_RECOMPUTE: each day's lambda is summed again from the final state over the
 * same entries in the same order as the forward, so the result is bitwise that of
 * GABM_STORE_LAMBDA.  The reverse sweep runs in fp32 at a power-of-two scale per day
 * that follows the adjoint's growth (FP64 for the sums); each m_t gD_t enters it as an
 * fp32 value, so |gD| must stay below about 1e30 (a loss gradient of that size is not
 * a meaningful input; beyond the fp32 range the results are not finite). */
gabm_status gabm_backward(gabm_ctx *ctx, const double *gD, double *dR, double *dm,
                          double *dS_age, int mem_space);

/* gabm_backward that also writes dc [I][L] (double): the gradient of the loss with
 * respect to the infectiousness table c[k] of the model (lambda is linear in each
 * neighbour's c[t - e_j], Sec. 3.1 Eq. 3; adjoint of App. B).  With the hard
 * trajectory, dc[i][k] = sum_j gx_j(E_j + k) over agents j exposed on day E_j (seeds at
 * their negative exposure day) and days 0 <= E_j + k < T, where gx_j(t) is the adjoint of
 * agent j's infectiousness on day t.  dc[i][0] = 0 (c[0] = 0 is fixed, A2 of App. A).
 * Gradients of stage factors or profile parameters that define c (T_E, T_I, iota)
 * follow by the chain rule on the caller's side.  With several sets per graph, each
 * instance i = graph * sets_per_graph + set gets its own dc[i].  Under GABM_SOFT the
 * exposed mass replaces the indicator: dc[i][k] = sum_t sum_j n_j(t - k) gx_j(t) with
 * n_j(d) = s_j(d) y_j(d), the seeds' unit mass before day 0.  Same preconditions as
 * gabm_backward; GABM_EINVAL if dc is NULL; GABM_EUNSUPPORTED for several sets per graph
 * under GABM_RECOMPUTE. */
gabm_status gabm_backward_table(gabm_ctx *ctx, const double *gD, double *dR, double *dm,
                                double *dS_age, double *dc, int mem_space);

/* Current exposure-day vector e [sets_per_graph][n_total] (int16; per set, the
 * graphs' agents concatenated in graph order, caller ids within each graph).
 * After a forward over T days this is the final state. */
gabm_status gabm_get_state(gabm_ctx *ctx, int16_t *e_out, int mem_space);

/* Replace the state with e [sets_per_graph][n_total] as the start of day `day` (0 <= day <=
 * GABM_MAX_DAYS).  The next gabm_forward then runs days day..T-1 without
 * seeding; a gabm_forward with T == day only records its parameters, after
 * which gabm_backward (GABM_RECOMPUTE, one set per graph) replays the trajectory e
 * encodes.  With several sets per graph a backward needs a forward over days 0..T-1
 * (GABM_ESTATE after a forward from a set state at day > 0).  GABM_EUNSUPPORTED under
 * SIRS reinfection (tau_RS > 0), whose trajectory the last exposure days do not fix.
 * Values must be GABM_NEVER or in [-GABM_MAX_L, day). */
gabm_status gabm_set_state(gabm_ctx *ctx, int day, const int16_t *e_in, int mem_space);

/* lambda_i(t) for day t, [sets_per_graph][n_total] float, 0 for agents not
 * susceptible on day t (GABM_SOFT: 0 for the seeds, which hold no susceptible mass).
 * GABM_STORE_LAMBDA: the stored value; t must have been run by the last forward.
 * GABM_RECOMPUTE: recomputed from the current state, which fixes every earlier day
 * (no reinfection); 0 <= t < the last forward's T; one-hop graphs of one set per graph
 * (GABM_EUNSUPPORTED otherwise).  GABM_ESTATE otherwise. */
gabm_status gabm_get_lambda(gabm_ctx *ctx, int t, float *lam_out, int mem_space);

/* Kernel schedule of a ctx.  Schedules change how rows and parameter sets map
 * onto lanes, never what is summed or in which order, so every schedule gives
 * bitwise the same results.
 *   fwd_sets_per_lane, bwd_sets_per_lane: sets_per_graph > 1 only -- each lane
 *     carries 2, 4 or 8 parameter sets of a row (Bp / that many lanes share a
 *     row, Bp = sets_per_graph rounded up to a power of two; at most Bp);
 *   fwd_smem_bitmap: sets_per_graph == 1 only -- 1 keeps the day's bitmap of
 *     infectious agents in shared memory (when it fits), 0 reads it through L1;
 *   bwd_sets_per_launch: sets_per_graph > 1 only -- the backward runs a row's Bp
 *     sets in launches of this many (a power of two dividing Bp, at least
 *     bwd_sets_per_lane; 0 on input means Bp), so that the coefficients one
 *     launch gathers can stay in L2.
 * Fields that do not apply are reported as 0 and ignored on input. */
typedef struct {
    int fwd_sets_per_lane;
    int bwd_sets_per_lane;
    int fwd_smem_bitmap;
    int bwd_sets_per_launch;
} gabm_schedule;

gabm_status gabm_get_schedule(const gabm_ctx *ctx, gabm_schedule *out);
/* GABM_EINVAL (schedule unchanged) for a value this build has no kernel for. */
gabm_status gabm_set_schedule(gabm_ctx *ctx, const gabm_schedule *sched);

/* Autotuner: times every schedule this build has for the ctx on the ctx's own
 * workload -- the last forward's T, parameters and seeds, and a backward over
 * the same days -- `repetitions` times each (>= 1), keeps the fastest forward
 * and backward schedules, and re-runs that forward so the state, the stored
 * lambdas and D are as before the call (the trajectory does not depend on the
 * schedule).  Needs a preceding gabm_forward that started from seeding
 * (GABM_ESTATE otherwise).  Synchronises the ctx stream. */
gabm_status gabm_autotune(gabm_ctx *ctx, int repetitions);

/* Device bytes the ctx holds now and at most so far. */
gabm_status gabm_mem_stats(const gabm_ctx *ctx, size_t *current, size_t *peak);

/* Kernel launches this ctx has issued since creation. */
uint64_t gabm_launch_count(const gabm_ctx *ctx);

/* Per-kind kernel timing with CUDA events recorded on the ctx stream around
 * each launch of that kind (kind 0: forward day, 1: backward day).  Enable,
 * run, then read the summed milliseconds and launch count (syncs the stream). */
gabm_status gabm_set_profiling(gabm_ctx *ctx, int enable);
gabm_status gabm_get_profile(gabm_ctx *ctx, int kind, double *total_ms, int64_t *launches);

/* Evaluate the device Philox4x32-10 (Salmon et al., SC'11) for test use:
 * ctr [count][4] uint32 and out [count][4] uint32, both device memory. */
gabm_status gabm_philox(uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t count,
                        void *cuda_stream);

/* Message for the last failing call on ctx (or for the last failing
 * gabm_create when ctx is NULL).  Valid until the next call on that ctx. */
const char *gabm_last_error(const gabm_ctx *ctx);

/* Release everything a ctx owns (waits for its stream).  NULL-safe. */
void gabm_destroy(gabm_ctx *ctx);

/* Library version string. */
const char *gabm_version(void);

/* ---------------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart: this exists for
 * callers that cannot let a library allocate device memory -- code running
 * under a fixed device-memory budget, inside another framework's memory pool,
 * or in a host that hands over only the buffers to be filled.
 *
 * gabm_seed_state_noalloc writes the day-0 state that gabm_forward starts
 * from, for num_instances instances of one n-agent population:
 * e_out [num_instances][n] (int16, device memory owned by the caller) gets
 * GABM_NEVER everywhere except, in each instance i, the n_seed[i] agents with
 * the smallest Philox key at (agent id, 0, i, 1), which get -tau_EI.
 * n_seed is host memory.  All work is enqueued on cuda_stream (a
 * cudaStream_t, NULL = legacy default stream); the call does not wait for it.
 *
 * Its scratch (selection state, digit histograms, tie lists; about 25 KB per
 * instance) is one fixed array of device memory inside the library, sized for
 * GABM_NOALLOC_MAX_INSTANCES instances, which every device that loads the
 * library keeps until the process exits.  The call performs no device
 * allocation or release.  Limits: 1 <= num_instances <=
 * GABM_NOALLOC_MAX_INSTANCES, n >= 1 and n * num_instances < 2^31; anything
 * else returns GABM_EINVAL with a message in gabm_noalloc_last_error().
 * Each call outside a stream capture looks up the array's device address on
 * the current device; a call on a capturing stream reuses the address of the
 * last uncaptured call on that device (GABM_ECUDA if there was none), so make
 * the first call on a device before any stream capture.  All calls
 * share the array: calls whose GPU work overlaps (different streams without
 * ordering) race on it and must not be issued.
 */
#define GABM_NOALLOC_MAX_INSTANCES 16

gabm_status gabm_seed_state_noalloc(uint64_t seed, int64_t n, int num_instances, const int32_t *n_seed,
                                    int tau_EI, int16_t *e_out, void *cuda_stream);

/* Message for the last failing gabm_seed_state_noalloc call of this thread. */
const char *gabm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GABM_H */
