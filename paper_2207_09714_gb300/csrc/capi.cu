// capi.cu -- the C ABI (include/gabm.h) and the host runtime behind it:
// input validation, the device memory plan of a ctx, CSR concatenation and
// transpose, the per-day launch sequences of the forward and the reverse
// sweep, and the host/device staging of arguments.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "gabm_internal.cuh"
#include "sirs.cuh"

using namespace gabm;

#ifndef GABM_DAY_WAVES
#define GABM_DAY_WAVES 1
#endif

namespace {

thread_local std::string g_create_error;

size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

}  // namespace

struct gabm_ctx {
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    int G = 0, B = 1, I = 0;
    int Bp = 1;                     // row stride of per-agent arrays: B rounded up to a power of two (1 if B == 1)
    bool batched = false;           // B > 1: the set-batched kernels over row-compressed edges
    bool kahan_b = false;           // batched sums: compensated (some row longer than kPlainSumMaxDegree)
    int spl_fwd = 2, spl_bwd = 2;   // batched schedules: sets per lane of the forward / backward day kernels
    int bwd_chunk = 1;              // batched backward: sets per launch (a power of two dividing Bp)
    bool soft = false;              // fixed-noise soft relaxation instead of hard draws
    float *s_soft = nullptr, *nh = nullptr, *x2 = nullptr;      // [n_rows], [L][n_rows], [2][n_rows]
    float *s_hist = nullptr, *y_hist = nullptr;                 // [Tcap][n_rows] soft histories
    double *P_nrm = nullptr, *newRM_real = nullptr;             // [Tcap][ntiles], [I][Tcap]
    int32_t *sig = nullptr, *emax = nullptr;   // [G][Tcap+1] reverse-sweep scale exponents per graph and day
    int tau_EI = 0, tau_IR = 0, L = 0;   // L: the table's length, the longest infectious window
    int tau_IM = 0, L_R = 0, L_M = 0;    // sampled R/M split (tau_IM > 0): exits at L_R and L_M
    bool fate = false;
    double *Pm = nullptr;                // [Tcap][ntiles] fate-draw shares of dL/dm by draw day
    DurRef dur{};                        // stochastic I-stage durations (dur.n > 0)
    bool sirs = false;                   // SIRS reinfection (tau_RS > 0)
    int tau_RS = 0, cycle = 0;           // days in RM before S again; L + tau_RS
    int sirs_H = 0;                      // history entries per row
    int16_t *sirs_hist = nullptr;        // [n_rows][sirs_H] exposure days
    uint16_t *sirs_cnt = nullptr;        // [n_rows] (H <= GABM_MAX_DAYS / 3 + 2 fits)
    uint8_t *flags = nullptr;            // [3][n_rows] rows with an infectious in-neighbour (day t mod 3)
    float *sirs_Gh = nullptr;            // [n_rows][sirs_H] G at each exposure
    float *sirs_Lh = nullptr;            // [n_rows][sirs_H] G's own-day terms at each exposure
    int grid_sirs_f = 0, grid_sirs_b = 0;
    float c[kMaxL] = {0};
    uint64_t seed = 0;
    int policy = GABM_STORE_LAMBDA;

    int64_t n_total = 0, n_rows = 0, nnz = 0, nnz_pad = 0;
    int ntiles = 0;
    std::vector<int32_t> h_row0, h_rows, h_tile0, h_ntiles;
    std::vector<double> h_Dbar;
    bool symmetric = false;

    // SELL-32 edges: in-edges, and out-edges when the weights are not symmetric
    uint32_t *slice_ptr = nullptr, *row_len = nullptr, *scol = nullptr;
    float *sw = nullptr;
    uint32_t *t_slice_ptr = nullptr, *t_row_len = nullptr, *t_scol = nullptr;
    float *t_sw = nullptr;
    int64_t sell_entries = 0;
    // row-compressed edges (batched kernels): in-edges, and out-edges when not symmetric
    uint32_t *csr_rowptr = nullptr, *csr_col = nullptr, *t_csr_rowptr = nullptr, *t_csr_col = nullptr;
    float *csr_w = nullptr, *t_csr_w = nullptr;
    uint32_t *rbits = nullptr;      // [Bp/2][2][ntiles] rows susceptible in some set of a chunk (batched backward)
    double *Pc = nullptr;           // [Tcap][G][max_chunks][9][Bp] first-level gradient sums (batched)
    int max_chunks = 0, max_graph_tiles = 0;
    uint8_t *tile_new = nullptr;    // [Tcap][ntiles][Bp] exposures per tile, set and day (batched)
    int32_t *hist0 = nullptr;       // [I][L+2] exposure-day histogram of the forward's starting state
    int32_t *newinf = nullptr;      // [I][Tcap] exposures per instance and day
    int sigma = 1024;
    uint8_t *age = nullptr;
    int32_t *d_row0 = nullptr, *d_rows = nullptr, *d_tile0 = nullptr, *d_ntiles = nullptr;
    int64_t *d_goff = nullptr;      // [G] caller offset of each graph
    uint32_t *d_orig_id = nullptr;  // [n_rows] caller id of each row (nullptr: input order)
    uint16_t *d_tile_graph = nullptr;
    float *d_inv_Dbar = nullptr;
    int16_t *e = nullptr;

    int Tcap = 0;
    float *lam = nullptr;
    int32_t *counts = nullptr, *newRM = nullptr, *newRM_b = nullptr;
    double *D = nullptr, *gD = nullptr, *y = nullptr, *P = nullptr, *Q = nullptr;
    float *R = nullptr, *m = nullptr, *S = nullptr;
    double *dR_s = nullptr, *dm_s = nullptr, *dS_s = nullptr, *loss_s = nullptr;
    double *dc_tile = nullptr;      // [ntiles][kMaxL] table-adjoint accumulators (on request)
    double *dc_s = nullptr;         // [I][L] staging of the table adjoint for host outputs
    bool want_dc = false;           // the running backward accumulates the table adjoint

    SeedState *seedst = nullptr;
    uint32_t *hist = nullptr, *ties = nullptr;
    int32_t *d_nseed = nullptr;

    float *ring = nullptr, *A = nullptr, *r = nullptr, *rows_f = nullptr, *stage_f = nullptr;
    float *lam_tmp = nullptr;       // [n_rows] recomputed lambda of one day (in- != out-edges)
    float *c_dev = nullptr;         // [kMaxL] infectiousness table
    int16_t *rows_e = nullptr;

    int t0_next = 0;
    bool resumed = false;
    bool last_from_seeding = false;  // the last forward started from seeding (not from gabm_set_state)
    bool gD_staged = false;
    std::vector<int32_t> last_seeds;  // n_seed of the last seeded forward
    int T_last = -1;
    int lam_from = -1;
    int bits_from = -1;             // first day whose infectious bitmap the last forward wrote

    int grid_fwd = 0, grid_bwd = 0, grid_bwd_dc = 0;   // grid_bwd_dc: the table-adjoint instance
    int grid_bwd_fate = 0;                              // the sampled R/M split's instance
    bool smem_bits = false;         // forward keeps the infectious bitmap in shared memory
    // agent-location graphs: the location hop (SELL-32 of locations -> members) and its values
    bool two_hop = false;
    int64_t n_loc = 0;
    int loc_ntiles = 0, grid_loc = 0;
    uint32_t *loc_slice_ptr = nullptr, *loc_row_len = nullptr, *loc_col = nullptr;
    float *loc_w = nullptr;
    float *locv = nullptr;          // [loc_ntiles * 32] location pressures (forward) or adjoints (backward)
    float *self_q = nullptr;        // [n_rows] sum over the agent's locations of w_il^2
    uint32_t *big_rowptr = nullptr, *big_col = nullptr;   // locations of more than 32 members (CSR)
    float *big_w = nullptr;
    int n_big = 0;
    int *tile_ctr = nullptr;        // batched: [1 + max chunks][Tcap] per-launch tile counters (forward, backward chunks)
    uint32_t *bits = nullptr;       // [Tcap][ntiles] per-day bitmaps of infectious rows

    size_t mem_cur = 0, mem_peak = 0;
    std::unordered_map<void *, size_t> sizes;
    long fail_alloc_after = -1, alloc_calls = 0;
    uint64_t launches = 0;

    // day loops captured as CUDA graphs (GABM_CUDA_GRAPHS=0: launched eagerly)
    struct LoopGraph {
        cudaGraphExec_t exec = nullptr;
        int t0 = -1, T = -1;
        bool dc = false;           // captured with the table adjoint
        uint64_t generation = 0;
        uint64_t kernels = 0;      // kernel launches in the graph
    };
    bool use_graphs = true;
    cudaStream_t cap_stream = nullptr;
    LoopGraph loop_graph[2];
    uint64_t buffer_generation = 0;   // bumped whenever per-day buffers are reallocated

    bool profiling = false;
    std::vector<cudaEvent_t> ev[2];
    size_t ev_used[2] = {0, 0};
    double prof_ms[2] = {0, 0};
    int64_t prof_n[2] = {0, 0};

    std::string err;
};

namespace {

gabm_status fail(gabm_ctx *c, gabm_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_create_error = buf;
    return st;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(c, GABM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define LAUNCH(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        c->launches++;                                                                        \
        if (e_ != cudaSuccess) return fail(c, GABM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define TRY(call)                        \
    do {                                 \
        gabm_status s_ = (call);         \
        if (s_ != GABM_OK) return s_;    \
    } while (0)

template <typename T>
gabm_status dalloc(gabm_ctx *c, T **p, size_t count) {
    c->alloc_calls++;
    if (c->fail_alloc_after >= 0 && c->alloc_calls > c->fail_alloc_after)
        return fail(c, GABM_ENOMEM, "device allocation %ld refused (injected allocation failure)", c->alloc_calls);
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GABM_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    c->sizes[q] = bytes;
    c->mem_cur += bytes;
    if (c->mem_cur > c->mem_peak) c->mem_peak = c->mem_cur;
    *p = (T *)q;
    return GABM_OK;
}

template <typename T>
void dfree(gabm_ctx *c, T *&p) {
    if (!p) return;
    auto it = c->sizes.find((void *)p);
    if (it != c->sizes.end()) {
        c->mem_cur -= it->second;
        c->sizes.erase(it);
        cudaFree((void *)p);
    }
    p = nullptr;
}

cudaMemcpyKind h2d_kind(int ms) { return ms == GABM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice; }
cudaMemcpyKind d2h_kind(int ms) { return ms == GABM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice; }

// ---------------------------------------------------------------------------
// Host-side validation (runs before any CUDA call for host-resident inputs)
// ---------------------------------------------------------------------------
struct HostGraph {
    int64_t n = 0, nnz = 0;
    std::vector<uint64_t> rowptr;
    std::vector<uint32_t> col;
    std::vector<float> w;
    std::vector<uint8_t> age;
};

gabm_status validate_model(const gabm_model_desc *md) {
    if (!md) return fail(nullptr, GABM_EINVAL, "model descriptor is NULL");
    if (md->tau_EI < 1 || md->tau_IR < 1) return fail(nullptr, GABM_EINVAL, "tau_EI and tau_IR must be >= 1");
    if (md->tau_IM < 0) return fail(nullptr, GABM_EINVAL, "tau_IM must be >= 0 (0: a single RM exit)");
    if (md->tau_RS < 0) return fail(nullptr, GABM_EINVAL, "tau_RS must be >= 0 (0: no return to S)");
    if (md->p_IR) {
        double sum = 0.0;
        for (int j = 0; j < md->tau_IR && j < kMaxL; ++j) {
            if (!std::isfinite(md->p_IR[j]) || md->p_IR[j] < 0.0f)
                return fail(nullptr, GABM_EINVAL, "p_IR[%d] must be finite and >= 0", j);
            sum += md->p_IR[j];
        }
        if (!(sum > 0.0)) return fail(nullptr, GABM_EINVAL, "p_IR has no mass");
    }
    const int L = md->tau_EI + std::max(md->tau_IR, md->tau_IM);
    if (L > kMaxL) return fail(nullptr, GABM_EINVAL, "tau_EI + max(tau_IR, tau_IM) = %d exceeds %d", L, kMaxL);
    if (!md->c) return fail(nullptr, GABM_EINVAL, "infectiousness table c is NULL");
    if (md->c[0] != 0.0f) return fail(nullptr, GABM_EINVAL, "c[0] must be 0 (no onward infection on the day of exposure)");
    for (int k = 0; k < L; ++k)
        if (!std::isfinite(md->c[k]) || md->c[k] < 0.0f)
            return fail(nullptr, GABM_EINVAL, "c[%d] must be finite and >= 0", k);
    if (md->relax_mode != GABM_HARD_ST && md->relax_mode != GABM_SOFT)
        return fail(nullptr, GABM_EINVAL, "unknown relax_mode %d", md->relax_mode);
    if (!(md->gumbel_tau == 1.0f)) return fail(nullptr, GABM_EUNSUPPORTED, "only gumbel_tau = 1 is implemented");
    if (md->lambda_policy != GABM_STORE_LAMBDA && md->lambda_policy != GABM_RECOMPUTE)
        return fail(nullptr, GABM_EINVAL, "unknown lambda_policy %d", md->lambda_policy);
    if (md->agent_order != GABM_ORDER_INPUT && md->agent_order != GABM_ORDER_BFS &&
        md->agent_order != GABM_ORDER_COMMUNITY)
        return fail(nullptr, GABM_EINVAL, "unknown agent_order %d", md->agent_order);
    return GABM_OK;
}

gabm_status fetch_graph(const gabm_graph_desc &d, int g, HostGraph &h) {
    if (d.n < 0 || d.nnz < 0) return fail(nullptr, GABM_EINVAL, "graph %d: negative n or nnz", g);
    if (d.n >= ((int64_t)1 << 31) - 64) return fail(nullptr, GABM_EUNSUPPORTED, "graph %d: n >= 2^31", g);
    if (d.nnz >= ((int64_t)1 << 32) - 64) return fail(nullptr, GABM_EUNSUPPORTED, "graph %d: nnz >= 2^32", g);
    if (!d.rowptr || (d.nnz > 0 && (!d.col || !d.w)) || (d.n > 0 && !d.age))
        return fail(nullptr, GABM_EINVAL, "graph %d: NULL array", g);
    if (d.mem_space != GABM_HOST && d.mem_space != GABM_DEVICE)
        return fail(nullptr, GABM_EINVAL, "graph %d: bad mem_space", g);
    h.n = d.n;
    h.nnz = d.nnz;
    h.rowptr.resize((size_t)d.n + 1);
    h.col.resize((size_t)d.nnz);
    h.w.resize((size_t)d.nnz);
    h.age.resize((size_t)d.n);
    if (d.mem_space == GABM_HOST) {
        memcpy(h.rowptr.data(), d.rowptr, sizeof(uint64_t) * h.rowptr.size());
        if (d.nnz) memcpy(h.col.data(), d.col, sizeof(uint32_t) * h.col.size());
        if (d.nnz) memcpy(h.w.data(), d.w, sizeof(float) * h.w.size());
        if (d.n) memcpy(h.age.data(), d.age, h.age.size());
    } else {
        cudaError_t e = cudaMemcpy(h.rowptr.data(), d.rowptr, sizeof(uint64_t) * h.rowptr.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && d.nnz) e = cudaMemcpy(h.col.data(), d.col, sizeof(uint32_t) * h.col.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && d.nnz) e = cudaMemcpy(h.w.data(), d.w, sizeof(float) * h.w.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && d.n) e = cudaMemcpy(h.age.data(), d.age, h.age.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(nullptr, GABM_ECUDA, "graph %d: copy to host: %s", g, cudaGetErrorString(e));
    }
    if (h.rowptr[0] != 0) return fail(nullptr, GABM_EINVAL, "graph %d: rowptr[0] != 0", g);
    for (int64_t i = 0; i < h.n; ++i)
        if (h.rowptr[i + 1] < h.rowptr[i]) return fail(nullptr, GABM_EINVAL, "graph %d: rowptr decreases at row %lld", g, (long long)i);
    if ((int64_t)h.rowptr[h.n] != h.nnz) return fail(nullptr, GABM_EINVAL, "graph %d: rowptr[n] != nnz", g);
    for (int64_t p = 0; p < h.nnz; ++p) {
        if ((int64_t)h.col[p] >= h.n) return fail(nullptr, GABM_EINVAL, "graph %d: col[%lld] = %u out of range", g, (long long)p, h.col[p]);
        if (!std::isfinite(h.w[p]) || h.w[p] < 0.0f) return fail(nullptr, GABM_EINVAL, "graph %d: w[%lld] not finite and >= 0", g, (long long)p);
    }
    for (int64_t i = 0; i < h.n; ++i)
        if (h.age[i] >= kAges) return fail(nullptr, GABM_EINVAL, "graph %d: age[%lld] = %u > 8", g, (long long)i, h.age[i]);
    return GABM_OK;
}

// Source-sorted CSR of one graph (rows of the transpose in ascending source order).
void transpose_graph(const HostGraph &h, std::vector<uint64_t> &trp, std::vector<uint32_t> &tcol,
                     std::vector<float> &tw) {
    trp.assign((size_t)h.n + 1, 0);
    tcol.resize((size_t)h.nnz);
    tw.resize((size_t)h.nnz);
    for (int64_t p = 0; p < h.nnz; ++p) trp[(size_t)h.col[p] + 1]++;
    for (int64_t i = 0; i < h.n; ++i) trp[i + 1] += trp[i];
    std::vector<uint64_t> pos(trp.begin(), trp.end() - 1);
    for (int64_t i = 0; i < h.n; ++i)
        for (uint64_t p = h.rowptr[i]; p < h.rowptr[i + 1]; ++p) {
            const uint64_t q = pos[h.col[p]]++;
            tcol[q] = (uint32_t)i;
            tw[q] = h.w[p];
        }
}

// Breadth-first order over the in-edges: every dequeued agent appends its
// not-yet-seen neighbours, so groups of mutual contacts (households, schools,
// workplaces) become adjacent rows and one warp's gathers share cache lines.
std::vector<uint32_t> bfs_order(const HostGraph &h) {
    std::vector<uint32_t> order;
    order.reserve((size_t)h.n);
    std::vector<uint8_t> seen((size_t)h.n, 0);
    for (int64_t s = 0; s < h.n; ++s) {
        if (seen[s]) continue;
        seen[s] = 1;
        size_t head = order.size();
        order.push_back((uint32_t)s);
        while (head < order.size()) {
            const uint32_t v = order[head++];
            for (uint64_t p = h.rowptr[v]; p < h.rowptr[v + 1]; ++p) {
                const uint32_t u = h.col[p];
                if (!seen[u]) {
                    seen[u] = 1;
                    order.push_back(u);
                }
            }
        }
    }
    return order;
}

// Community order: agents of one densely connected group (a school, a workplace) become
// consecutive rows, which breadth-first order does not give on a small-world contact
// graph (a group's members are reached over many paths, long before the first of them is
// expanded).  A few sweeps of label propagation find the groups: every agent, visited in
// breadth-first order, takes the label most frequent among its in-neighbours (ties broken
// by a seeded reservoir draw), labels updated in place.  Groups are then laid out at the
// breadth-first position of their first member, and members in breadth-first order.
std::vector<uint32_t> community_order(const HostGraph &h, int sweeps) {
    const int64_t n = h.n;
    std::vector<uint32_t> bfs = bfs_order(h);
    std::vector<uint32_t> lab((size_t)n);
    for (int64_t i = 0; i < n; ++i) lab[i] = (uint32_t)i;
    std::vector<uint32_t> nl;
    uint64_t rng = 0x243F6A8885A308D3ull;   // fixed: the layout is a function of the graph
    for (int sw = 0; sw < sweeps; ++sw) {
        for (int64_t q = 0; q < n; ++q) {
            const uint32_t v = bfs[q];
            const uint64_t p0 = h.rowptr[v], p1 = h.rowptr[v + 1];
            if (p0 == p1) continue;
            nl.resize(p1 - p0);
            for (uint64_t p = p0; p < p1; ++p) nl[p - p0] = lab[h.col[p]];
            std::sort(nl.begin(), nl.end());
            uint32_t best = lab[v];
            size_t best_c = 0, ties = 0;
            for (size_t i = 0; i < nl.size();) {
                size_t j = i;
                while (j < nl.size() && nl[j] == nl[i]) ++j;
                const size_t c = j - i;
                if (c > best_c) {
                    best_c = c;
                    best = nl[i];
                    ties = 1;
                } else if (c == best_c) {   // keep each tied label with probability 1 / ties
                    ++ties;
                    rng = rng * 6364136223846793005ull + 1442695040888963407ull;
                    if ((rng >> 33) % ties == 0) best = nl[i];
                }
                i = j;
            }
            lab[v] = best;
        }
    }
    std::vector<uint64_t> bpos((size_t)n), first((size_t)n, (uint64_t)n);
    for (int64_t q = 0; q < n; ++q) bpos[bfs[q]] = (uint64_t)q;
    for (int64_t v = 0; v < n; ++v) first[lab[v]] = std::min(first[lab[v]], bpos[v]);
    std::vector<uint64_t> key((size_t)n);
    for (int64_t v = 0; v < n; ++v) key[v] = first[lab[v]] * (uint64_t)n + bpos[v];   // unique: bpos is
    std::vector<uint32_t> order((size_t)n);
    for (int64_t i = 0; i < n; ++i) order[i] = (uint32_t)i;
    std::sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return key[a] < key[b]; });
    return order;
}

// Within consecutive windows of `sigma` positions of an order, sort the agents by
// decreasing degree (stable), so that each 32-row slice holds rows of similar
// length: little padding in the SELL-32 layout, while agents stay near their
// breadth-first neighbourhood.
void sort_windows_by_degree(const HostGraph &h, std::vector<uint32_t> &order, int sigma) {
    if (sigma <= 1) return;
    for (size_t w0 = 0; w0 < order.size(); w0 += (size_t)sigma) {
        const size_t w1 = std::min(order.size(), w0 + (size_t)sigma);
        std::stable_sort(order.begin() + w0, order.begin() + w1, [&](uint32_t a, uint32_t b) {
            return (h.rowptr[a + 1] - h.rowptr[a]) > (h.rowptr[b + 1] - h.rowptr[b]);
        });
    }
}

// Rows much longer than the rest (hubs of a power-law contact graph) cost a SELL tile
// its longest row in every lane's loop.  Rows of more than kLongRow entries therefore
// leave their degree window: they are sorted by length and put, 32 to a tile, at evenly
// spaced window boundaries of the order, so that each such tile holds rows of similar
// length and the heavy tiles spread over the launch's tile ranges.
constexpr uint64_t kLongRow = 128;

void group_long_rows(const HostGraph &h, std::vector<uint32_t> &order, int sigma) {
    auto len = [&](uint32_t a) { return h.rowptr[a + 1] - h.rowptr[a]; };
    std::vector<uint32_t> rest, lng;
    rest.reserve(order.size());
    for (uint32_t a : order) (len(a) > kLongRow ? lng : rest).push_back(a);
    if (lng.empty()) return;
    std::stable_sort(lng.begin(), lng.end(), [&](uint32_t a, uint32_t b) { return len(a) > len(b); });
    const size_t groups = (lng.size() + kTile - 1) / kTile;
    const size_t win = (size_t)std::max(sigma, kTile);
    const size_t nwin = rest.size() / win;   // whole windows of the other rows
    order.clear();
    size_t r = 0, gi = 0;
    for (size_t wi = 0; wi <= nwin; ++wi) {
        // group gi goes after window floor((gi + 1) * nwin / (groups + 1))
        while (gi < groups && (wi == nwin || (gi + 1) * nwin / (groups + 1) <= wi)) {
            const size_t b = gi * kTile, e = std::min(lng.size(), b + kTile);
            order.insert(order.end(), lng.begin() + (long)b, lng.begin() + (long)e);
            ++gi;
            if (e - b < (size_t)kTile) break;   // a partial group only at the very end
        }
        const size_t r1 = (wi == nwin) ? rest.size() : std::min(rest.size(), r + win);
        order.insert(order.end(), rest.begin() + (long)r, rest.begin() + (long)r1);
        r = r1;
    }
    while (gi < groups) {   // a partial last group (it completes no window)
        const size_t b = gi * kTile, e = std::min(lng.size(), b + kTile);
        order.insert(order.end(), lng.begin() + (long)b, lng.begin() + (long)e);
        ++gi;
    }
}

// SELL-32 of a device-order CSR: slice s = rows [32 s, 32 s + 32), max_len(s) x 32
// entries, entry k of the row in lane l at slice_ptr[s] + 32 k + l; padding has
// column 0 and weight 0 and is never read.
struct HostSell {
    std::vector<uint32_t> slice_ptr, row_len, col;
    std::vector<float> w;
};

bool build_sell(const std::vector<uint32_t> &rowptr, const std::vector<uint32_t> &col, const std::vector<float> &w,
                int64_t n_rows, HostSell &hs) {
    const int64_t ns = n_rows / kTile;
    hs.slice_ptr.assign((size_t)ns + 1, 0u);
    hs.row_len.assign((size_t)n_rows, 0u);
    uint64_t total = 0;
    for (int64_t sl = 0; sl < ns; ++sl) {
        uint32_t mx = 0;
        for (int l = 0; l < kTile; ++l) {
            const int64_t r = sl * kTile + l;
            const uint32_t len = rowptr[r + 1] - rowptr[r];
            hs.row_len[r] = len;
            mx = std::max(mx, len);
        }
        hs.slice_ptr[sl] = (uint32_t)total;
        total += (uint64_t)mx * kTile;
        if (total >= ((uint64_t)1 << 32) - 64) return false;
    }
    hs.slice_ptr[ns] = (uint32_t)total;
    hs.col.assign((size_t)std::max<uint64_t>(total, 32), 0u);
    hs.w.assign((size_t)std::max<uint64_t>(total, 32), 0.f);
    for (int64_t r = 0; r < n_rows; ++r) {
        const uint32_t base = hs.slice_ptr[r / kTile] + (uint32_t)(r % kTile);
        for (uint32_t k = 0; k < hs.row_len[r]; ++k) {
            hs.col[base + (size_t)k * kTile] = col[rowptr[r] + k];
            hs.w[base + (size_t)k * kTile] = w[rowptr[r] + k];
        }
    }
    return true;
}

// Relabel a graph: new row k is old agent order[k]; each row's entries sorted by new column.
// The device order of one graph's agents (order[r] = the caller's id of row r): the agent
// order, then degree windows of sigma rows (GABM_SELL_SIGMA, default 1024), then, with one
// set per graph, the long rows grouped.
int sell_sigma() {
    int sigma = 1024;
    if (const char *f = getenv("GABM_SELL_SIGMA")) sigma = std::max(1, atoi(f));
    return sigma;
}

std::vector<uint32_t> layout_order(const HostGraph &h, int agent_order, int sets_per_graph) {
    const int sigma = sell_sigma();
    std::vector<uint32_t> order;
    if (agent_order == GABM_ORDER_BFS) {
        order = bfs_order(h);
    } else if (agent_order == GABM_ORDER_COMMUNITY) {
        order = community_order(h, 3);
    } else {
        order.resize((size_t)h.n);
        for (int64_t i = 0; i < h.n; ++i) order[i] = (uint32_t)i;
    }
    sort_windows_by_degree(h, order, sigma);
    if (sets_per_graph == 1) group_long_rows(h, order, sigma);
    return order;
}

HostGraph permute_graph(const HostGraph &h, const std::vector<uint32_t> &order) {
    HostGraph o;
    o.n = h.n;
    o.nnz = h.nnz;
    std::vector<uint32_t> inv((size_t)h.n);
    for (int64_t k = 0; k < h.n; ++k) inv[order[k]] = (uint32_t)k;
    o.rowptr.assign((size_t)h.n + 1, 0);
    o.col.resize((size_t)h.nnz);
    o.w.resize((size_t)h.nnz);
    o.age.resize((size_t)h.n);
    for (int64_t k = 0; k < h.n; ++k) {
        const uint32_t v = order[k];
        o.rowptr[k + 1] = o.rowptr[k] + (h.rowptr[v + 1] - h.rowptr[v]);
        o.age[k] = h.age[v];
    }
    std::vector<std::pair<uint32_t, float>> tmp;
    for (int64_t k = 0; k < h.n; ++k) {
        const uint32_t v = order[k];
        tmp.clear();
        for (uint64_t p = h.rowptr[v]; p < h.rowptr[v + 1]; ++p) tmp.emplace_back(inv[h.col[p]], h.w[p]);
        std::sort(tmp.begin(), tmp.end(),
                  [](const std::pair<uint32_t, float> &a, const std::pair<uint32_t, float> &b) { return a.first < b.first; });
        uint64_t q = o.rowptr[k];
        for (const auto &e : tmp) {
            o.col[q] = e.first;
            o.w[q] = e.second;
            ++q;
        }
    }
    return o;
}

// Launches per backward day at most (the batched backward may split a row's sets).
int max_bwd_chunks(const gabm_ctx *c) { return c->batched ? std::max(1, c->Bp / 2) : 1; }

gabm_status ensure_days(gabm_ctx *c, int T) {
    if (T <= c->Tcap) return GABM_OK;
    int cap = c->Tcap > 0 ? c->Tcap : 8;
    while (cap < T) cap *= 2;
    if (cap > GABM_MAX_DAYS) cap = GABM_MAX_DAYS;
    CK(cudaStreamSynchronize(c->stream));
    dfree(c, c->lam); dfree(c, c->counts); dfree(c, c->newRM); dfree(c, c->newRM_b);
    dfree(c, c->D); dfree(c, c->gD); dfree(c, c->y); dfree(c, c->P); dfree(c, c->Q);
    dfree(c, c->R); dfree(c, c->m);
    dfree(c, c->dR_s); dfree(c, c->dm_s); dfree(c, c->tile_ctr); dfree(c, c->bits); dfree(c, c->Pc);
    dfree(c, c->tile_new); dfree(c, c->newinf);
    dfree(c, c->s_hist); dfree(c, c->y_hist); dfree(c, c->P_nrm); dfree(c, c->newRM_real);
    dfree(c, c->sig); dfree(c, c->emax); dfree(c, c->Pm);
    c->Tcap = 0;
    const size_t IT = (size_t)c->I * cap;
    if (c->policy == GABM_STORE_LAMBDA) TRY(dalloc(c, &c->lam, (size_t)cap * c->n_rows * c->Bp));
    TRY(dalloc(c, &c->counts, IT * 4));
    TRY(dalloc(c, &c->newRM, IT));
    TRY(dalloc(c, &c->newRM_b, IT));
    TRY(dalloc(c, &c->D, IT));
    TRY(dalloc(c, &c->gD, IT));
    TRY(dalloc(c, &c->y, IT));
    TRY(dalloc(c, &c->P, (size_t)cap * c->ntiles * kAges * c->Bp));
    if (c->fate) TRY(dalloc(c, &c->Pm, (size_t)cap * c->ntiles));
    if (c->soft) {
        TRY(dalloc(c, &c->s_hist, (size_t)cap * c->n_rows));
        TRY(dalloc(c, &c->y_hist, (size_t)cap * c->n_rows));
        TRY(dalloc(c, &c->P_nrm, (size_t)cap * c->ntiles));
        TRY(dalloc(c, &c->newRM_real, IT));
    }
    if (c->batched) {
        TRY(dalloc(c, &c->Pc, (size_t)cap * c->G * c->max_chunks * kAges * c->Bp));
        TRY(dalloc(c, &c->tile_new, (size_t)cap * c->ntiles * c->Bp));
        TRY(dalloc(c, &c->newinf, IT));
    }
    TRY(dalloc(c, &c->Q, IT * kAges));
    TRY(dalloc(c, &c->R, IT));
    TRY(dalloc(c, &c->m, IT));
    TRY(dalloc(c, &c->dR_s, IT));
    TRY(dalloc(c, &c->dm_s, IT));
    if (c->batched) TRY(dalloc(c, &c->tile_ctr, (size_t)(1 + max_bwd_chunks(c)) * cap));
    TRY(dalloc(c, &c->bits, (size_t)(cap + 1) * c->ntiles));
    TRY(dalloc(c, &c->sig, (size_t)c->G * (cap + 1)));
    TRY(dalloc(c, &c->emax, (size_t)c->G * (cap + 1)));
    CK(cudaMemsetAsync(c->D, 0, IT * sizeof(double), c->stream));
    c->Tcap = cap;
    c->T_last = -1;
    c->lam_from = -1;
    c->buffer_generation++;
    return GABM_OK;
}

void prof_begin(gabm_ctx *c, int kind) {
    if (!c->profiling) return;
    auto &v = c->ev[kind];
    if (c->ev_used[kind] + 2 > v.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        v.push_back(a);
        v.push_back(b);
    }
    cudaEventRecord(v[c->ev_used[kind]], c->stream);
}

void prof_end(gabm_ctx *c, int kind) {
    if (!c->profiling) return;
    cudaEventRecord(c->ev[kind][c->ev_used[kind] + 1], c->stream);
    c->ev_used[kind] += 2;
}

gabm_status prof_collect(gabm_ctx *c) {
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 2; ++k) {
        for (size_t i = 0; i + 1 < c->ev_used[k]; i += 2) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->ev[k][i], c->ev[k][i + 1]));
            c->prof_ms[k] += ms;
            c->prof_n[k] += 1;
        }
        c->ev_used[k] = 0;
    }
    return GABM_OK;
}

Sell sell_view(const gabm_ctx *c, bool out_edges) {
    Sell m;
    m.slice_ptr = out_edges ? c->t_slice_ptr : c->slice_ptr;
    m.row_len = out_edges ? c->t_row_len : c->row_len;
    m.col = out_edges ? c->t_scol : c->scol;
    m.w = out_edges ? c->t_sw : c->sw;
    return m;
}

Sell loc_sell_view(const gabm_ctx *c) {
    Sell m;
    m.slice_ptr = c->loc_slice_ptr;
    m.row_len = c->loc_row_len;
    m.col = c->loc_col;
    m.w = c->loc_w;
    return m;
}

LocCsr loc_big_view(const gabm_ctx *c) {
    LocCsr b;
    b.rowptr = c->big_rowptr;
    b.col = c->big_col;
    b.w = c->big_w;
    b.n = c->n_big;
    b.base = c->loc_ntiles * kTile;
    return b;
}

GraphRef graph_ref(const gabm_ctx *c) {
    GraphRef gr;
    gr.row0 = c->d_row0;
    gr.tile_graph = c->G > 1 ? c->d_tile_graph : nullptr;
    gr.inv_Dbar = c->d_inv_Dbar;
    gr.orig_id = c->d_orig_id;
    return gr;
}

// The sampled R/M split's constants and the staged mortality (L_M = 0: the single RM exit).
FateRef fate_ref(const gabm_ctx *c) {
    FateRef f;
    f.mort = c->m;
    f.ldP = c->Tcap;
    f.tau_EI = c->tau_EI;
    f.L_R = c->fate ? c->L_R : 0;
    f.L_M = c->fate ? c->L_M : 0;
    f.seed = c->seed;
    return f;
}

gabm_status check_ms(gabm_ctx *c, int ms) {
    if (ms != GABM_HOST && ms != GABM_DEVICE) return fail(c, GABM_EINVAL, "mem_space must be GABM_DEVICE or GABM_HOST");
    return GABM_OK;
}

SetLayout set_layout(const gabm_ctx *c) {
    SetLayout sl;
    sl.B = c->B;
    sl.Bp = c->Bp;
    sl.n_total = c->n_total;
    return sl;
}

Csr csr_view(const gabm_ctx *c, bool out_edges) {
    Csr m;
    m.rowptr = out_edges ? c->t_csr_rowptr : c->csr_rowptr;
    m.col = out_edges ? c->t_csr_col : c->csr_col;
    m.w = out_edges ? c->t_csr_w : c->csr_w;
    return m;
}

// Day loop of the forward for B > 1 sets per graph (parameters already staged).
gabm_status forward_days_batched(gabm_ctx *c, int t0, int T, cudaStream_t s) {
    const size_t nb = (size_t)c->n_rows * c->Bp;
    FwdBatchArgs a;
    a.m = csr_view(c, false);
    a.age = c->age;
    a.gr = graph_ref(c);
    a.e = c->e;
    a.R = c->R;
    a.S = c->S;
    a.ldP = c->Tcap;
    a.ntiles = c->ntiles;
    a.tau_EI = c->tau_EI;
    a.L = c->L;
    a.B = c->B;
    CK(cudaMemsetAsync(c->hist0, 0, sizeof(int32_t) * (size_t)c->I * (c->L + 2), s));
    CK(cudaMemsetAsync(c->newinf, 0, sizeof(int32_t) * (size_t)c->I * c->Tcap, s));
    LAUNCH(launch_exposure_hist_b(c->e, graph_ref(c), c->n_rows, c->B, c->Bp, t0, c->L, c->hist0, s));
    a.seed = c->seed;
    for (int k = 0; k < kMaxL; ++k) a.c[k] = k < c->L ? c->c[k] : 0.f;
    if (t0 < T)
        LAUNCH(launch_infectious_bits_b(c->e, c->Bp, t0, c->L, c->ntiles, c->bits + (size_t)t0 * c->ntiles, s));
    for (int t = t0; t < T; ++t) {
        a.t = t;
        a.lam_out = c->policy == GABM_STORE_LAMBDA ? c->lam + (size_t)t * nb : nullptr;
        a.tile_ctr = c->tile_ctr + t;
        a.bits_cur = c->bits + (size_t)t * c->ntiles;
        a.bits_next = c->bits + (size_t)(t + 1) * c->ntiles;
        a.tile_new = c->tile_new + (size_t)t * c->ntiles * c->Bp;
        prof_begin(c, 0);
        LAUNCH(launch_fwd_day_b(a, c->Bp, c->spl_fwd, c->kahan_b, c->grid_fwd, s));
        prof_end(c, 0);
    }
    LAUNCH(launch_counts_b(c->tile_new, c->ntiles, c->d_tile0, c->d_ntiles, c->d_rows, c->G, c->B, c->Bp,
                           c->max_graph_tiles, t0, T, c->Tcap, c->tau_EI, c->L, c->hist0, c->newinf, c->counts,
                           c->newRM, s));
    return GABM_OK;
}

// Reverse sweep for B > 1 sets per graph (gD already staged; r and counters cleared).
gabm_status backward_days_batched(gabm_ctx *c, int T, cudaStream_t s) {
    const int ld = c->Tcap;
    const size_t nb = (size_t)c->n_rows * c->Bp;
    const int nch = c->Bp / c->bwd_chunk;
    CK(cudaMemsetAsync(c->rbits, 0, sizeof(uint32_t) * 2 * (size_t)c->ntiles * nch, s));
    BwdBatchArgs a;
    a.m = csr_view(c, true);
    a.age = c->age;
    a.gr = graph_ref(c);
    a.E = c->e;
    a.ring = c->ring;
    a.ring_stride = nb;
    a.A = c->A;
    a.R = c->R;
    a.m_t = c->m;
    a.S = c->S;
    a.gD = c->gD;
    a.ldP = ld;
    a.ntiles = c->ntiles;
    a.T = T;
    a.tau_EI = c->tau_EI;
    a.L = c->L;
    a.B = c->B;
    a.seed = c->seed;
    for (int k = 0; k < kMaxL; ++k) a.c[k] = k < c->L ? c->c[k] : 0.f;
    a.sig = c->sig;
    a.emax = c->emax;
    a.ld_sig = ld + 1;
    a.Bw = c->Bp;
    a.dc_tile = c->want_dc ? c->dc_tile : nullptr;
    const bool rec = c->policy != GABM_STORE_LAMBDA;   // the last forward wrote every day's bitmap
    const int Lm1 = c->L - 1;
    for (int t = T - 1; t >= 0; --t) {
        a.t = t;
        a.lam_t = rec ? nullptr : c->lam + (size_t)t * nb;
        a.bits_t = c->bits + (size_t)t * c->ntiles;
        a.r_next = c->r + (size_t)((t + 1) & 1) * nb;
        a.r_cur = c->r + (size_t)(t & 1) * nb;

        a.P_t = c->P + (size_t)t * c->ntiles * kAges * c->Bp;
        for (int k = 0; k < kMaxL; ++k) a.ring_slot[k] = (k >= 1 && k < c->L) ? (t + k) % Lm1 : 0;
        prof_begin(c, 1);
        for (int ch = 0; ch < nch; ++ch) {   // the row's sets in launches of bwd_chunk sets
            a.s0 = ch * c->bwd_chunk;
            uint32_t *rb = c->rbits + (size_t)ch * 2 * c->ntiles;
            a.rbits_next = rb + (size_t)((t + 1) & 1) * c->ntiles;
            a.rbits_cur = rb + (size_t)(t & 1) * c->ntiles;
            a.tile_ctr = c->tile_ctr + (size_t)(1 + ch) * ld + t;
            LAUNCH(launch_bwd_day_b(a, c->bwd_chunk, c->spl_bwd, c->kahan_b, c->grid_bwd, s));
        }
        prof_end(c, 1);
    }
    if (a.dc_tile)   // the seeds' share through day 0 (r of day 0 is in slot 0)
        LAUNCH(launch_dc_seeds_b(csr_view(c, true), c->e, c->r, graph_ref(c), c->sig, ld + 1, c->ntiles, c->L, c->B,
                                 c->Bp, c->dc_tile, s));
    LAUNCH(launch_bwd_reduce_b(c->P, c->ntiles, c->d_tile0, c->d_ntiles, c->G, c->B, c->Bp, T, c->Pc, c->max_chunks,
                               c->sig, ld + 1, c->Q, s));
    return GABM_OK;
}

// SIRS reinfection: the forward from the seeded state, recording every exposure.
gabm_status forward_days_sirs(gabm_ctx *c, int t0, int T, cudaStream_t s) {
    if (t0 != 0) return fail(c, GABM_EUNSUPPORTED, "SIRS reinfection runs from the seeded state (day 0)");
    LAUNCH(launch_sirs_hist_init(c->e, c->n_rows, c->sirs_H, c->sirs_hist, c->sirs_cnt, s));
    if (T > 0) LAUNCH(launch_infectious_bits(c->e, 0, 1, c->L, c->ntiles, c->bits, (size_t)c->ntiles, s));
    SirsFwdArgs a;
    a.m = sell_view(c, false);
    a.age = c->age;
    a.gr = graph_ref(c);
    a.e = c->e;
    a.hist = c->sirs_hist;
    a.cnt = c->sirs_cnt;
    a.H = c->sirs_H;
    a.R = c->R;
    a.S = c->S;
    a.ldP = c->Tcap;
    a.counts = c->counts;
    a.newRM = c->newRM;
    a.ntiles = c->ntiles;
    a.tau_EI = c->tau_EI;
    a.L = c->L;
    a.cycle = c->cycle;
    a.seed = c->seed;
    for (int k = 0; k < kMaxL; ++k) a.c[k] = k < c->L ? c->c[k] : 0.f;
    // rows with an infectious in-neighbour, in three rotating buffers (as forward_days_plain)
    a.m_out = sell_view(c, true);
    auto fbuf = [&](int d) { return c->flags + (size_t)(d % 3) * c->n_rows; };
    if (c->flags && T > 0) {
        CK(cudaMemsetAsync(fbuf(0), 0, (size_t)c->n_rows, s));
        CK(cudaMemsetAsync(fbuf(1), 0, (size_t)c->n_rows, s));
        LAUNCH(launch_flags_from_bits(c->bits, a.m_out, c->ntiles, fbuf(0), s));
    }
    for (int t = 0; t < T; ++t) {
        a.t = t;
        a.lam_out = c->lam + (size_t)t * c->n_rows;
        a.bits_cur = c->bits + (size_t)t * c->ntiles;
        a.bits_next = c->bits + (size_t)(t + 1) * c->ntiles;
        a.flag_cur = c->flags ? fbuf(t) : nullptr;
        a.flag_next = c->flags ? fbuf(t + 1) : nullptr;
        a.flag_clear = c->flags ? fbuf(t + 2) : nullptr;
        prof_begin(c, 0);
        LAUNCH(launch_fwd_day_sirs(a, c->grid_sirs_f, s));
        prof_end(c, 0);
    }
    return GABM_OK;
}

// SIRS reinfection: the reverse sweep over the recorded exposure histories.
gabm_status backward_days_sirs(gabm_ctx *c, int T, cudaStream_t s) {
    const int ld = c->Tcap;
    SirsBwdArgs a;
    a.m = sell_view(c, true);
    a.age = c->age;
    a.gr = graph_ref(c);
    a.E = c->e;
    a.hist = c->sirs_hist;
    a.cnt = c->sirs_cnt;
    a.H = c->sirs_H;
    a.Gh = c->sirs_Gh;
    a.Lh = c->sirs_Lh;
    a.ring = c->ring;
    a.ring_stride = (size_t)c->n_rows;
    a.R = c->R;
    a.m_t = c->m;
    a.S = c->S;
    a.gD = c->gD;
    a.ldP = ld;
    a.newRM = c->newRM_b;
    a.sig = c->sig;
    a.emax = c->emax;
    a.ld_sig = ld + 1;
    a.ntiles = c->ntiles;
    a.T = T;
    a.tau_EI = c->tau_EI;
    a.L = c->L;
    a.cycle = c->cycle;
    a.seed = c->seed;
    for (int k = 0; k < kMaxL; ++k) a.c[k] = k < c->L ? c->c[k] : 0.f;
    const int Lm1 = c->L - 1;
    for (int t = T - 1; t >= 0; --t) {
        a.t = t;
        a.lam_t = c->lam + (size_t)t * c->n_rows;
        a.r_next = c->r + (size_t)((t + 1) & 1) * c->n_rows;
        a.r_cur = c->r + (size_t)(t & 1) * c->n_rows;
        a.P_t = c->P + (size_t)t * c->ntiles * kAges;
        for (int k = 0; k < kMaxL; ++k) a.ring_slot[k] = (k >= 1 && k < c->L) ? (t + k) % Lm1 : 0;
        prof_begin(c, 1);
        LAUNCH(launch_bwd_day_sirs(a, c->grid_sirs_b, s));
        prof_end(c, 1);
    }
    LAUNCH(launch_bwd_reduce(c->P, c->ntiles, ld, c->d_tile0, c->d_ntiles, T, c->I, c->sig, ld + 1, c->Q, s));
    return GABM_OK;
}

// History capacity of SIRS reinfection for a horizon of T days: a seed's exposure plus
// exposures at least `cycle` days apart.
gabm_status ensure_sirs(gabm_ctx *c, int T) {
    const int H = (T + c->tau_EI) / c->cycle + 2;
    if (H <= c->sirs_H) return GABM_OK;
    CK(cudaStreamSynchronize(c->stream));
    dfree(c, c->sirs_hist); dfree(c, c->sirs_cnt); dfree(c, c->sirs_Gh); dfree(c, c->sirs_Lh);
    c->sirs_H = 0;
    TRY(dalloc(c, &c->sirs_hist, (size_t)c->n_rows * H));
    TRY(dalloc(c, &c->sirs_cnt, (size_t)c->n_rows));
    TRY(dalloc(c, &c->sirs_Gh, (size_t)c->n_rows * H));
    TRY(dalloc(c, &c->sirs_Lh, (size_t)c->n_rows * H));
    c->sirs_H = H;
    c->T_last = -1;
    c->buffer_generation++;
    return GABM_OK;
}

// Day loop of the forward, one set per graph (parameters staged, seeding done).
gabm_status forward_days_plain(gabm_ctx *c, int t0, int T, cudaStream_t s) {
    if (c->sirs) return forward_days_sirs(c, t0, T, s);
    const int ld = c->Tcap;
    FwdDayArgs a;
    a.m = sell_view(c, false);
    a.age = c->age;
    a.gr = graph_ref(c);
    a.e = c->e;
    a.R = c->R;
    a.S = c->S;
    a.ldP = ld;
    a.counts = c->counts;
    a.newRM = c->newRM;
    a.ntiles = c->ntiles;
    a.tau_EI = c->tau_EI;
    a.L = c->L;
    a.seed = c->seed;
    a.fate = fate_ref(c);
    a.dur = c->dur;
    for (int k = 0; k < kMaxL; ++k) a.c[k] = k < c->L ? c->c[k] : 0.f;
    if (t0 < T && c->dur.n > 0)
        LAUNCH(launch_infectious_bits_dur(c->e, graph_ref(c), c->dur, t0, c->ntiles, c->bits + (size_t)t0 * c->ntiles, s));
    else if (t0 < T && c->fate)
        LAUNCH(launch_infectious_bits_fate(c->e, graph_ref(c), a.fate, t0, c->ntiles, c->bits + (size_t)t0 * c->ntiles, s));
    else if (t0 < T)
        LAUNCH(launch_infectious_bits(c->e, t0, 1, c->L, c->ntiles, c->bits + (size_t)t0 * c->ntiles,
                                      (size_t)c->ntiles, s));
    // Rows with an infectious in-neighbour, per day, in three rotating buffers: day t
    // reads buffer t mod 3, fills t + 1 mod 3 and clears t + 2 mod 3.
    const bool flagged = c->flags && !c->two_hop;
    a.m_out = sell_view(c, true);
    a.t_first = t0;
    auto fbuf = [&](int d) { return c->flags + (size_t)(d % 3) * c->n_rows; };
    if (flagged && t0 < T) {
        CK(cudaMemsetAsync(fbuf(t0), 0, (size_t)c->n_rows, s));
        CK(cudaMemsetAsync(fbuf(t0 + 1), 0, (size_t)c->n_rows, s));
        LAUNCH(launch_flags_from_bits(c->bits + (size_t)t0 * c->ntiles, a.m_out, c->ntiles, fbuf(t0), s));
    }
    for (int t = t0; t < T; ++t) {
        a.t = t;
        a.lam_out = c->policy == GABM_STORE_LAMBDA ? c->lam + (size_t)t * c->n_rows : nullptr;
        a.bits_cur = c->bits + (size_t)t * c->ntiles;
        a.bits_next = c->bits + (size_t)(t + 1) * c->ntiles;
        a.flag_cur = flagged ? fbuf(t) : nullptr;
        a.flag_next = flagged ? fbuf(t + 1) : nullptr;
        a.flag_clear = flagged ? fbuf(t + 2) : nullptr;
        a.pull = nullptr;
        prof_begin(c, 0);
        if (c->two_hop) {   // location pressures of day t, then the agents' pull over their locations
            LAUNCH(launch_loc_pressure(loc_sell_view(c), c->loc_ntiles, loc_big_view(c), c->e, a.bits_cur, t, c->L, c->c_dev, c->locv,
                                       c->grid_loc, s));
            a.pull = c->locv;
        }
        LAUNCH(launch_fwd_day(a, c->grid_fwd, c->smem_bits, s));
        prof_end(c, 0);
    }
    return GABM_OK;
}

// Reverse sweep, one set per graph (gD staged; r and counters cleared).
gabm_status backward_days_plain(gabm_ctx *c, int T, cudaStream_t s) {
    if (c->sirs) return backward_days_sirs(c, T, s);
    const int ld = c->Tcap;
    BwdDayArgs a;
    const int mode = c->soft ? kBwdSoft
                             : (c->policy == GABM_STORE_LAMBDA ? kBwdStore : (c->symmetric ? kBwdFused : kBwdSplit));
    a.mode = mode == kBwdSplit ? kBwdStore : mode;
    a.m = sell_view(c, true);
    a.age = c->age;
    a.gr = graph_ref(c);
    a.E = c->e;
    a.ring = c->ring;
    a.ring_stride = (size_t)c->n_rows;
    a.A = c->A;
    a.R = c->R;
    a.m_t = c->m;
    a.S = c->S;
    a.gD = c->gD;
    a.ldP = ld;
    a.newRM = c->newRM_b;
    a.ntiles = c->ntiles;
    a.T = T;
    a.tau_EI = c->tau_EI;
    a.L = c->L;
    a.seed = c->seed;
    for (int k = 0; k < kMaxL; ++k) a.c[k] = k < c->L ? c->c[k] : 0.f;
    const int Lm1 = c->L - 1;
    if (mode == kBwdFused || mode == kBwdSplit)   // every day's infectious rows, from the final state
        LAUNCH(launch_infectious_bits(c->e, 0, T, c->L, c->ntiles, c->bits, (size_t)c->ntiles, s));
    a.s_hist_t = a.y_hist_t = nullptr;
    a.s_hist = c->s_hist;
    a.y_hist = c->y_hist;
    a.hist_stride = (size_t)c->n_rows;
    a.sig = c->sig;
    a.emax = c->emax;
    a.ld_sig = ld + 1;
    a.dc_tile = c->want_dc ? c->dc_tile : nullptr;
    a.self_r = a.self_q = nullptr;
    a.fate = fate_ref(c);
    a.Pm_t = nullptr;
    a.dur = c->dur;
    const int grid = (c->fate || c->dur.n > 0) ? c->grid_bwd_fate : (a.dc_tile ? c->grid_bwd_dc : c->grid_bwd);
    if (c->fate)   // draw days 0..tau_EI-1 hold only the seeds' shares (k_fate_seeds)
        CK(cudaMemsetAsync(c->Pm, 0, sizeof(double) * (size_t)std::min(c->tau_EI, T) * c->ntiles, s));
    for (int t = T - 1; t >= 0; --t) {
        a.bits_t = (mode == kBwdFused || mode == kBwdSplit) ? c->bits + (size_t)t * c->ntiles : nullptr;
        a.t = t;
        a.lam_t = (mode == kBwdStore || mode == kBwdSoft) ? c->lam + (size_t)t * c->n_rows
                                                          : (mode == kBwdSplit ? c->lam_tmp : nullptr);
        if (mode == kBwdSoft) {
            a.s_hist_t = c->s_hist + (size_t)t * c->n_rows;
            a.y_hist_t = c->y_hist + (size_t)t * c->n_rows;
        }
        if (mode == kBwdSplit)
            LAUNCH(launch_lam_day(sell_view(c, false), c->e, c->bits + (size_t)t * c->ntiles, graph_ref(c), t, c->L,
                                  c->ntiles, c->c_dev, c->lam_tmp, c->grid_bwd, s));
        a.r_next = c->r + (size_t)((t + 1) & 1) * c->n_rows;
        a.r_cur = c->r + (size_t)(t & 1) * c->n_rows;
        if (c->two_hop) {   // the location hop of the transpose gather: gP = sum over members of w r(t+1)
            LAUNCH(launch_loc_adjoint(loc_sell_view(c), c->loc_ntiles, loc_big_view(c), a.r_next, c->c_dev, c->locv,
                                      c->grid_loc, s));
            a.self_r = a.r_next;
            a.self_q = c->self_q;
            a.r_next = c->locv;
        }
        a.P_t = c->P + (size_t)t * c->ntiles * kAges;
        if (c->fate) a.Pm_t = (t + c->tau_EI < T) ? c->Pm + (size_t)(t + c->tau_EI) * c->ntiles : nullptr;
        for (int k = 0; k < kMaxL; ++k) a.ring_slot[k] = (k >= 1 && k < c->L) ? (t + k) % Lm1 : 0;
        prof_begin(c, 1);
        LAUNCH(launch_bwd_day(a, grid, s));
        prof_end(c, 1);
    }
    if (c->fate)   // the fate draws of agents exposed before day 0 (r of day 0 is in slot 0)
        LAUNCH(launch_fate_seeds(sell_view(c, true), c->e, c->r, c->ring, (size_t)c->n_rows, Lm1, graph_ref(c), a.fate,
                                 c->gD, c->sig, ld + 1, c->ntiles, T, c->c_dev, c->Pm, c->grid_bwd, s));
    if (a.dc_tile) {   // the seeds' share through day 0 (r of day 0 is in slot 0)
        const float *r0 = c->r;
        if (c->two_hop) {
            LAUNCH(launch_loc_adjoint(loc_sell_view(c), c->loc_ntiles, loc_big_view(c), c->r, c->c_dev, c->locv,
                                      c->grid_loc, s));
            r0 = c->locv;
        }
        LAUNCH(launch_dc_seeds(sell_view(c, true), c->e, r0, graph_ref(c), c->sig, ld + 1, c->ntiles, c->L,
                               c->dc_tile, c->grid_bwd, s));
    }
    LAUNCH(launch_bwd_reduce(c->P, c->ntiles, ld, c->d_tile0, c->d_ntiles, T, c->I, c->sig, ld + 1, c->Q, s));
    return GABM_OK;
}

// Day loop of the soft relaxation (from day 0: the state comes from the seeded exposure days).
gabm_status forward_days_soft(gabm_ctx *c, int T, cudaStream_t s) {
    const size_t n = (size_t)c->n_rows;
    LAUNCH(launch_soft_init(c->e, c->n_rows, c->L, c->c_dev, c->s_soft, c->nh, c->x2, s));
    SoftDayArgs a;
    a.m = sell_view(c, false);
    a.age = c->age;
    a.gr = graph_ref(c);
    a.e = c->e;
    a.s = c->s_soft;
    a.nh = c->nh;
    a.R = c->R;
    a.S = c->S;
    a.ldP = c->Tcap;
    a.ntiles = c->ntiles;
    a.L = c->L;
    a.seed = c->seed;
    for (int k = 0; k < kMaxL; ++k) a.c[k] = k < c->L ? c->c[k] : 0.f;
    for (int t = 0; t < T; ++t) {
        a.t = t;
        a.x_cur = c->x2 + (size_t)(t & 1) * n;
        a.x_next = c->x2 + (size_t)((t + 1) & 1) * n;
        a.s_hist_t = c->s_hist + (size_t)t * n;
        a.y_hist_t = c->y_hist + (size_t)t * n;
        a.lam_t = c->lam + (size_t)t * n;
        a.P_nrm_t = c->P_nrm + (size_t)t * c->ntiles;
        prof_begin(c, 0);
        LAUNCH(launch_fwd_day_soft(a, c->grid_fwd, s));
        prof_end(c, 0);
    }
    return GABM_OK;
}

enum { kLoopForward = 0, kLoopBackward = 1 };

gabm_status day_loop(gabm_ctx *c, int which, int t0, int T, cudaStream_t s) {
    if (which == kLoopForward && c->soft) return forward_days_soft(c, T, s);
    if (which == kLoopForward) return c->batched ? forward_days_batched(c, t0, T, s) : forward_days_plain(c, t0, T, s);
    return c->batched ? backward_days_batched(c, T, s) : backward_days_plain(c, T, s);
}

void drop_graph(gabm_ctx::LoopGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = gabm_ctx::LoopGraph();
}

// Runs a day loop on the ctx stream: eagerly, or as a CUDA graph captured once
// per (loop, t0, T, buffer generation) and replayed on later calls.
gabm_status run_day_loop(gabm_ctx *c, int which, int t0, int T) {
    if (!c->use_graphs || c->profiling) return day_loop(c, which, t0, T, c->stream);
    gabm_ctx::LoopGraph &g = c->loop_graph[which];
    if (!g.exec || g.t0 != t0 || g.T != T || g.dc != c->want_dc || g.generation != c->buffer_generation) {
        drop_graph(g);
        if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        const uint64_t before = c->launches;
        gabm_status st = day_loop(c, which, t0, T, c->cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
        const uint64_t captured = c->launches - before;
        c->launches = before;
        if (st != GABM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return fail(c, GABM_ECUDA, "stream capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g.exec = nullptr;
            return fail(c, GABM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
        g.t0 = t0;
        g.T = T;
        g.dc = c->want_dc;
        g.generation = c->buffer_generation;
        g.kernels = captured;
    }
    CK(cudaGraphLaunch(g.exec, c->stream));
    c->launches += g.kernels;
    return GABM_OK;
}

// Forward over days t0..T-1 from the staged parameters: clears the per-day
// outputs, seeds the state (from last_seeds) when `seeding`, runs the day loop.
gabm_status forward_core(gabm_ctx *c, int t0, int T, bool seeding) {
    const int ld = c->Tcap;
    cudaStream_t s = c->stream;
    CK(cudaMemsetAsync(c->counts, 0, sizeof(int32_t) * 4 * (size_t)c->I * ld, s));
    CK(cudaMemsetAsync(c->newRM, 0, sizeof(int32_t) * (size_t)c->I * ld, s));
    CK(cudaMemsetAsync(c->D, 0, sizeof(double) * (size_t)c->I * ld, s));
    if (c->batched) CK(cudaMemsetAsync(c->tile_ctr, 0, sizeof(int) * (size_t)ld, s));

    if (seeding) {
        CK(cudaMemcpyAsync(c->d_nseed, c->last_seeds.data(), sizeof(int32_t) * c->I, cudaMemcpyHostToDevice, s));
        const int grid = (int)std::min<int64_t>((c->n_rows + 255) / 256, 65535);
        LAUNCH(launch_init_state(c->e, c->d_row0, c->d_rows, c->G, c->n_rows, c->B, c->Bp, grid, s));
        SeedArgs sa;
        sa.row0 = c->d_row0;
        sa.rows = c->d_rows;
        sa.orig_id = c->d_orig_id;
        sa.e = c->e;
        sa.B = c->B;
        sa.Bp = c->Bp;
        sa.st = c->seedst;
        sa.hist = c->hist;
        sa.ties = c->ties;
        sa.seed = c->seed;
        sa.tau_EI = c->tau_EI;
        int max_rows = 1;
        for (int g = 0; g < c->G; ++g) max_rows = std::max(max_rows, c->h_rows[g]);
        const int gx = std::max(1, std::min((max_rows + 255) / 256, 4 * c->num_sms / std::max(1, c->I) + 1));
        LAUNCH(launch_seed_reset(c->seedst, c->d_nseed, c->I, s));
        for (int pass = 0; pass < 3; ++pass) {
            sa.pass = pass;
            LAUNCH(launch_seed_hist(sa, c->I, gx, s));
            LAUNCH(launch_seed_scan(sa, c->I, s));
        }
        LAUNCH(launch_seed_mark(sa, c->I, gx, s));
        LAUNCH(launch_seed_ties(sa, c->I, s));
    }

    TRY(run_day_loop(c, kLoopForward, t0, T));
    return GABM_OK;
}

// Reverse sweep over days T-1..0 from the staged gD (per-tile sums into Q).
gabm_status backward_core(gabm_ctx *c, int T) {
    const int ld = c->Tcap;
    cudaStream_t s = c->stream;
    CK(cudaMemsetAsync(c->r, 0, sizeof(float) * 2 * (size_t)c->n_rows * c->Bp, s));
    CK(cudaMemsetAsync(c->newRM_b, 0, sizeof(int32_t) * (size_t)c->I * ld, s));
    if (c->batched) CK(cudaMemsetAsync(c->tile_ctr + ld, 0, sizeof(int) * (size_t)ld * max_bwd_chunks(c), s));
    // sigma(T) = 0 and no stored exponent yet
    CK(cudaMemsetAsync(c->sig, 0, sizeof(int32_t) * (size_t)c->G * (ld + 1), s));
    CK(cudaMemsetAsync(c->emax, 0, sizeof(int32_t) * (size_t)c->G * (ld + 1), s));
    if (c->soft) CK(cudaMemsetAsync(c->A, 0, sizeof(float) * (size_t)c->n_rows, s));   // dL/ds(T) = 0

    if (!c->batched && c->policy != GABM_STORE_LAMBDA && !c->symmetric && !c->lam_tmp)
        TRY(dalloc(c, &c->lam_tmp, (size_t)c->n_rows));
    return run_day_loop(c, kLoopBackward, 0, T);
}

// Grid sizes for the current schedule (resident blocks per SM x SMs, at most one warp per tile).
void apply_schedule(gabm_ctx *c) {
    const int mode = c->soft ? kBwdSoft
                             : (c->policy == GABM_STORE_LAMBDA ? kBwdStore : (c->symmetric ? kBwdFused : kBwdSplit));
    if (c->soft) {
        c->smem_bits = false;
        c->grid_fwd = c->num_sms * occupancy_fwd_soft();
        c->grid_bwd = c->num_sms * occupancy_bwd(mode);
        c->grid_bwd_dc = c->num_sms * occupancy_bwd(mode, true);
    } else if (c->batched) {
        c->grid_fwd = c->num_sms * occupancy_fwd_b(c->Bp, c->spl_fwd, c->kahan_b);
        c->grid_bwd = c->num_sms * occupancy_bwd_b(c->bwd_chunk, c->spl_bwd, c->kahan_b);
    } else {
        if (c->fate || c->dur.n > 0 || c->sirs) c->smem_bits = false;   // these forwards read the bitmap from global memory
        const int bps = c->smem_bits ? occupancy_fwd(c->ntiles, true) : 0;
        if (c->smem_bits && bps <= 0) c->smem_bits = false;
        // GABM_DAY_WAVES waves of blocks, each block a contiguous range of tiles: blocks that
        // finish early leave their SM to the next wave's blocks
        const int waves = std::max(1, GABM_DAY_WAVES);
        c->grid_fwd = c->num_sms * (c->smem_bits ? bps : occupancy_fwd(c->ntiles, false) * waves);
        c->grid_bwd = c->num_sms * occupancy_bwd(mode) * waves;
        c->grid_bwd_dc = c->num_sms * occupancy_bwd(mode, true);
        c->grid_bwd_fate = c->num_sms * occupancy_bwd(mode, false, c->fate ? kExitFate : kExitDur);
    }
    if (c->two_hop) {
        c->smem_bits = false;
        const int units = std::max(c->loc_ntiles, c->n_big);   // warp work units of the larger launch
        c->grid_loc = std::min(c->num_sms * occupancy_loc(), std::max(1, (units + kBlock / 32 - 1) / (kBlock / 32)));
    }
    const int max_grid = (c->ntiles + kBlock / 32 - 1) / (kBlock / 32);
    if (!c->smem_bits && c->grid_fwd > max_grid) c->grid_fwd = max_grid;
    if (c->grid_bwd > max_grid) c->grid_bwd = max_grid;
    if (c->grid_bwd_dc > max_grid) c->grid_bwd_dc = max_grid;
    if (c->grid_bwd_fate > max_grid) c->grid_bwd_fate = max_grid;
    c->grid_sirs_f = std::min(max_grid, c->num_sms * occupancy_sirs(false));
    c->grid_sirs_b = std::min(max_grid, c->num_sms * occupancy_sirs(true));
    for (auto &g : c->loop_graph) drop_graph(g);   // captured launches carry the old schedule
}

void destroy_all(gabm_ctx *c) {
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &g : c->loop_graph) drop_graph(g);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (auto &kv : c->sizes) cudaFree(kv.first);
    c->sizes.clear();
    for (int k = 0; k < 2; ++k)
        for (auto ev : c->ev[k]) cudaEventDestroy(ev);
}

}  // namespace

extern "C" {

const char *gabm_version(void) { return "gabm-gb300 0.1 (sm_103a)"; }

const char *gabm_last_error(const gabm_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

gabm_status gabm_agent_layout(const gabm_graph_desc *graph, int agent_order, int sets_per_graph,
                              uint32_t *order_out) {
    if (!graph) return fail(nullptr, GABM_EINVAL, "graph is NULL");
    if (!order_out) return fail(nullptr, GABM_EINVAL, "order_out is NULL");
    if (sets_per_graph < 1) return fail(nullptr, GABM_EINVAL, "sets_per_graph must be >= 1");
    if (agent_order != GABM_ORDER_INPUT && agent_order != GABM_ORDER_BFS && agent_order != GABM_ORDER_COMMUNITY)
        return fail(nullptr, GABM_EINVAL, "unknown agent_order %d", agent_order);
    HostGraph h;
    TRY(fetch_graph(*graph, 0, h));
    const std::vector<uint32_t> order = layout_order(h, agent_order, sets_per_graph);
    if (!order.empty()) memcpy(order_out, order.data(), sizeof(uint32_t) * order.size());
    return GABM_OK;
}

// Host-side layout of a ctx's graphs, ready for upload (built by gabm_create and
// gabm_create_bipartite).
struct HostLayout {
    HostSell sell_in, sell_out;
    std::vector<uint32_t> h_rowptr, h_col, t_rowptr, t_col;
    std::vector<float> h_w, t_w;
    std::vector<uint8_t> h_age;
    std::vector<uint16_t> tile_graph;
    std::vector<uint32_t> h_orig;
    std::vector<int64_t> goff;
    std::vector<int32_t> row0, rows, tile0, ntl;
    std::vector<double> Dbar;
    bool symmetric = true, batched = false, reorder = true;
    uint32_t max_degree = 0;
    int64_t n_rows = 0, nnz = 0, nnz_pad = 0, n_total = 0;
    int ntiles = 0, sigma = 1024, num_graphs = 1;
};

// Device side of ctx creation: upload the layout, allocate the state and buffers.
static gabm_status create_on_device(const HostLayout &H, const gabm_model_desc *model, int sets_per_graph,
                                    void *cuda_stream, gabm_ctx **out) {
    const HostSell &sell_in = H.sell_in, &sell_out = H.sell_out;
    const std::vector<uint32_t> &h_rowptr = H.h_rowptr, &h_col = H.h_col, &t_rowptr = H.t_rowptr, &t_col = H.t_col;
    const std::vector<float> &h_w = H.h_w, &t_w = H.t_w;
    const std::vector<uint8_t> &h_age = H.h_age;
    const std::vector<uint16_t> &tile_graph = H.tile_graph;
    const std::vector<uint32_t> &h_orig = H.h_orig;
    const std::vector<int64_t> &goff = H.goff;
    const std::vector<int32_t> &row0 = H.row0, &rows = H.rows, &tile0 = H.tile0, &ntl = H.ntl;
    const std::vector<double> &Dbar = H.Dbar;
    const bool symmetric = H.symmetric, batched = H.batched, reorder = H.reorder;
    const uint32_t max_degree = H.max_degree;
    const int64_t n_rows = H.n_rows, nnz = H.nnz, nnz_pad = H.nnz_pad, n_total = H.n_total;
    const int ntiles = H.ntiles, sigma = H.sigma, num_graphs = H.num_graphs;
    gabm_ctx *c = new gabm_ctx();
    c->stream = (cudaStream_t)cuda_stream;
    c->G = num_graphs;
    c->B = sets_per_graph;
    c->I = num_graphs * sets_per_graph;
    c->batched = batched;
    c->soft = model->relax_mode == GABM_SOFT;
    c->Bp = 1;
    if (batched) {
        c->Bp = 2;
        while (c->Bp < sets_per_graph) c->Bp *= 2;
    }
    c->kahan_b = max_degree > (uint32_t)kPlainSumMaxDegree;
    {
        int mx = 1;
        for (int g = 0; g < num_graphs; ++g) mx = std::max(mx, ntl[g]);
        c->max_chunks = (mx + kReduceChunkTiles - 1) / kReduceChunkTiles;
        c->max_graph_tiles = mx;
    }
    if (batched) {
        // widest vectors first: eight sets per lane keeps 32 / (Bp / 8) rows in flight per warp
        c->spl_fwd = c->spl_bwd = std::min(c->Bp, 8);
        c->bwd_chunk = c->Bp;
        if (const char *f = getenv("GABM_BATCH_SPL")) {
            const int v = atoi(f);
            if (batch_config_ok(c->Bp, v)) c->spl_fwd = c->spl_bwd = v;
        }
    }
    c->tau_EI = model->tau_EI;
    c->tau_IR = model->tau_IR;
    c->tau_IM = model->tau_IM;
    c->fate = model->tau_IM > 0;
    c->L_R = model->tau_EI + model->tau_IR;
    c->L_M = model->tau_EI + model->tau_IM;
    c->L = model->tau_EI + std::max(model->tau_IR, model->tau_IM);
    c->sirs = model->tau_RS > 0;
    c->tau_RS = model->tau_RS;
    c->cycle = c->L + model->tau_RS;
    c->dur = DurRef{};
    if (model->p_IR) {   // running sums of the duration pmf, in order, in FP64
        c->dur.n = model->tau_IR;
        c->dur.tau_EI = model->tau_EI;
        c->dur.seed = model->seed;
        double acc = 0.0;
        for (int j = 0; j < model->tau_IR; ++j) {
            acc += (double)model->p_IR[j];
            c->dur.F[j] = acc;
        }
    }
    for (int k = 0; k < c->L; ++k) c->c[k] = model->c[k];
    c->seed = model->seed;
    c->policy = model->lambda_policy;
    c->n_total = n_total;
    c->n_rows = n_rows;
    c->nnz = nnz;
    c->nnz_pad = nnz_pad;
    c->ntiles = ntiles;
    c->h_row0 = row0;
    c->h_rows = rows;
    c->h_tile0 = tile0;
    c->h_ntiles = ntl;
    c->h_Dbar = Dbar;
    c->symmetric = symmetric;
    if (const char *f = getenv("GABM_FAIL_ALLOC_AFTER")) c->fail_alloc_after = atol(f);
    if (const char *f = getenv("GABM_CUDA_GRAPHS")) c->use_graphs = atoi(f) != 0;

    auto bail = [&](gabm_status st) {
        g_create_error = c->err;
        destroy_all(c);
        delete c;
        return st;
    };
#define CTRY(call)                              \
    do {                                        \
        gabm_status s_ = (call);                \
        if (s_ != GABM_OK) return bail(s_);     \
    } while (0)
#define CCK(call)                                                                                       \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return bail(fail(c, GABM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_))); \
    } while (0)

    CCK(cudaGetDevice(&c->device));
    CCK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));

    c->sigma = sigma;
    c->sell_entries = batched ? 0 : (int64_t)sell_in.slice_ptr.back();
    auto upload_sell = [&](const HostSell &hs, uint32_t *&sp, uint32_t *&rl, uint32_t *&cl, float *&ww) -> gabm_status {
        TRY(dalloc(c, &sp, hs.slice_ptr.size()));
        TRY(dalloc(c, &rl, hs.row_len.size()));
        TRY(dalloc(c, &cl, hs.col.size()));
        TRY(dalloc(c, &ww, hs.w.size()));
        CK(cudaMemcpyAsync(sp, hs.slice_ptr.data(), sizeof(uint32_t) * hs.slice_ptr.size(), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(rl, hs.row_len.data(), sizeof(uint32_t) * hs.row_len.size(), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(cl, hs.col.data(), sizeof(uint32_t) * hs.col.size(), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(ww, hs.w.data(), sizeof(float) * hs.w.size(), cudaMemcpyHostToDevice, c->stream));
        return GABM_OK;
    };
    auto upload_csr = [&](const std::vector<uint32_t> &rp, const std::vector<uint32_t> &cl, const std::vector<float> &ww,
                          uint32_t *&drp, uint32_t *&dcl, float *&dw) -> gabm_status {
        TRY(dalloc(c, &drp, rp.size()));
        TRY(dalloc(c, &dcl, cl.size()));
        TRY(dalloc(c, &dw, ww.size()));
        CK(cudaMemcpyAsync(drp, rp.data(), sizeof(uint32_t) * rp.size(), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(dcl, cl.data(), sizeof(uint32_t) * cl.size(), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(dw, ww.data(), sizeof(float) * ww.size(), cudaMemcpyHostToDevice, c->stream));
        return GABM_OK;
    };
    if (batched) {
        CTRY(upload_csr(h_rowptr, h_col, h_w, c->csr_rowptr, c->csr_col, c->csr_w));
        if (symmetric) {
            c->t_csr_rowptr = c->csr_rowptr;
            c->t_csr_col = c->csr_col;
            c->t_csr_w = c->csr_w;
        } else {
            CTRY(upload_csr(t_rowptr, t_col, t_w, c->t_csr_rowptr, c->t_csr_col, c->t_csr_w));
        }
    } else {
        CTRY(upload_sell(sell_in, c->slice_ptr, c->row_len, c->scol, c->sw));
        if (symmetric) {
            c->t_slice_ptr = c->slice_ptr;
            c->t_row_len = c->row_len;
            c->t_scol = c->scol;
            c->t_sw = c->sw;
        } else {
            CTRY(upload_sell(sell_out, c->t_slice_ptr, c->t_row_len, c->t_scol, c->t_sw));
        }
    }
    CTRY(dalloc(c, &c->age, (size_t)n_rows));
    CCK(cudaMemcpyAsync(c->age, h_age.data(), h_age.size(), cudaMemcpyHostToDevice, c->stream));
    // the host copies above read vectors that go out of scope at return
    CCK(cudaStreamSynchronize(c->stream));
    std::vector<float> inv((size_t)num_graphs);
    for (int g = 0; g < num_graphs; ++g) inv[g] = Dbar[g] > 0.0 ? (float)(1.0 / Dbar[g]) : 0.0f;
    CTRY(dalloc(c, &c->d_row0, (size_t)num_graphs));
    CTRY(dalloc(c, &c->d_rows, (size_t)num_graphs));
    CTRY(dalloc(c, &c->d_tile0, (size_t)num_graphs));
    CTRY(dalloc(c, &c->d_ntiles, (size_t)num_graphs));
    CTRY(dalloc(c, &c->d_inv_Dbar, (size_t)num_graphs));
    CTRY(dalloc(c, &c->d_tile_graph, (size_t)ntiles));
    CTRY(dalloc(c, &c->d_goff, (size_t)num_graphs));
    CCK(cudaMemcpyAsync(c->d_goff, goff.data(), sizeof(int64_t) * num_graphs, cudaMemcpyHostToDevice, c->stream));
    if (reorder) {
        CTRY(dalloc(c, &c->d_orig_id, (size_t)n_rows));
        CCK(cudaMemcpyAsync(c->d_orig_id, h_orig.data(), sizeof(uint32_t) * n_rows, cudaMemcpyHostToDevice, c->stream));
    }
    CCK(cudaMemcpyAsync(c->d_row0, row0.data(), sizeof(int32_t) * num_graphs, cudaMemcpyHostToDevice, c->stream));
    CCK(cudaMemcpyAsync(c->d_rows, rows.data(), sizeof(int32_t) * num_graphs, cudaMemcpyHostToDevice, c->stream));
    CCK(cudaMemcpyAsync(c->d_tile0, tile0.data(), sizeof(int32_t) * num_graphs, cudaMemcpyHostToDevice, c->stream));
    CCK(cudaMemcpyAsync(c->d_ntiles, ntl.data(), sizeof(int32_t) * num_graphs, cudaMemcpyHostToDevice, c->stream));
    CCK(cudaMemcpyAsync(c->d_inv_Dbar, inv.data(), sizeof(float) * num_graphs, cudaMemcpyHostToDevice, c->stream));
    CCK(cudaMemcpyAsync(c->d_tile_graph, tile_graph.data(), sizeof(uint16_t) * ntiles, cudaMemcpyHostToDevice, c->stream));

    const size_t nb = (size_t)n_rows * c->Bp;   // agent-set slots
    CTRY(dalloc(c, &c->e, nb));
    CTRY(dalloc(c, &c->ring, (size_t)(c->L - 1) * nb));
    CTRY(dalloc(c, &c->A, nb));
    CTRY(dalloc(c, &c->r, (size_t)2 * nb));
    CTRY(dalloc(c, &c->rows_f, nb));
    CTRY(dalloc(c, &c->rows_e, nb));
    CTRY(dalloc(c, &c->stage_f, nb));
    if (batched) {
        CTRY(dalloc(c, &c->rbits, (size_t)2 * ntiles * std::max(1, c->Bp / 2)));
        CTRY(dalloc(c, &c->hist0, (size_t)c->I * (c->L + 2)));
    } else if (!c->soft) {
        CTRY(dalloc(c, &c->flags, (size_t)3 * n_rows));
    }
    if (c->soft) {
        CTRY(dalloc(c, &c->s_soft, (size_t)n_rows));
        CTRY(dalloc(c, &c->nh, (size_t)c->L * n_rows));
        CTRY(dalloc(c, &c->x2, (size_t)2 * n_rows));
    }
    CTRY(dalloc(c, &c->S, (size_t)c->I * kAges));
    CTRY(dalloc(c, &c->dS_s, (size_t)c->I * kAges));
    CTRY(dalloc(c, &c->loss_s, (size_t)c->I));
    CTRY(dalloc(c, &c->seedst, (size_t)c->I));
    CTRY(dalloc(c, &c->hist, (size_t)c->I * kHistBins));
    CTRY(dalloc(c, &c->ties, (size_t)c->I * kTieCap));
    CTRY(dalloc(c, &c->d_nseed, (size_t)c->I));
    CTRY(dalloc(c, &c->c_dev, (size_t)kMaxL));
    CCK(cudaMemcpyAsync(c->c_dev, c->c, sizeof(float) * kMaxL, cudaMemcpyHostToDevice, c->stream));
    CCK(cudaMemsetAsync(c->hist, 0, sizeof(uint32_t) * (size_t)c->I * kHistBins, c->stream));
    {
        int grid = (int)std::min<int64_t>((n_rows + 255) / 256, 65535);
        cudaError_t e = launch_init_state(c->e, c->d_row0, c->d_rows, c->G, n_rows, c->B, c->Bp, grid, c->stream);
        c->launches++;
        if (e != cudaSuccess) return bail(fail(c, GABM_ECUDA, "init state: %s", cudaGetErrorString(e)));
    }
    {
        // the bitmap read through L1 is the default: with branch-free gathers it beats the
        // shared-memory copy, whose one large block per SM limits the warps in flight
        const char *f = getenv("GABM_FWD_SMEM_BITS");
        c->smem_bits = !batched && f && atoi(f) == 1;
    }
    apply_schedule(c);
    CTRY(ensure_days(c, 8));
    CCK(cudaStreamSynchronize(c->stream));
#undef CTRY
#undef CCK
    *out = c;
    return GABM_OK;
}

gabm_status gabm_create(const gabm_graph_desc *graphs, int num_graphs, int sets_per_graph,
                        const gabm_model_desc *model, void *cuda_stream, gabm_ctx **out) {
    g_create_error.clear();
    if (!out) return fail(nullptr, GABM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!graphs || num_graphs < 1 || num_graphs > 65535) return fail(nullptr, GABM_EINVAL, "need 1..65535 graphs");
    if (sets_per_graph < 1) return fail(nullptr, GABM_EINVAL, "sets_per_graph must be >= 1");
    if (sets_per_graph > kMaxSets) return fail(nullptr, GABM_EUNSUPPORTED, "sets_per_graph > %d", kMaxSets);
    TRY(validate_model(model));
    if (model->relax_mode == GABM_SOFT && (sets_per_graph > 1 || model->lambda_policy != GABM_STORE_LAMBDA))
        return fail(nullptr, GABM_EUNSUPPORTED, "GABM_SOFT needs sets_per_graph = 1 and GABM_STORE_LAMBDA in this build");
    if ((model->tau_IM > 0 || model->p_IR) && (model->relax_mode != GABM_HARD_ST || sets_per_graph > 1 ||
                                               model->lambda_policy != GABM_STORE_LAMBDA))
        return fail(nullptr, GABM_EUNSUPPORTED, "the sampled R/M split (tau_IM > 0) and stochastic durations (p_IR) "
                    "need GABM_HARD_ST, sets_per_graph = 1 and GABM_STORE_LAMBDA in this build");
    if (model->tau_IM > 0 && model->p_IR)
        return fail(nullptr, GABM_EUNSUPPORTED, "tau_IM > 0 with p_IR is not built");
    if (model->tau_RS > 0 && (model->relax_mode != GABM_HARD_ST || sets_per_graph > 1 ||
                              model->lambda_policy != GABM_STORE_LAMBDA || model->tau_IM > 0 || model->p_IR))
        return fail(nullptr, GABM_EUNSUPPORTED, "SIRS reinfection (tau_RS > 0) needs GABM_HARD_ST, sets_per_graph = 1, "
                    "GABM_STORE_LAMBDA, tau_IM = 0 and p_IR = NULL in this build");

    // ---- host side: validate, concatenate, transpose ----
    std::vector<HostGraph> hg((size_t)num_graphs);
    bool any_device = false;
    for (int g = 0; g < num_graphs; ++g) any_device |= (graphs[g].mem_space == GABM_DEVICE);
    for (int g = 0; g < num_graphs; ++g) TRY(fetch_graph(graphs[g], g, hg[g]));
    (void)any_device;

    std::vector<int32_t> row0(num_graphs), rows(num_graphs), tile0(num_graphs), ntl(num_graphs);
    std::vector<double> Dbar(num_graphs);
    int64_t n_rows = 0, nnz = 0, n_total = 0;
    for (int g = 0; g < num_graphs; ++g) {
        row0[g] = (int32_t)n_rows;
        rows[g] = (int32_t)hg[g].n;
        tile0[g] = (int32_t)(n_rows / kTile);
        const int64_t padded = (int64_t)round_up((size_t)hg[g].n, kTile);
        ntl[g] = (int32_t)(padded / kTile);
        n_rows += padded;
        nnz += hg[g].nnz;
        n_total += hg[g].n;
        double s = 0.0;
        for (int64_t p = 0; p < hg[g].nnz; ++p) s += (double)hg[g].w[p];
        Dbar[g] = hg[g].n > 0 ? s / (double)hg[g].n : 0.0;
    }
    // device layout: relabel each graph's agents (D-bar above uses the caller's order)
    std::vector<std::vector<uint32_t>> orders((size_t)num_graphs);
    const bool reorder = true;
    for (int g = 0; g < num_graphs; ++g) {
        orders[g] = layout_order(hg[g], model->agent_order, sets_per_graph);
        hg[g] = permute_graph(hg[g], orders[g]);
    }
    if (n_rows >= ((int64_t)1 << 31) - 64) return fail(nullptr, GABM_EUNSUPPORTED, "total rows >= 2^31");
    if (nnz >= ((int64_t)1 << 32) - 64) return fail(nullptr, GABM_EUNSUPPORTED, "total nnz >= 2^32");
    if (n_rows == 0) n_rows = kTile;  // keep one (padding) tile so every buffer is non-empty
    const int64_t nnz_pad = (int64_t)round_up((size_t)(nnz > 0 ? nnz : 1), 4);
    const int ntiles = (int)(n_rows / kTile);

    std::vector<uint32_t> h_rowptr((size_t)n_rows + 1), h_col((size_t)nnz_pad, 0u);
    std::vector<float> h_w((size_t)nnz_pad, 0.f);
    std::vector<uint8_t> h_age((size_t)n_rows, 0);
    std::vector<uint32_t> t_rowptr((size_t)n_rows + 1), t_col((size_t)nnz_pad, 0u);
    std::vector<float> t_w((size_t)nnz_pad, 0.f);
    std::vector<uint16_t> tile_graph((size_t)ntiles, 0);
    std::vector<uint32_t> h_orig(reorder ? (size_t)n_rows : 0, 0u);
    std::vector<int64_t> goff((size_t)num_graphs, 0);
    for (int g = 1; g < num_graphs; ++g) goff[g] = goff[g - 1] + hg[g - 1].n;
    bool symmetric = true;
    {
        int64_t e0 = 0;
        for (int g = 0; g < num_graphs; ++g) {
            const HostGraph &h = hg[g];
            std::vector<uint64_t> trp;
            std::vector<uint32_t> tc;
            std::vector<float> tw;
            transpose_graph(h, trp, tc, tw);
            const int64_t padded = (int64_t)ntl[g] * kTile;
            for (int64_t i = 0; i < padded; ++i) {
                const int64_t r = row0[g] + i;
                h_rowptr[r] = (uint32_t)(e0 + (int64_t)h.rowptr[i < h.n ? i : h.n]);
                t_rowptr[r] = (uint32_t)(e0 + (int64_t)trp[i < h.n ? i : h.n]);
                if (i < h.n) h_age[r] = h.age[i];
                if (reorder && i < h.n) h_orig[r] = orders[g][i];
            }
            for (int64_t p = 0; p < h.nnz; ++p) {
                h_col[e0 + p] = h.col[p] + (uint32_t)row0[g];
                h_w[e0 + p] = h.w[p];
                t_col[e0 + p] = tc[p] + (uint32_t)row0[g];
                t_w[e0 + p] = tw[p];
            }
            for (int k = 0; k < ntl[g]; ++k) tile_graph[tile0[g] + k] = (uint16_t)g;
            e0 += h.nnz;
        }
        h_rowptr[n_rows] = (uint32_t)e0;
        t_rowptr[n_rows] = (uint32_t)e0;
        symmetric = (h_rowptr == t_rowptr) && (h_col == t_col) &&
                    (memcmp(h_w.data(), t_w.data(), sizeof(float) * h_w.size()) == 0);
    }
    HostSell sell_in, sell_out;
    const bool batched = sets_per_graph > 1;
    if (batched && model->lambda_policy != GABM_STORE_LAMBDA && !symmetric)
        return fail(nullptr, GABM_EUNSUPPORTED, "sets_per_graph > 1 with GABM_RECOMPUTE needs symmetric weights in this build");
    if (!batched && (!build_sell(h_rowptr, h_col, h_w, n_rows, sell_in) ||
                     (!symmetric && !build_sell(t_rowptr, t_col, t_w, n_rows, sell_out))))
        return fail(nullptr, GABM_EUNSUPPORTED, "SELL-32 layout needs >= 2^32 entries");
    uint32_t max_degree = 0;
    for (int64_t r = 0; r < n_rows; ++r) {
        max_degree = std::max(max_degree, h_rowptr[r + 1] - h_rowptr[r]);
        max_degree = std::max(max_degree, t_rowptr[r + 1] - t_rowptr[r]);
    }

    HostLayout H;
    H.sell_in = std::move(sell_in);
    H.sell_out = std::move(sell_out);
    H.h_rowptr = std::move(h_rowptr);
    H.h_col = std::move(h_col);
    H.h_w = std::move(h_w);
    H.t_rowptr = std::move(t_rowptr);
    H.t_col = std::move(t_col);
    H.t_w = std::move(t_w);
    H.h_age = std::move(h_age);
    H.tile_graph = std::move(tile_graph);
    H.h_orig = std::move(h_orig);
    H.goff = std::move(goff);
    H.row0 = row0;
    H.rows = rows;
    H.tile0 = tile0;
    H.ntl = ntl;
    H.Dbar = Dbar;
    H.symmetric = symmetric;
    H.batched = batched;
    H.reorder = reorder;
    H.max_degree = max_degree;
    H.n_rows = n_rows;
    H.nnz = nnz;
    H.nnz_pad = nnz_pad;
    H.ntiles = ntiles;
    H.n_total = n_total;
    H.sigma = sell_sigma();
    H.num_graphs = num_graphs;
    return create_on_device(H, model, sets_per_graph, cuda_stream, out);
}

gabm_status gabm_create_bipartite(const gabm_bipartite_desc *graphs, int num_graphs, const gabm_model_desc *model,
                                  void *cuda_stream, gabm_ctx **out) {
    g_create_error.clear();
    if (!out) return fail(nullptr, GABM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!graphs || num_graphs < 1 || num_graphs > 65535) return fail(nullptr, GABM_EINVAL, "need 1..65535 graphs");
    TRY(validate_model(model));
    if (model->relax_mode != GABM_HARD_ST || model->lambda_policy != GABM_STORE_LAMBDA || model->tau_IM > 0 ||
        model->p_IR || model->tau_RS > 0)
        return fail(nullptr, GABM_EUNSUPPORTED, "agent-location graphs need GABM_HARD_ST, GABM_STORE_LAMBDA, "
                    "tau_IM = 0 and p_IR = NULL in this build");
    int sigma = 1024;
    if (const char *f = getenv("GABM_SELL_SIGMA")) sigma = std::max(1, atoi(f));
    const int G = num_graphs;

    // per graph: validate; each agent's attendances by location, repeats merged (their
    // weights add); Dbar of W_ij = sum_l w_il w_jl (i != j) = (1/n) sum_l [(sum_i w_il)^2 - sum_i w_il^2];
    // agents in input order sorted by attendance count within windows.  Locations of all
    // graphs form one pool (graph g's location l is loc_off[g] + l): no location is shared
    // between graphs, so the graphs stay independent.
    std::vector<std::vector<uint64_t>> arow((size_t)G);
    std::vector<std::vector<uint32_t>> aloc((size_t)G), order((size_t)G);
    std::vector<std::vector<float>> aw((size_t)G);
    std::vector<double> Dbar((size_t)G);
    std::vector<int64_t> loc_off((size_t)G + 1, 0);
    int64_t n_total = 0, m_total = 0, n_rows = 0;
    std::vector<int32_t> row0((size_t)G), rows((size_t)G), tile0((size_t)G), ntl((size_t)G);
    for (int g = 0; g < G; ++g) {
        const gabm_bipartite_desc *bip = graphs + g;
        const int64_t n = bip->n_agents, nl = bip->n_locations, nnz = bip->nnz;
        if (n < 1 || nl < 1 || nnz < 0) return fail(nullptr, GABM_EINVAL, "graph %d: need n_agents >= 1, n_locations >= 1 and nnz >= 0", g);
        if (!bip->rowptr || !bip->age || (nnz > 0 && (!bip->loc || !bip->w)))
            return fail(nullptr, GABM_EINVAL, "graph %d: rowptr, loc, w and age are required", g);
        if (n >= ((int64_t)1 << 31) - 64 || nl >= ((int64_t)1 << 31) - 64 || nnz >= ((int64_t)1 << 32) - 64)
            return fail(nullptr, GABM_EUNSUPPORTED, "graph %d: agents, locations and attendances must stay below 2^31, 2^31, 2^32", g);
        if (bip->rowptr[0] != 0 || (int64_t)bip->rowptr[n] != nnz)
            return fail(nullptr, GABM_EINVAL, "graph %d: rowptr[0] must be 0 and rowptr[n] = nnz", g);
        for (int64_t i = 0; i < n; ++i) {
            if (bip->rowptr[i + 1] < bip->rowptr[i]) return fail(nullptr, GABM_EINVAL, "graph %d: rowptr decreases at agent %lld", g, (long long)i);
            if (bip->age[i] >= kAges) return fail(nullptr, GABM_EINVAL, "graph %d: age[%lld] = %d out of 0..8", g, (long long)i, (int)bip->age[i]);
        }
        for (int64_t p = 0; p < nnz; ++p) {
            if ((int64_t)bip->loc[p] >= nl) return fail(nullptr, GABM_EINVAL, "graph %d: loc[%lld] = %u out of range", g, (long long)p, bip->loc[p]);
            if (!std::isfinite(bip->w[p]) || bip->w[p] < 0.0f) return fail(nullptr, GABM_EINVAL, "graph %d: w[%lld] not finite and >= 0", g, (long long)p);
        }
        std::vector<uint64_t> &ar = arow[g];
        std::vector<uint32_t> &al = aloc[g];
        std::vector<float> &awg = aw[g];
        ar.assign((size_t)n + 1, 0);
        al.reserve((size_t)nnz);
        awg.reserve((size_t)nnz);
        std::vector<std::pair<uint32_t, float>> tmp;
        for (int64_t i = 0; i < n; ++i) {
            tmp.clear();
            for (uint64_t p = bip->rowptr[i]; p < bip->rowptr[i + 1]; ++p) tmp.emplace_back(bip->loc[p], bip->w[p]);
            std::stable_sort(tmp.begin(), tmp.end(), [](const std::pair<uint32_t, float> &a, const std::pair<uint32_t, float> &b) {
                return a.first < b.first;
            });
            for (size_t k = 0; k < tmp.size(); ++k) {
                if (ar[i] < al.size() && al.back() == tmp[k].first) awg.back() += tmp[k].second;
                else { al.push_back(tmp[k].first); awg.push_back(tmp[k].second); }
            }
            ar[i + 1] = al.size();
        }
        std::vector<double> s1((size_t)nl, 0.0), s2((size_t)nl, 0.0);
        for (size_t p = 0; p < al.size(); ++p) {
            s1[al[p]] += (double)awg[p];
            s2[al[p]] += (double)awg[p] * (double)awg[p];
        }
        double D = 0.0;
        for (int64_t l = 0; l < nl; ++l) D += s1[l] * s1[l] - s2[l];
        Dbar[g] = D / (double)n;
        HostGraph h;
        h.n = n;
        h.nnz = (int64_t)al.size();
        h.rowptr = ar;
        order[g].resize((size_t)n);
        for (int64_t i = 0; i < n; ++i) order[g][i] = (uint32_t)i;
        sort_windows_by_degree(h, order[g], sigma);
        loc_off[g + 1] = loc_off[g] + nl;
        row0[g] = (int32_t)n_rows;
        rows[g] = (int32_t)n;
        tile0[g] = (int32_t)(n_rows / kTile);
        ntl[g] = (int32_t)(round_up((size_t)n, kTile) / kTile);
        n_rows += (int64_t)ntl[g] * kTile;
        n_total += n;
        m_total += (int64_t)al.size();
    }
    if (n_rows >= ((int64_t)1 << 31) - 64 || loc_off[G] >= ((int64_t)1 << 31) - 64 || m_total >= ((int64_t)1 << 32) - 64)
        return fail(nullptr, GABM_EUNSUPPORTED, "total agents, locations and attendances must stay below 2^31, 2^31, 2^32");
    const int64_t nl = loc_off[G], m = m_total, n = n_total;
    // locations of up to 32 members: SELL-32 tiles, sorted by member count within windows;
    // larger ones: a CSR taken one warp per location, sorted by member count
    constexpr uint32_t kSmallLoc = 32;
    std::vector<uint32_t> lcnt((size_t)nl, 0), lsmall, lbig, linv((size_t)nl);
    for (int g = 0; g < G; ++g)
        for (uint32_t l : aloc[g]) lcnt[loc_off[g] + l]++;
    for (int64_t l = 0; l < nl; ++l) (lcnt[l] <= kSmallLoc ? lsmall : lbig).push_back((uint32_t)l);
    for (size_t w0 = 0; w0 < lsmall.size(); w0 += (size_t)sigma) {
        const size_t w1 = std::min(lsmall.size(), w0 + (size_t)sigma);
        std::stable_sort(lsmall.begin() + w0, lsmall.begin() + w1, [&](uint32_t a, uint32_t b) { return lcnt[a] > lcnt[b]; });
    }
    std::stable_sort(lbig.begin(), lbig.end(), [&](uint32_t a, uint32_t b) { return lcnt[a] > lcnt[b]; });
    const int64_t ns_rows = (int64_t)round_up(lsmall.size(), kTile);
    const int64_t n_big = (int64_t)lbig.size();
    for (size_t k = 0; k < lsmall.size(); ++k) linv[lsmall[k]] = (uint32_t)k;
    for (int64_t k = 0; k < n_big; ++k) linv[lbig[k]] = (uint32_t)(ns_rows + k);

    HostLayout H;
    const int ntiles = (int)(n_rows / kTile);
    const int64_t nnz_pad = (int64_t)round_up((size_t)(m > 0 ? m : 1), 4);
    H.h_rowptr.assign((size_t)n_rows + 1, 0u);
    H.h_col.assign((size_t)nnz_pad, 0u);
    H.h_w.assign((size_t)nnz_pad, 0.f);
    H.h_age.assign((size_t)n_rows, 0);
    H.h_orig.assign((size_t)n_rows, 0u);
    H.tile_graph.assign((size_t)ntiles, 0);
    H.goff.assign((size_t)G, 0);
    for (int g = 1; g < G; ++g) H.goff[g] = H.goff[g - 1] + rows[g - 1];
    uint32_t max_degree = 0;
    {
        std::vector<std::pair<uint32_t, float>> tmp;
        uint32_t q = 0;
        for (int g = 0; g < G; ++g) {
            const gabm_bipartite_desc *bip = graphs + g;
            for (int32_t k = 0; k < ntl[g] * kTile; ++k) {
                const int64_t r = row0[g] + k;
                H.h_rowptr[r] = q;
                if (k >= rows[g]) continue;
                const uint32_t v = order[g][k];
                tmp.clear();
                for (uint64_t p = arow[g][v]; p < arow[g][v + 1]; ++p) tmp.emplace_back(linv[loc_off[g] + aloc[g][p]], aw[g][p]);
                std::sort(tmp.begin(), tmp.end(), [](const std::pair<uint32_t, float> &a, const std::pair<uint32_t, float> &b) {
                    return a.first < b.first;
                });
                for (const auto &e : tmp) { H.h_col[q] = e.first; H.h_w[q] = e.second; ++q; }
                max_degree = std::max(max_degree, (uint32_t)tmp.size());
                H.h_age[r] = bip->age[v];
                H.h_orig[r] = v;
            }
            for (int k = 0; k < ntl[g]; ++k) H.tile_graph[tile0[g] + k] = (uint16_t)g;
        }
        H.h_rowptr[n_rows] = q;
    }
    // locations -> members (agent rows ascending): small ones padded to whole tiles, large ones a CSR
    std::vector<uint32_t> lrow((size_t)ns_rows + 1, 0u), brow((size_t)n_big + 1, 0u);
    for (int64_t p = 0; p < m; ++p) {
        const uint32_t l = H.h_col[p];
        if (l < (uint32_t)ns_rows) lrow[l + 1]++;
        else brow[l - ns_rows + 1]++;
    }
    for (int64_t k = 0; k < ns_rows; ++k) lrow[k + 1] += lrow[k];
    for (int64_t k = 0; k < n_big; ++k) brow[k + 1] += brow[k];
    std::vector<uint32_t> lcol((size_t)std::max<uint32_t>(lrow.back(), 1), 0u), bcol((size_t)std::max<uint32_t>(brow.back(), 1), 0u);
    std::vector<float> lw(lcol.size(), 0.f), bw(bcol.size(), 0.f);
    {
        std::vector<uint32_t> pos(lrow.begin(), lrow.end() - 1), bpos(brow.begin(), brow.end() - 1);
        for (int64_t k = 0; k < n_rows; ++k)
            for (uint32_t p = H.h_rowptr[k]; p < H.h_rowptr[k + 1]; ++p) {
                const uint32_t l = H.h_col[p];
                const uint32_t q = (l < (uint32_t)ns_rows) ? pos[l]++ : bpos[l - ns_rows]++;
                (l < (uint32_t)ns_rows ? lcol : bcol)[q] = (uint32_t)k;
                (l < (uint32_t)ns_rows ? lw : bw)[q] = H.h_w[p];
            }
    }
    HostSell loc_sell;
    if (!build_sell(H.h_rowptr, H.h_col, H.h_w, n_rows, H.sell_in) || !build_sell(lrow, lcol, lw, ns_rows, loc_sell))
        return fail(nullptr, GABM_EUNSUPPORTED, "SELL-32 layout needs >= 2^32 entries");
    H.t_rowptr = H.h_rowptr;
    H.t_col = H.h_col;
    H.t_w = H.h_w;
    H.row0 = row0;
    H.rows = rows;
    H.tile0 = tile0;
    H.ntl = ntl;
    H.Dbar = Dbar;
    H.symmetric = true;
    H.batched = false;
    H.reorder = true;
    H.max_degree = max_degree;
    H.n_rows = n_rows;
    H.nnz = m;
    H.nnz_pad = nnz_pad;
    H.ntiles = ntiles;
    H.n_total = n;
    H.sigma = sigma;
    H.num_graphs = G;
    gabm_ctx *c = nullptr;
    TRY(create_on_device(H, model, 1, cuda_stream, &c));
    auto bail = [&](gabm_status st) {
        g_create_error = c->err;
        destroy_all(c);
        delete c;
        return st;
    };
    // the location hop: its SELL-32 and one value per location
    c->two_hop = true;
    c->n_loc = nl;
    c->loc_ntiles = (int)(ns_rows / kTile);
    c->n_big = (int)n_big;
    gabm_status st = GABM_OK;
    auto up = [&](auto *&dst, const auto &src) -> gabm_status {
        TRY(dalloc(c, &dst, src.size()));
        CK(cudaMemcpy(dst, src.data(), sizeof(src[0]) * src.size(), cudaMemcpyHostToDevice));
        return GABM_OK;
    };
    if (st == GABM_OK) st = up(c->loc_slice_ptr, loc_sell.slice_ptr);
    if (st == GABM_OK) st = up(c->loc_row_len, loc_sell.row_len);
    if (st == GABM_OK) st = up(c->loc_col, loc_sell.col);
    if (st == GABM_OK) st = up(c->loc_w, loc_sell.w);
    if (st == GABM_OK) st = up(c->big_rowptr, brow);
    if (st == GABM_OK) st = up(c->big_col, bcol);
    if (st == GABM_OK) st = up(c->big_w, bw);
    if (st == GABM_OK) st = dalloc(c, &c->locv, (size_t)std::max<int64_t>(1, ns_rows + n_big));
    {
        std::vector<float> q((size_t)n_rows, 0.f);
        for (int64_t k = 0; k < n_rows; ++k) {
            double acc = 0.0;
            for (uint32_t p = H.h_rowptr[k]; p < H.h_rowptr[k + 1]; ++p) acc += (double)H.h_w[p] * (double)H.h_w[p];
            q[k] = (float)acc;
        }
        if (st == GABM_OK) st = up(c->self_q, q);
    }
    if (st != GABM_OK) return bail(st);
    apply_schedule(c);
    *out = c;
    return GABM_OK;
}

void gabm_destroy(gabm_ctx *ctx) {
    if (!ctx) return;
    destroy_all(ctx);
    delete ctx;
}

gabm_status gabm_forward(gabm_ctx *ctx, int T, const float *R, const float *m, const float *S_age,
                         const int32_t *n_seed, double *D, int32_t *counts, int mem_space) {
    gabm_ctx *c = ctx;
    if (!c) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    TRY(check_ms(c, mem_space));
    if (T < 1 || T > GABM_MAX_DAYS) return fail(c, GABM_EINVAL, "T = %d outside 1..%d", T, GABM_MAX_DAYS);
    if (!R || !m || !S_age) return fail(c, GABM_EINVAL, "R, m and S_age are required");
    const int t0 = c->resumed ? c->t0_next : 0;
    if (t0 > T) return fail(c, GABM_EINVAL, "state was set for day %d > T = %d", t0, T);
    if (c->soft && counts) return fail(c, GABM_EINVAL, "counts are not defined for GABM_SOFT (masses, not agents)");
    if (!c->resumed) {
        if (!n_seed) return fail(c, GABM_EINVAL, "n_seed is required when not resuming");
        for (int i = 0; i < c->I; ++i) {
            const int g = i / c->B;
            if (n_seed[i] < 0 || n_seed[i] > c->h_rows[g])
                return fail(c, GABM_EINVAL, "n_seed[%d] = %d outside 0..%d", i, n_seed[i], c->h_rows[g]);
        }
    }
    TRY(ensure_days(c, T));
    if (c->sirs) TRY(ensure_sirs(c, T));
    const int ld = c->Tcap;
    cudaStream_t s = c->stream;
    CK(cudaMemcpy2DAsync(c->R, ld * sizeof(float), R, T * sizeof(float), T * sizeof(float), c->I, h2d_kind(mem_space), s));
    CK(cudaMemcpy2DAsync(c->m, ld * sizeof(float), m, T * sizeof(float), T * sizeof(float), c->I, h2d_kind(mem_space), s));
    CK(cudaMemcpyAsync(c->S, S_age, sizeof(float) * c->I * kAges, h2d_kind(mem_space), s));
    if (!c->resumed) c->last_seeds.assign(n_seed, n_seed + c->I);
    TRY(forward_core(c, t0, T, !c->resumed));
    const bool dev = mem_space == GABM_DEVICE;
    if (c->soft)
        LAUNCH(launch_soft_finalize(c->P_nrm, c->ntiles, c->d_tile0, c->d_ntiles, c->m, ld, T, c->G, c->newRM_real,
                                    c->D, dev ? D : nullptr, s));
    else
        LAUNCH(launch_fwd_finalize(c->newRM, c->counts, c->fate ? nullptr : c->m, ld, t0, T, c->I, c->D, dev ? D : nullptr,
                                   dev ? counts : nullptr, s));
    c->T_last = T;
    c->lam_from = c->policy == GABM_STORE_LAMBDA ? t0 : -1;
    c->bits_from = t0;
    c->last_from_seeding = !c->resumed;
    c->resumed = false;
    c->t0_next = 0;
    if (!dev) {
        if (D) CK(cudaMemcpy2DAsync(D, T * sizeof(double), c->D, ld * sizeof(double), T * sizeof(double), c->I, cudaMemcpyDeviceToHost, s));
        if (counts) CK(cudaMemcpy2DAsync(counts, T * 4 * sizeof(int32_t), c->counts, ld * 4 * sizeof(int32_t), T * 4 * sizeof(int32_t), c->I, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return GABM_OK;
}

gabm_status gabm_mse_loss(gabm_ctx *ctx, const double *y, double *loss, double *gD, int mem_space) {
    gabm_ctx *c = ctx;
    if (!c) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    TRY(check_ms(c, mem_space));
    if (c->T_last < 1) return fail(c, GABM_ESTATE, "no forward has run");
    if (!y) return fail(c, GABM_EINVAL, "y is required");
    const int T = c->T_last, ld = c->Tcap;
    cudaStream_t s = c->stream;
    const double *y_dev = y;
    if (mem_space == GABM_HOST) {
        CK(cudaMemcpyAsync(c->y, y, sizeof(double) * (size_t)c->I * T, cudaMemcpyHostToDevice, s));
        y_dev = c->y;
    }
    const bool dev = mem_space == GABM_DEVICE;
    LAUNCH(launch_mse(c->D, ld, y_dev, T, c->I, dev && loss ? loss : c->loss_s, c->gD, dev ? gD : nullptr, s));
    if (!dev) {
        if (loss) CK(cudaMemcpyAsync(loss, c->loss_s, sizeof(double) * c->I, cudaMemcpyDeviceToHost, s));
        if (gD) CK(cudaMemcpy2DAsync(gD, T * sizeof(double), c->gD, ld * sizeof(double), T * sizeof(double), c->I, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return GABM_OK;
}

static gabm_status backward_impl(gabm_ctx *c, const double *gD, double *dR, double *dm, double *dS_age, double *dc,
                                 int mem_space);

gabm_status gabm_backward(gabm_ctx *ctx, const double *gD, double *dR, double *dm, double *dS_age,
                          int mem_space) {
    return backward_impl(ctx, gD, dR, dm, dS_age, nullptr, mem_space);
}

gabm_status gabm_backward_table(gabm_ctx *ctx, const double *gD, double *dR, double *dm, double *dS_age,
                                double *dc, int mem_space) {
    if (!ctx) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    if (!dc) return fail(ctx, GABM_EINVAL, "dc is required");
    if (ctx->batched && ctx->policy != GABM_STORE_LAMBDA)
        return fail(ctx, GABM_EUNSUPPORTED, "the table adjoint of several sets per graph needs GABM_STORE_LAMBDA in this build");
    if (ctx->fate || ctx->dur.n > 0 || ctx->sirs)
        return fail(ctx, GABM_EUNSUPPORTED, "the table adjoint of the sampled R/M split or stochastic durations is not built");
    return backward_impl(ctx, gD, dR, dm, dS_age, dc, mem_space);
}

// gabm_backward, with the table adjoint accumulated into dc when dc is not NULL.
static gabm_status backward_impl(gabm_ctx *c, const double *gD, double *dR, double *dm, double *dS_age, double *dc,
                                 int mem_space) {
    if (!c) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    TRY(check_ms(c, mem_space));
    if (c->T_last < 1) return fail(c, GABM_ESTATE, "backward needs a forward first");
    if (c->batched && c->bits_from != 0)
        return fail(c, GABM_ESTATE, "several sets per graph: the backward needs a forward over days 0..T-1 "
                    "(its day bitmaps and counts)");
    if (c->policy == GABM_STORE_LAMBDA && c->lam_from != 0)
        return fail(c, GABM_ESTATE, "stored lambdas do not cover days 0..T-1 (use GABM_RECOMPUTE to replay a set state)");
    if (!gD || !dR || !dm || !dS_age) return fail(c, GABM_EINVAL, "gD, dR, dm and dS_age are required");
    const int T = c->T_last, ld = c->Tcap;
    cudaStream_t s = c->stream;
    CK(cudaMemcpy2DAsync(c->gD, ld * sizeof(double), gD, T * sizeof(double), T * sizeof(double), c->I, h2d_kind(mem_space), s));
    c->gD_staged = true;
    // table-adjoint accumulators: [ntiles][kMaxL] (one set per graph) or [ntiles][L][Bp]
    const size_t dc_len = c->batched ? (size_t)c->ntiles * c->L * c->Bp : (size_t)c->ntiles * kMaxL;
    if (dc) {
        if (!c->dc_tile) TRY(dalloc(c, &c->dc_tile, dc_len));
        if (!c->dc_s) TRY(dalloc(c, &c->dc_s, (size_t)c->I * c->L));
        CK(cudaMemsetAsync(c->dc_tile, 0, sizeof(double) * dc_len, s));
    }
    c->want_dc = dc != nullptr;
    const gabm_status bst = backward_core(c, T);
    c->want_dc = false;
    TRY(bst);
    const bool dev = mem_space == GABM_DEVICE;
    if (dc) {
        double *out = dev ? dc : c->dc_s;
        if (c->batched) LAUNCH(launch_dc_reduce_b(c->dc_tile, c->d_tile0, c->d_ntiles, c->G, c->B, c->Bp, c->L, out, s));
        else LAUNCH(launch_dc_reduce(c->dc_tile, c->d_tile0, c->d_ntiles, c->G, c->L, out, s));
    }
    LAUNCH(launch_bwd_finalize(c->Q, c->R, c->S, c->gD,
                               c->fate ? nullptr : (c->batched ? c->newRM : c->newRM_b),
                               c->soft ? c->newRM_real : nullptr, ld, T, c->I,
                               dev ? dR : c->dR_s,
                               dev ? dm : c->dm_s, dev ? dS_age : c->dS_s, s));
    if (c->fate) LAUNCH(launch_fate_dm(c->Pm, c->ntiles, c->d_tile0, c->d_ntiles, c->G, T, dev ? dm : c->dm_s, s));
    if (!dev) {
        CK(cudaMemcpyAsync(dR, c->dR_s, sizeof(double) * (size_t)c->I * T, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(dm, c->dm_s, sizeof(double) * (size_t)c->I * T, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(dS_age, c->dS_s, sizeof(double) * (size_t)c->I * kAges, cudaMemcpyDeviceToHost, s));
        if (dc) CK(cudaMemcpyAsync(dc, c->dc_s, sizeof(double) * (size_t)c->I * c->L, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return GABM_OK;
}

gabm_status gabm_get_state(gabm_ctx *ctx, int16_t *e_out, int mem_space) {
    gabm_ctx *c = ctx;
    if (!c) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    TRY(check_ms(c, mem_space));
    if (!e_out) return fail(c, GABM_EINVAL, "e_out is NULL");
    if (c->soft) return fail(c, GABM_EUNSUPPORTED, "GABM_SOFT has masses, not exposure days");
    const bool dev = mem_space == GABM_DEVICE;
    LAUNCH(launch_rows_to_caller_i16(c->e, dev ? e_out : c->rows_e, graph_ref(c), c->d_rows, c->d_goff, c->n_rows,
                                     set_layout(c), c->stream));
    if (!dev) {
        CK(cudaMemcpyAsync(e_out, c->rows_e, sizeof(int16_t) * (size_t)c->n_total * c->B, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return GABM_OK;
}

gabm_status gabm_set_state(gabm_ctx *ctx, int day, const int16_t *e_in, int mem_space) {
    gabm_ctx *c = ctx;
    if (!c) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    TRY(check_ms(c, mem_space));
    if (!e_in) return fail(c, GABM_EINVAL, "e_in is NULL");
    if (c->soft) return fail(c, GABM_EUNSUPPORTED, "GABM_SOFT has masses, not exposure days");
    if (c->sirs)
        return fail(c, GABM_EUNSUPPORTED, "SIRS reinfection: the last exposure days do not fix the trajectory "
                    "(a set state would need the exposure histories)");
    if (day < 0 || day > GABM_MAX_DAYS) return fail(c, GABM_EINVAL, "day %d outside 0..%d", day, GABM_MAX_DAYS);
    std::vector<int16_t> h((size_t)c->n_total * c->B);
    if (mem_space == GABM_HOST) {
        memcpy(h.data(), e_in, sizeof(int16_t) * h.size());
    } else {
        CK(cudaMemcpyAsync(h.data(), e_in, sizeof(int16_t) * h.size(), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    for (size_t i = 0; i < h.size(); ++i) {
        const int v = h[i];
        if (v != kNever && (v < -c->L || v >= day))
            return fail(c, GABM_EINVAL, "e[%zu] = %d: must be NEVER or in [-%d, %d)", i, v, c->L, day);
    }
    CK(cudaStreamSynchronize(c->stream));
    if (c->n_total > 0) {
        CK(cudaMemcpyAsync(c->rows_e, h.data(), sizeof(int16_t) * h.size(), cudaMemcpyHostToDevice, c->stream));
        LAUNCH(launch_caller_to_rows_i16(c->rows_e, c->e, graph_ref(c), c->d_rows, c->d_goff, c->n_rows, set_layout(c),
                                         c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    c->t0_next = day;
    c->resumed = true;
    c->T_last = -1;
    c->lam_from = -1;
    return GABM_OK;
}

gabm_status gabm_get_lambda(gabm_ctx *ctx, int t, float *lam_out, int mem_space) {
    gabm_ctx *c = ctx;
    if (!c) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    TRY(check_ms(c, mem_space));
    if (!lam_out) return fail(c, GABM_EINVAL, "lam_out is NULL");
    const float *lam_t = nullptr;
    if (c->policy == GABM_STORE_LAMBDA) {
        if (c->T_last < 1 || t < c->lam_from || t >= c->T_last || c->lam_from < 0)
            return fail(c, GABM_ESTATE, "day %d was not run by the last forward", t);
        lam_t = c->lam + (size_t)t * c->n_rows * c->Bp;
    } else {
        // recomputed from the current state, which (no reinfection) fixes every earlier day
        if (c->batched || c->two_hop)
            return fail(c, GABM_EUNSUPPORTED, "lambda on request under GABM_RECOMPUTE is built for one-hop graphs of one set");
        if (c->T_last < 1 || t < 0 || t >= c->T_last)
            return fail(c, GABM_ESTATE, "day %d is not before the last forward's horizon", t);
        if (!c->lam_tmp) TRY(dalloc(c, &c->lam_tmp, (size_t)c->n_rows));
        uint32_t *bits_t = c->bits + (size_t)c->Tcap * c->ntiles;   // the last day slot, free after a forward
        LAUNCH(launch_infectious_bits(c->e, t, 1, c->L, c->ntiles, bits_t, (size_t)c->ntiles, c->stream));
        LAUNCH(launch_lam_day(sell_view(c, false), c->e, bits_t, graph_ref(c), t, c->L, c->ntiles, c->c_dev,
                              c->lam_tmp, c->grid_bwd, c->stream));
        lam_t = c->lam_tmp;
    }
    LAUNCH(launch_get_lambda(lam_t, c->e, c->age, graph_ref(c), c->R, c->S, c->Tcap, t,
                             c->n_rows, c->B, c->Bp, c->rows_f, c->stream));
    const bool dev = mem_space == GABM_DEVICE;
    LAUNCH(launch_rows_to_caller_f32(c->rows_f, dev ? lam_out : c->stage_f, graph_ref(c), c->d_rows, c->d_goff,
                                     c->n_rows, set_layout(c), c->stream));
    if (!dev) {
        CK(cudaMemcpyAsync(lam_out, c->stage_f, sizeof(float) * (size_t)c->n_total * c->B, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return GABM_OK;
}

gabm_status gabm_get_schedule(const gabm_ctx *ctx, gabm_schedule *out) {
    if (!ctx) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    if (!out) return GABM_EINVAL;
    out->fwd_sets_per_lane = ctx->batched ? ctx->spl_fwd : 0;
    out->bwd_sets_per_lane = ctx->batched ? ctx->spl_bwd : 0;
    out->bwd_sets_per_launch = ctx->batched ? ctx->bwd_chunk : 0;
    out->fwd_smem_bitmap = ctx->batched ? 0 : (ctx->smem_bits ? 1 : 0);
    return GABM_OK;
}

gabm_status gabm_set_infectiousness(gabm_ctx *ctx, const float *c_in) {
    gabm_ctx *c = ctx;
    if (!c) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    if (!c_in) return fail(c, GABM_EINVAL, "c is NULL");
    if (c_in[0] != 0.0f) return fail(c, GABM_EINVAL, "c[0] must be 0 (no onward infection on the day of exposure)");
    for (int k = 0; k < c->L; ++k)
        if (!std::isfinite(c_in[k]) || c_in[k] < 0.0f) return fail(c, GABM_EINVAL, "c[%d] must be finite and >= 0", k);
    CK(cudaStreamSynchronize(c->stream));   // launches in flight still read the old table
    for (int k = 0; k < c->L; ++k) c->c[k] = c_in[k];
    CK(cudaMemcpy(c->c_dev, c->c, sizeof(float) * kMaxL, cudaMemcpyHostToDevice));
    for (auto &g : c->loop_graph) drop_graph(g);   // captured launches carry the table by value
    c->T_last = -1;                                // the last trajectory used the old table
    return GABM_OK;
}

gabm_status gabm_set_schedule(gabm_ctx *ctx, const gabm_schedule *sched) {
    gabm_ctx *c = ctx;
    if (!c) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    if (!sched) return fail(c, GABM_EINVAL, "schedule is NULL");
    if (c->batched) {
        const int chunk = sched->bwd_sets_per_launch > 0 ? sched->bwd_sets_per_launch : c->Bp;
        if (!batch_config_ok(c->Bp, sched->fwd_sets_per_lane))
            return fail(c, GABM_EINVAL, "forward sets per lane must be 2, 4 or 8 and at most %d", c->Bp);
        if (chunk > c->Bp || c->Bp % chunk != 0 || !batch_config_ok(chunk, sched->bwd_sets_per_lane))
            return fail(c, GABM_EINVAL, "backward: sets per launch must be a power of two dividing %d, sets per lane "
                        "2, 4 or 8 and at most that", c->Bp);
        c->spl_fwd = sched->fwd_sets_per_lane;
        c->spl_bwd = sched->bwd_sets_per_lane;
        c->bwd_chunk = chunk;
    } else {
        if (sched->fwd_smem_bitmap && (c->soft || c->two_hop || c->fate || c->dur.n > 0 || c->sirs ||
                                       occupancy_fwd(c->ntiles, true) <= 0))
            return fail(c, GABM_EINVAL, "the infectious bitmap (%d words) does not fit in shared memory", c->ntiles);
        c->smem_bits = sched->fwd_smem_bitmap != 0;
    }
    apply_schedule(c);
    return GABM_OK;
}

gabm_status gabm_autotune(gabm_ctx *ctx, int repetitions) {
    gabm_ctx *c = ctx;
    if (!c) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    if (repetitions < 1) return fail(c, GABM_EINVAL, "repetitions must be >= 1");
    if (c->T_last < 1 || !c->last_from_seeding)
        return fail(c, GABM_ESTATE, "autotune needs a preceding forward that started from seeding");
    const int T = c->T_last, ld = c->Tcap;
    cudaStream_t s = c->stream;
    if (!c->gD_staged) CK(cudaMemsetAsync(c->gD, 0, sizeof(double) * (size_t)c->I * ld, s));
    gabm_schedule cur{};
    TRY(gabm_get_schedule(c, &cur));
    // forward schedules (the backward schedule does not change the forward) ...
    std::vector<gabm_schedule> fc, bc;
    if (c->batched) {
        for (int spl : {2, 4, 8})
            if (batch_config_ok(c->Bp, spl)) fc.push_back(gabm_schedule{spl, cur.bwd_sets_per_lane, 0, cur.bwd_sets_per_launch});
    } else {
        fc.push_back(gabm_schedule{0, 0, 0, 0});
        if (!c->soft && !c->two_hop && !c->fate && c->dur.n == 0 && !c->sirs && occupancy_fwd(c->ntiles, true) > 0)
            fc.push_back(gabm_schedule{0, 0, 1, 0});
    }
    cudaEvent_t ev[2];
    for (auto &e : ev) CK(cudaEventCreate(&e));
    auto release = [&]() { for (auto &e : ev) cudaEventDestroy(e); };
    // mean time of `reps` runs of fn after one untimed run (which also captures the CUDA graph)
    auto timed = [&](auto fn, float &ms) -> gabm_status {
        gabm_status st = fn();
        ms = 0.f;
        for (int r = 0; r < repetitions && st == GABM_OK; ++r) {
            cudaEventRecord(ev[0], s);
            st = fn();
            cudaEventRecord(ev[1], s);
            if (cudaEventSynchronize(ev[1]) != cudaSuccess)
                return fail(c, GABM_ECUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
            float a = 0.f;
            cudaEventElapsedTime(&a, ev[0], ev[1]);
            ms += a;
        }
        return st;
    };
    float best_f = 1e30f, best_b = 1e30f;
    gabm_schedule bf = fc[0];
    for (const gabm_schedule &cand : fc) {
        float ms = 0.f;
        gabm_status st = gabm_set_schedule(c, &cand);
        if (st == GABM_OK) st = timed([&]() { return forward_core(c, 0, T, true); }, ms);
        if (st != GABM_OK) { release(); return st; }
        if (ms < best_f) { best_f = ms; bf = cand; }
    }
    // ... then backward schedules after one forward with the best forward schedule
    if (c->batched) {
        for (int spl : {2, 4, 8})
            for (int chunk = c->Bp; chunk >= 2 && chunk >= c->Bp / 4; chunk /= 2)
                if (batch_config_ok(chunk, spl))
                    bc.push_back(gabm_schedule{bf.fwd_sets_per_lane, spl, 0, chunk});
    } else {
        bc.push_back(bf);
    }
    gabm_schedule bb = bc[0];
    {
        gabm_status st = gabm_set_schedule(c, &bf);
        if (st == GABM_OK) st = forward_core(c, 0, T, true);
        if (st != GABM_OK) { release(); return st; }
    }
    for (const gabm_schedule &cand : bc) {
        float ms = 0.f;
        gabm_status st = gabm_set_schedule(c, &cand);
        if (st == GABM_OK) st = timed([&]() { return backward_core(c, T); }, ms);
        if (st != GABM_OK) { release(); return st; }
        if (ms < best_b) { best_b = ms; bb = cand; }
    }
    release();
    const gabm_schedule chosen{bf.fwd_sets_per_lane, bb.bwd_sets_per_lane, bf.fwd_smem_bitmap, bb.bwd_sets_per_launch};
    TRY(gabm_set_schedule(c, &chosen));
    // the last forward's outputs again (the trajectory does not depend on the schedule)
    TRY(forward_core(c, 0, T, true));
    if (c->soft)
        LAUNCH(launch_soft_finalize(c->P_nrm, c->ntiles, c->d_tile0, c->d_ntiles, c->m, ld, T, c->G, c->newRM_real,
                                    c->D, nullptr, s));
    else
        LAUNCH(launch_fwd_finalize(c->newRM, c->counts, c->fate ? nullptr : c->m, ld, 0, T, c->I, c->D, nullptr, nullptr, s));
    CK(cudaStreamSynchronize(s));
    return GABM_OK;
}

gabm_status gabm_mem_stats(const gabm_ctx *ctx, size_t *current, size_t *peak) {
    if (!ctx) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    if (current) *current = ctx->mem_cur;
    if (peak) *peak = ctx->mem_peak;
    return GABM_OK;
}

uint64_t gabm_launch_count(const gabm_ctx *ctx) { return ctx ? ctx->launches : 0; }

gabm_status gabm_set_profiling(gabm_ctx *ctx, int enable) {
    gabm_ctx *c = ctx;
    if (!c) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    TRY(prof_collect(c));
    c->profiling = enable != 0;
    for (int k = 0; k < 2; ++k) { c->prof_ms[k] = 0; c->prof_n[k] = 0; }
    return GABM_OK;
}

gabm_status gabm_get_profile(gabm_ctx *ctx, int kind, double *total_ms, int64_t *launches) {
    gabm_ctx *c = ctx;
    if (!c) return fail(nullptr, GABM_EINVAL, "ctx is NULL");
    if (kind < 0 || kind > 1) return fail(c, GABM_EINVAL, "kind must be 0 or 1");
    TRY(prof_collect(c));
    if (total_ms) *total_ms = c->prof_ms[kind];
    if (launches) *launches = c->prof_n[kind];
    return GABM_OK;
}

gabm_status gabm_philox(uint64_t seed, const uint32_t *ctr, uint32_t *out, int64_t count, void *cuda_stream) {
    gabm_ctx *c = nullptr;
    if (count < 0 || (count > 0 && (!ctr || !out))) return fail(nullptr, GABM_EINVAL, "bad arguments");
    if (count == 0) return GABM_OK;
    CK(launch_philox(seed, ctr, out, count, (cudaStream_t)cuda_stream));
    return GABM_OK;
}

}  // extern "C"
