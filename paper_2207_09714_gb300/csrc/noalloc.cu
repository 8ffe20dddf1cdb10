// noalloc.cu -- initial-state construction that never allocates device memory.
//
// Some callers cannot allocate device memory themselves or let a library do
// it: code that runs while a memory pool is being reserved for another
// framework, processes started under a fixed device-memory budget, or hosts
// that hand this library only the buffers it must fill.  For them
// gabm_seed_state_noalloc builds the day-0 state (the same radix selection of
// the seed agents that gabm_forward runs) with its scratch in one fixed array
// of device memory that is part of the library image.
#include <algorithm>
#include <mutex>
#include <string>

#include "gabm_internal.cuh"

namespace {

using namespace gabm;

constexpr int kNoallocMaxInstances = GABM_NOALLOC_MAX_INSTANCES;

// Scratch of gabm_seed_state_noalloc, for up to kNoallocMaxInstances instances:
// selection state, digit histograms, tie lists, and the per-instance row
// offsets the seeding kernels read.  Every loaded copy of the library holds it
// on every device it runs on until the process exits.
struct NoallocScratch {
    SeedState st[kNoallocMaxInstances];
    uint32_t hist[kNoallocMaxInstances][kHistBins];
    uint32_t ties[kNoallocMaxInstances][kTieCap];
    int32_t row0[kNoallocMaxInstances];
    int32_t rows[kNoallocMaxInstances];
    int32_t n_seed[kNoallocMaxInstances];
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
NoallocScratch *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  It is looked up
// afresh on every call made outside a stream capture, so a module reloaded at
// another address (after cudaDeviceReset, say) is followed; a call on a
// capturing stream reuses the address found by the last uncaptured call on
// that device and fails if there was none.
cudaError_t scratch_address(cudaStream_t s, NoallocScratch **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<NoallocScratch *>(p);
    } else if (!g_scratch_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

struct SeedCounts {
    int32_t n_seed[kNoallocMaxInstances];
};

// Per-instance row offsets and seed counts, written from kernel arguments so
// that no host buffer is copied.
__global__ void k_fill_offsets(NoallocScratch *sc, int32_t n, int num_instances, SeedCounts counts) {
    const int i = threadIdx.x;
    if (i < num_instances) {
        sc->row0[i] = n * i;
        sc->rows[i] = n;
        sc->n_seed[i] = counts.n_seed[i];
    }
}

thread_local std::string g_noalloc_error;

gabm_status fail_noalloc(gabm_status st, const std::string &msg) {
    g_noalloc_error = msg;
    return st;
}

}  // namespace

extern "C" {

const char *gabm_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

gabm_status gabm_seed_state_noalloc(uint64_t seed, int64_t n, int num_instances, const int32_t *n_seed,
                                    int tau_EI, int16_t *e_out, void *cuda_stream) {
    g_noalloc_error.clear();
    if (num_instances < 1 || num_instances > kNoallocMaxInstances)
        return fail_noalloc(GABM_EINVAL, "num_instances must be 1.." + std::to_string(kNoallocMaxInstances) +
                                             " (the fixed scratch holds that many)");
    if (n < 1 || n * (int64_t)num_instances >= ((int64_t)1 << 31))
        return fail_noalloc(GABM_EINVAL, "need 1 <= n and n * num_instances < 2^31");
    if (!n_seed || !e_out) return fail_noalloc(GABM_EINVAL, "n_seed and e_out are required");
    if (tau_EI < 1 || tau_EI > GABM_MAX_L) return fail_noalloc(GABM_EINVAL, "tau_EI outside 1..GABM_MAX_L");
    SeedCounts counts;
    for (int i = 0; i < kNoallocMaxInstances; ++i) counts.n_seed[i] = 0;
    for (int i = 0; i < num_instances; ++i) {
        if (n_seed[i] < 0 || n_seed[i] > n) return fail_noalloc(GABM_EINVAL, "n_seed[i] outside 0..n");
        counts.n_seed[i] = n_seed[i];
    }
    NoallocScratch *sc = nullptr;
    cudaError_t e = scratch_address((cudaStream_t)cuda_stream, &sc);
    if (e != cudaSuccess) return fail_noalloc(GABM_ECUDA, std::string("scratch address: ") + cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t ni = (size_t)num_instances;
    // the scratch keeps the previous call's contents: histograms must start at zero
#define NA_CK(call)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return fail_noalloc(GABM_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)
    NA_CK(cudaMemsetAsync(sc->hist, 0, sizeof(uint32_t) * kHistBins * ni, s));
    k_fill_offsets<<<1, kNoallocMaxInstances, 0, s>>>(sc, (int32_t)n, num_instances, counts);
    NA_CK(cudaGetLastError());
    const int64_t n_rows = n * num_instances;
    const int grid = (int)std::min<int64_t>((n_rows + 255) / 256, 65535);
    NA_CK(launch_init_state(e_out, sc->row0, sc->rows, num_instances, n_rows, 1, 1, grid, s));
    SeedArgs sa;
    sa.row0 = sc->row0;
    sa.rows = sc->rows;
    sa.orig_id = nullptr;
    sa.e = e_out;
    sa.B = 1;
    sa.Bp = 1;
    sa.st = sc->st;
    sa.hist = &sc->hist[0][0];
    sa.ties = &sc->ties[0][0];
    sa.seed = seed;
    sa.tau_EI = tau_EI;
    sa.pass = 0;
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 1024));
    NA_CK(launch_seed_reset(sc->st, sc->n_seed, num_instances, s));
    for (int pass = 0; pass < 3; ++pass) {
        sa.pass = pass;
        NA_CK(launch_seed_hist(sa, num_instances, gx, s));
        NA_CK(launch_seed_scan(sa, num_instances, s));
    }
    NA_CK(launch_seed_mark(sa, num_instances, gx, s));
    NA_CK(launch_seed_ties(sa, num_instances, s));
#undef NA_CK
    return GABM_OK;
}

}  // extern "C"
