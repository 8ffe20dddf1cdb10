// twohop.cu -- the location hop of agent-location graphs (GradABM-JUNE, Sec. 5).
//
// Agents interact through shared locations: with attendance weights w_il the pair
// weight is W_ij = sum_l w_il w_jl, and each sum over W is computed in two hops over
// the attendance entries.  This file holds the location half: one value per
// location, a pull over the location's members in a SELL-32 layout of locations
// (32 locations per warp tile, every lane its own location, members in entry
// order).  The agent half is the ordinary day kernel gathering these values over
// the agent's locations (forward.cu with a pull array, backward.cu with the
// location adjoint in place of r).
//   forward:  P_l(t)  = sum_{j at l} w_jl x_j(t), x_j(t) = c[t - e_j] for members
//             marked infectious in the day's bitmap (Sec. 3.1, Eq. 3);
//   backward: gP_l    = sum_{i at l} w_il r_i(t+1), so that the agent gather gives
//             gx_j = sum_l w_jl gP_l = sum_i W_ji r_i (App. B, the transpose of the
//             forward's two hops).
#include "gabm_internal.cuh"
#include "rowsum.cuh"

namespace gabm {

namespace {

template <bool FWD>
__global__ void __launch_bounds__(kBlock) k_loc_sum(Sell ml, int nloc_tiles, const int16_t *e,
                                                    const uint32_t *bits, const float *r, int t, int L,
                                                    const float *c, float *out) {
    __shared__ float c_s[kMaxL];
    if (threadIdx.x < kMaxL) c_s[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    auto contrib = [&](uint32_t j, float w, bool valid, float (&o)[1]) {
        if constexpr (FWD) {
            const bool mk = valid && marked(bits, j);
            const int ej = ld_if(e + j, mk, kNever);
            o[0] = mk ? w * infectiousness(ej, c_s, t, L) : 0.f;
        } else {
            o[0] = w * ld_if(r + j, valid);
        }
    };
    const bool want[1] = {true};
    BlockTiles disp;
    disp.init(nloc_tiles, lane);
    for (int tile = disp.get(); tile < nloc_tiles; tile = disp.get()) {
        const int row = tile * kTile + lane;
        const uint32_t len = ml.row_len[row];
        float sum[1];
        row_sums<1>(ml, ml.slice_ptr[tile], len, len > 0, lane, contrib, want, sum);
        out[row] = sum[0];
    }
}

}  // namespace

cudaError_t launch_loc_pressure(Sell ml, int nloc_tiles, const int16_t *e, const uint32_t *bits, int t, int L,
                                const float *c, float *P, int grid, cudaStream_t s) {
    k_loc_sum<true><<<grid, kBlock, 0, s>>>(ml, nloc_tiles, e, bits, nullptr, t, L, c, P);
    return cudaGetLastError();
}

cudaError_t launch_loc_adjoint(Sell ml, int nloc_tiles, const float *r, const float *c, float *gP, int grid,
                               cudaStream_t s) {
    k_loc_sum<false><<<grid, kBlock, 0, s>>>(ml, nloc_tiles, nullptr, nullptr, r, 0, 0, c, gP);
    return cudaGetLastError();
}

int occupancy_loc() {
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_loc_sum<true>, kBlock, 0);
    return blocks > 0 ? blocks : 1;
}

}  // namespace gabm
