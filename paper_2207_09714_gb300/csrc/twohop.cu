// twohop.cu -- the location hop of agent-location graphs (GradABM-JUNE, Sec. 6).
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
    auto contrib = [&](uint32_t j, float w, bool valid, float (&o)[1], bool (&take)[1]) {
        if constexpr (FWD) {
            const bool mk = valid && marked(bits, j);
            const int ej = ld_if(e + j, mk, kNever);
            o[0] = mk ? w * infectiousness(ej, c_s, t, L) : 0.f;
            take[0] = mk;
        } else {
            o[0] = w * ld_if(r + j, valid);
            take[0] = valid;
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

// Large locations (more than 32 members): one warp per location, the lanes taking
// every 32nd member in turn (four loads in flight), each lane summing with
// compensation, then a fixed shuffle tree: deterministic, and a school of hundreds
// takes a few steps instead of hundreds of steps of one lane.
template <bool FWD>
__global__ void __launch_bounds__(kBlock) k_loc_big(LocCsr big, const int16_t *e, const uint32_t *bits,
                                                    const float *r, int t, int L, const float *c, float *out) {
    __shared__ float c_s[kMaxL];
    if (threadIdx.x < kMaxL) c_s[threadIdx.x] = c[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (kBlock / 32);
    auto term = [&](uint32_t p, bool ok) {
        const uint32_t j = ld_if(big.col + p, ok);
        const float w = ld_if(big.w + p, ok);
        if constexpr (FWD) {
            const bool mk = ok && marked(bits, j);
            const int ej = ld_if(e + j, mk, kNever);
            return mk ? w * infectiousness(ej, c_s, t, L) : 0.f;
        } else {
            return w * ld_if(r + j, ok);
        }
    };
    for (int b = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5); b < big.n; b += nwarps) {
        const uint32_t p0 = big.rowptr[b], p1 = big.rowptr[b + 1];
        float s = 0.f, comp = 0.f;
        for (uint32_t p = p0 + (uint32_t)lane; p < p1; p += 128u) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = term(p + 32u * (uint32_t)u, p + 32u * (uint32_t)u < p1);
#pragma unroll
            for (int u = 0; u < 4; ++u) kahan_add(s, comp, v[u]);
        }
        s -= comp;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[big.base + b] = s;
    }
}

}  // namespace

cudaError_t launch_loc_pressure(Sell ml, int nloc_tiles, LocCsr big, const int16_t *e, const uint32_t *bits, int t,
                                int L, const float *c, float *P, int grid, cudaStream_t s) {
    if (nloc_tiles > 0) k_loc_sum<true><<<grid, kBlock, 0, s>>>(ml, nloc_tiles, e, bits, nullptr, t, L, c, P);
    if (big.n > 0) k_loc_big<true><<<grid, kBlock, 0, s>>>(big, e, bits, nullptr, t, L, c, P);
    return cudaGetLastError();
}

cudaError_t launch_loc_adjoint(Sell ml, int nloc_tiles, LocCsr big, const float *r, const float *c, float *gP,
                               int grid, cudaStream_t s) {
    if (nloc_tiles > 0) k_loc_sum<false><<<grid, kBlock, 0, s>>>(ml, nloc_tiles, nullptr, nullptr, r, 0, 0, c, gP);
    if (big.n > 0) k_loc_big<false><<<grid, kBlock, 0, s>>>(big, nullptr, nullptr, r, 0, 0, c, gP);
    return cudaGetLastError();
}

int occupancy_loc() {
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_loc_sum<true>, kBlock, 0);
    return blocks > 0 ? blocks : 1;
}

}  // namespace gabm
