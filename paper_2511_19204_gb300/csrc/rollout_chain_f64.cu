// FP64 check build of the lanes-per-chain rollout kernels: the same bodies as the FP32
// product (rollout_lanes.cuh, rollout_split.cuh) instantiated in double precision with the
// library's correctly rounded elementary functions, in namespace mppi::f64. The product's
// own specialisations (axis plans, hoisted leaf projections, power-basis setpoints, the
// base integrated by the arm warp) are thereby checked against the FP64 oracle at FP64
// tolerances, separating algorithmic differences from FP32 rounding (Alg. 1 "simulate",
// Eq. hermite_segment). Not on the product path: mppi_rollout_explicit runs it when a
// context's FP64 check is on and its mapping is lanes-per-chain.
#include <type_traits>

#include "internal.h"
#include "rollout_warp.cuh"

#define R_DOUBLE 1
#include "scalar_macros.h"
#include "rollout_lanes.cuh"
#include "rollout_split.cuh"

namespace mppi {

constexpr int F64_CHAIN_THREADS = 128;   // 32 lanes-per-chain samples, or 2 warp pairs of the split

template <int LMAX, bool BRANCH, bool PAPER, int AXP>
__global__ void __launch_bounds__(F64_CHAIN_THREADS) rollout_lanes_f64_kernel(RolloutArgs<double> a) {
    __shared__ __align__(16) DevModel<double> Ms;
    __shared__ uint64_t mbar;
    if (!bulk_load_to_smem(&Ms, a.model, (uint32_t)sizeof(DevModel<double>), &mbar)) {
        if (threadIdx.x == 0 && a.status) atomicOr(a.status, DEV_ERR_TMA_TIMEOUT);
        return;
    }
    const int g = threadIdx.x % f64::LANES;
    const int n = (blockIdx.x * blockDim.x + threadIdx.x) / f64::LANES;
    const bool active = n < a.N;
    const int ne = active ? n : a.N - 1;
    const int nj = Ms.nb - 1;
    const int E = a.nk * 2 * nj;
    const int nx = 13 + 2 * nj;
    double* xf = (active && a.finals) ? a.finals + (size_t)n * nx : nullptr;
    const double c = f64::lanes_rollout<LMAX, BRANCH, PAPER, AXP>(Ms, g, a.x0, a.knots + (size_t)ne * E, a.H, a.nk,
                                                                  a.dt, a.dtk, xf);
    if (active && g == 0) a.costs[n] = c;
}

template <bool PAPER>
__global__ void __launch_bounds__(F64_CHAIN_THREADS) rollout_split_f64_kernel(RolloutArgs<double> a) {
    __shared__ __align__(16) DevModel<double> Ms;
    __shared__ uint64_t mbar;
    __shared__ __align__(16) double xch[(F64_CHAIN_THREADS / 64) * f64::SPLIT_PAIR_FLOATS];
    if (!bulk_load_to_smem(&Ms, a.model, (uint32_t)sizeof(DevModel<double>), &mbar)) {
        if (threadIdx.x == 0 && a.status) atomicOr(a.status, DEV_ERR_TMA_TIMEOUT);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, pair = warp >> 1;
    const int n = blockIdx.x * (blockDim.x / f64::LANES) + pair * f64::SPLIT_SPP + (lane >> 1);
    const bool active = n < a.N;
    const int ne = active ? n : a.N - 1;
    const int nj = Ms.nb - 1;
    const int E = a.nk * 2 * nj;
    const int nx = 13 + 2 * nj;
    double* xf = (active && a.finals) ? a.finals + (size_t)n * nx : nullptr;
    const double c = f64::split_rollout<PAPER>(Ms, warp & 1, lane, xch + pair * f64::SPLIT_PAIR_FLOATS, 1 + pair,
                                               a.x0, a.knots + (size_t)ne * E, a.H, a.nk, a.dt, a.dtk, xf);
    if (active && (warp & 1) == 0 && (lane & 1) == 0) a.costs[n] = c;
}

cudaError_t launch_rollout_chain_f64(const RolloutArgs<double>& a, int topology, bool paper, int axis_plan,
                                     cudaStream_t s) {
    if (!chain_mapping_supported(topology)) return cudaErrorNotSupported;
    const int block = F64_CHAIN_THREADS;
    const int spb = block / f64::LANES;
    const int grid = (a.N + spb - 1) / spb;
    if (grid == 0) return cudaSuccess;
    if (topology == TOPO_QUADRUPED) {
        const bool xyy = axis_plan == AXP_XYY;
        if (paper) {
            if (xyy) rollout_lanes_f64_kernel<3, false, true, AXP_XYY><<<grid, block, 0, s>>>(a);
            else rollout_lanes_f64_kernel<3, false, true, AXP_GENERIC><<<grid, block, 0, s>>>(a);
        } else {
            if (xyy) rollout_lanes_f64_kernel<3, false, false, AXP_XYY><<<grid, block, 0, s>>>(a);
            else rollout_lanes_f64_kernel<3, false, false, AXP_GENERIC><<<grid, block, 0, s>>>(a);
        }
    } else if (axis_plan == AXP_HUM) {
        if (paper) rollout_split_f64_kernel<true><<<grid, block, 0, s>>>(a);
        else rollout_split_f64_kernel<false><<<grid, block, 0, s>>>(a);
    } else {
        if (paper) rollout_lanes_f64_kernel<6, true, true, AXP_GENERIC><<<grid, block, 0, s>>>(a);
        else rollout_lanes_f64_kernel<6, true, false, AXP_GENERIC><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace mppi
