// Lanes-per-chain rollout kernels (see rollout_lanes.cuh and rollout_split.cuh).
#pragma once
#include "chain_f32.cuh"

namespace mppi {

template <int LMAX, bool BRANCH, bool PAPER, int AXP>
__global__ void __launch_bounds__(256) rollout_lanes_kernel(RolloutArgs<float> a) {
    __shared__ __align__(16) DevModel<float> Ms;
    __shared__ uint64_t mbar;
    if (!bulk_load_to_smem(&Ms, a.model, (uint32_t)sizeof(DevModel<float>), &mbar)) {
        if (threadIdx.x == 0 && a.status) atomicOr(a.status, DEV_ERR_TMA_TIMEOUT);
        return;
    }
    const int g = threadIdx.x % LANES;
    const int n = (blockIdx.x * blockDim.x + threadIdx.x) / LANES;
    const bool active = n < a.N;
    const int ne = active ? n : a.N - 1;
    const int nj = Ms.nb - 1;
    const int E = a.nk * 2 * nj;
    const int nx = 13 + 2 * nj;
    double* xf = (active && a.finals) ? a.finals + (size_t)n * nx : nullptr;
    const float c = lanes_rollout<LMAX, BRANCH, PAPER, AXP>(Ms, g, a.x0, a.knots + (size_t)ne * E, a.H, a.nk, a.dt, a.dtk, xf);
    if (active && g == 0) a.costs[n] = c;
}

// The two-warp split (humanoid layout): 64-thread warp pairs, 16 samples each, so the
// same 4 threads per sample as the one-warp kernel; pair p of the block uses named
// barrier 1 + p and its own exchange area.
template <bool PAPER>
__global__ void __launch_bounds__(256) rollout_split_kernel(RolloutArgs<float> a) {
    __shared__ __align__(16) DevModel<float> Ms;
    __shared__ uint64_t mbar;
    __shared__ __align__(16) float xch[4 * SPLIT_PAIR_FLOATS];
    if (!bulk_load_to_smem(&Ms, a.model, (uint32_t)sizeof(DevModel<float>), &mbar)) {
        if (threadIdx.x == 0 && a.status) atomicOr(a.status, DEV_ERR_TMA_TIMEOUT);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int pair = warp >> 1;
    if (!MPPI_CHECK_OK(pair < 4, CHECK_SPLIT)) pair = 3;   // xch holds 4 pairs (launches allow <= 256 threads)
    const int n = blockIdx.x * (blockDim.x / LANES) + pair * SPLIT_SPP + (lane >> 1);
    const bool active = n < a.N;
    const int ne = active ? n : a.N - 1;
    const int nj = Ms.nb - 1;
    const int E = a.nk * 2 * nj;
    const int nx = 13 + 2 * nj;
    double* xf = (active && a.finals) ? a.finals + (size_t)n * nx : nullptr;
    const float c = split_rollout<PAPER>(Ms, warp & 1, lane, xch + pair * SPLIT_PAIR_FLOATS, 1 + pair, a.x0,
                                         a.knots + (size_t)ne * E, a.H, a.nk, a.dt, a.dtk, xf);
    if (active && (warp & 1) == 0 && (lane & 1) == 0) a.costs[n] = c;
}

bool chain_mapping_supported(int topology) { return topology == TOPO_QUADRUPED || topology == TOPO_HUMANOID; }

// a plain launch, or with programmatic stream serialisation (see launch_rollout_chain_f32)
static cudaError_t chain_launch(void (*kernel)(RolloutArgs<float>), int grid, int block, cudaStream_t s, bool pdl,
                                const RolloutArgs<float>& a) {
    if (!pdl) {
        kernel<<<grid, block, 0, s>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

cudaError_t launch_rollout_chain_f32(const RolloutArgs<float>& a, int topology, bool paper, int axis_plan, int block,
                                     cudaStream_t s, bool pdl) {
    if (!chain_mapping_supported(topology)) return cudaErrorNotSupported;
    if (block <= 0) block = 128;
    if (block % 32 != 0 || block > 256) return cudaErrorInvalidValue;
    const int spb = block / LANES;
    const int grid = (a.N + spb - 1) / spb;
    if (grid == 0) return cudaSuccess;
    void (*k)(RolloutArgs<float>);
    if (topology == TOPO_QUADRUPED) {
        const bool xyy = axis_plan == AXP_XYY;
        if (paper) k = xyy ? rollout_lanes_kernel<3, false, true, AXP_XYY> : rollout_lanes_kernel<3, false, true, AXP_GENERIC>;
        else k = xyy ? rollout_lanes_kernel<3, false, false, AXP_XYY> : rollout_lanes_kernel<3, false, false, AXP_GENERIC>;
    } else if (axis_plan == AXP_HUM) {
        if (block % 64 != 0) return cudaErrorInvalidValue;
        k = paper ? rollout_split_kernel<true> : rollout_split_kernel<false>;
        // launched early, the split kernel's 32 whole-SM blocks take the SMs the noise
        // kernel frees first; the instruction-fetch-bound launch ran 30 us longer that way
        pdl = false;
    } else {
        k = paper ? rollout_lanes_kernel<6, true, true, AXP_GENERIC> : rollout_lanes_kernel<6, true, false, AXP_GENERIC>;
    }
    return chain_launch(k, grid, block, s, pdl, a);
}

}  // namespace mppi
