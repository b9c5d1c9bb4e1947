// Device side of the sample-shard entry points: one iteration's weights (Sec. III-C,
// Eq. softmax_minmax) and knot average (Eq. update-nominal) over samples split into
// shards. Before the first exchange a shard scans its costs with the weights kernels' own
// scan; before the second it forms its unnormalised weights under the merged range and
// their sums. The knot sums reuse the FP64 average kernels of mppi_average.
#pragma once
#include "internal.h"
#include "reduce.cuh"

namespace mppi {

constexpr int SHARD_THREADS = 1024;

__global__ void __launch_bounds__(SHARD_THREADS) shard_range_kernel(const float* __restrict__ costs, int K,
                                                                    ShardScan* __restrict__ out) {
    // lambda and the normalisation only set MinMax::k, which this scan does not report
    const MinMax mm = block_minmax(costs, K, 1.0, MPPI_NORM_RAW);
    if (threadIdx.x == 0) {
        out->smin = mm.smin;
        out->smax = mm.smax;
        out->best = mm.best;
        out->nfinite = mm.nfinite;
    }
}

// w_n = exp(-(S_n - S_min) k) under the merged range, 0 for a non-finite cost
__global__ void shard_weights_kernel(const float* __restrict__ costs, int K, float smin, double k,
                                     double* __restrict__ w) {
    const MinMax mm{smin, smin, -1, 1, k};
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < K; n += gridDim.x * blockDim.x)
        w[n] = unnorm_weight(costs[n], mm);
}

// sum_n w_n in a fixed order: thread t sums n = t, t + 1024, ..., then a balanced tree
__global__ void __launch_bounds__(SHARD_THREADS) shard_wsum_kernel(const double* __restrict__ w, int K,
                                                                   double* __restrict__ out) {
    __shared__ double s[SHARD_THREADS];
    const int t = threadIdx.x;
    double acc = 0.0;
    for (int n = t; n < K; n += SHARD_THREADS) acc += w[n];
    s[t] = acc;
    __syncthreads();
    for (int h = SHARD_THREADS / 2; h > 0; h >>= 1) {
        if (t < h) s[t] += s[t + h];
        __syncthreads();
    }
    if (t == 0) *out = s[0];
}

cudaError_t launch_shard_range(const float* costs, int K, ShardScan* out, cudaStream_t s) {
    shard_range_kernel<<<1, SHARD_THREADS, 0, s>>>(costs, K, out);
    return cudaGetLastError();
}

cudaError_t launch_shard_weights(const float* costs, int K, float smin, double k, double* w, double* wsum,
                                 cudaStream_t s) {
    int grid = (K + 255) / 256;   // grid-stride beyond 1024 blocks
    if (grid > 1024) grid = 1024;
    shard_weights_kernel<<<grid, 256, 0, s>>>(costs, K, smin, k, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    shard_wsum_kernel<<<1, SHARD_THREADS, 0, s>>>(w, K, wsum);
    return cudaGetLastError();
}

}  // namespace mppi
