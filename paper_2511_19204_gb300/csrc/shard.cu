// Sample-shard entry points (C ABI): one iteration's weights and knot average over
// samples split into shards. Sec. III-C's min-max weights (Eq. softmax_minmax) need the
// global S_min and S_max before any exponential, so a sharded iteration exchanges twice:
// the shards' cost ranges, then their weight and weighted-knot sums. The merges are host
// functions on a few numbers; the exchange between devices is the caller's.
#include <cuda_runtime.h>
#include <math.h>

#include "capi_internal.h"
#include "nvtx.h"

using namespace mppi;

extern "C" {

mppi_status mppi_shard_range_local(int32_t K, const float* d_costs, int64_t index_base, mppi_shard_range* h_out,
                                   void* stream) {
    MPPI_NVTX("mppi_shard_range_local");
    if (K < 1 || index_base < 0 || !d_costs || !h_out) return MPPI_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ShardScan* d = nullptr;
    ShardScan h{};
    cudaError_t e = cudaMalloc(&d, sizeof(ShardScan));
    if (e == cudaSuccess) e = launch_shard_range(d_costs, K, d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(ShardScan), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (d) cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "shard range");
    h_out->n_finite = h.nfinite;
    h_out->s_min = h.nfinite ? (double)h.smin : INFINITY;
    h_out->s_max = h.nfinite ? (double)h.smax : -INFINITY;
    h_out->best_index = h.nfinite ? index_base + h.best : -1;
    return MPPI_OK;
}

void mppi_shard_range_merge(const mppi_shard_range* a, const mppi_shard_range* b, mppi_shard_range* out) {
    if (!a || !b || !out) return;
    mppi_shard_range r;
    r.n_finite = a->n_finite + b->n_finite;
    r.s_max = a->s_max > b->s_max ? a->s_max : b->s_max;
    // the first smallest cost: the lower cost, on a tie the lower global index
    const mppi_shard_range* m;
    if (a->n_finite == 0) m = b;
    else if (b->n_finite == 0) m = a;
    else if (a->s_min < b->s_min || (a->s_min == b->s_min && a->best_index < b->best_index)) m = a;
    else m = b;
    r.s_min = m->n_finite ? m->s_min : INFINITY;
    r.best_index = m->n_finite ? m->best_index : -1;
    if (r.n_finite == 0) r.s_max = -INFINITY;
    *out = r;
}

mppi_status mppi_shard_moments(int32_t K, int32_t E, const float* d_knots, const float* d_costs,
                               const mppi_shard_range* global, double lambda, int32_t normalize, double* h_out,
                               void* stream) {
    MPPI_NVTX("mppi_shard_moments");
    if (K < 1 || E < 1 || !d_knots || !d_costs || !global || !h_out || !(lambda > 0.0) ||
        (normalize != MPPI_NORM_MINMAX && normalize != MPPI_NORM_RAW))
        return MPPI_ERR_INVALID_ARG;
    if (global->n_finite <= 0) {
        set_error(nullptr, "shard moments: no finite cost in any shard");
        return MPPI_ERR_ALL_COSTS_NONFINITE;
    }
    // the merged S_min is one of the FP32 costs: exact as a float
    const float smin = (float)global->s_min;
    if ((double)smin != global->s_min || !(global->s_max >= global->s_min)) {
        set_error(nullptr, "shard moments: the range is not one of FP32 costs");
        return MPPI_ERR_INVALID_ARG;
    }
    // the weight scale as in the single-instance scan: one division in FP64
    const double range = global->s_max - global->s_min;
    const double k = normalize == MPPI_NORM_MINMAX ? (range > 0.0 ? 1.0 / (range * lambda) : 0.0) : 1.0 / lambda;
    cudaStream_t s = (cudaStream_t)stream;
    const int nch = num_chunks(K);
    double *d_w = nullptr, *d_p = nullptr, *d_o = nullptr;
    cudaError_t e = cudaMalloc(&d_w, sizeof(double) * K);
    if (e == cudaSuccess) e = cudaMalloc(&d_p, sizeof(double) * (size_t)nch * E);
    if (e == cudaSuccess) e = cudaMalloc(&d_o, sizeof(double) * ((size_t)E + 1));
    if (e == cudaSuccess) e = launch_shard_weights(d_costs, K, smin, k, d_w, d_o, s);
    if (e == cudaSuccess) e = launch_average_partial(d_knots, d_w, K, E, d_p, s);
    if (e == cudaSuccess) e = launch_average_reduce(d_p, nch, E, d_o + 1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d_o, sizeof(double) * ((size_t)E + 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (d_w) cudaFree(d_w);
    if (d_p) cudaFree(d_p);
    if (d_o) cudaFree(d_o);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "shard moments");
    return MPPI_OK;
}

void mppi_shard_moments_merge(int32_t E, const double* a, const double* b, double* out) {
    if (E < 1 || !a || !b || !out) return;
    for (int32_t i = 0; i <= E; ++i) out[i] = a[i] + b[i];
}

mppi_status mppi_shard_mean(int32_t E, const double* sums, float* h_mean) {
    if (E < 1 || !sums || !h_mean || !(sums[0] > 0.0) || !isfinite(sums[0])) return MPPI_ERR_INVALID_ARG;
    const double z = sums[0];
    for (int32_t e = 0; e < E; ++e) h_mean[e] = (float)(sums[1 + e] / z);
    return MPPI_OK;
}

}  // extern "C"
