// Host-side internal interface shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mppi.h"
#include "common.cuh"

namespace mppi {

constexpr int REDUCE_THREADS = 256;   // fixed: the weight reduction order depends on it
constexpr int AVG_CHUNK = 64;         // samples per FP64 partial sum of the knot average
constexpr int AVG_GROUP = 16;         // chunks per group total (the second level of the sum)
constexpr int AVG_THREADS = 128;

// Per-iteration weight information (device), written by the weights step.
struct DevIterInfo {
    double smin, smax, lse, ess;
    int32_t best, nfinite, status, pad;
};

// Per-solve state of a context (device), reset at the start of each solve.
struct DevSolve {
    double best_cost;
    int32_t best_index, best_iter, status, pad;
    uint32_t iter_counter;   // Philox counter word 2 of the solve's first iteration
    uint32_t blocks_done;    // groups of the running weights launch that finished (the last resets it)
    uint32_t dev_error;      // DEV_ERR_* bits from bounded device waits
    uint32_t pad3;
};

struct SampleArgs {
    const float* nominal;    // [E]
    const float* sigma_row;  // [nk]
    const DevModel<float>* model;
    float* knots;            // [N][E]
    const DevSolve* solve;   // iter_counter source (nullable -> iter_counter_override)
    uint32_t iter_offset;    // added to the counter
    uint32_t iter_counter_override;
    uint32_t inst;
    uint32_t seed_lo, seed_hi;
    int N, nk, nj, has_limits;
    float scale_q, scale_v, dtk;
    int spline = 0;          // MPPI_SPLINE_*
};

template <typename T>
struct RolloutArgs {
    const DevModel<T>* model;
    const double* x0;
    const float* knots;   // [N][E]
    T* costs;             // [N]
    double* finals;       // [N][nx] nullable
    uint32_t* status;     // DEV_ERR bits (nullable)
    int N, H, nk;
    T dt, dtk;
};

// launches (kernels.cu / rollout_*.cu)
// pdl: a programmatic dependent of the kernel before it (the previous iteration's finalize)
cudaError_t launch_sample_knots(const SampleArgs& a, cudaStream_t s, bool pdl = false);
cudaError_t launch_rollout_warp_f32(const RolloutArgs<float>& a, int G, int block, cudaStream_t s);
cudaError_t launch_rollout_warp_f64(const RolloutArgs<double>& a, int G, int block, cudaStream_t s);
// pdl: launched as a programmatic dependent of the kernel before it in the stream (the
// knot noise of a solve): its prologue overlaps that kernel; it waits for it before the
// first knot read (griddepcontrol.wait)
cudaError_t launch_rollout_chain_f32(const RolloutArgs<float>& a, int topology, bool paper, int axis_plan, int block,
                                     cudaStream_t s, bool pdl = false);
bool chain_mapping_supported(int topology);
// FP64 check build of the lanes-per-chain kernels (128-thread blocks)
cudaError_t launch_rollout_chain_f64(const RolloutArgs<double>& a, int topology, bool paper, int axis_plan,
                                     cudaStream_t s);
// state after the first nsteps steps of knots [nk][2][nj] from x0 (one warp, Sec. III-E)
cudaError_t launch_predict_f32(const DevModel<float>* m, const double* x0, const float* knots, int H, int nsteps,
                               int nk, float dt, float dtk, double* out, uint32_t* status, cudaStream_t s);
cudaError_t launch_predict_f64(const DevModel<double>* m, const double* x0, const float* knots, int H, int nsteps,
                               int nk, double dt, double dtk, double* out, uint32_t* status, cudaStream_t s);
// in-place shift of knots [nk][2][nj] by `steps` control steps, tail held (Sec. III-E)
cudaError_t launch_shift_knots(float* knots, int nj, int nk, int H, int steps, double dtk, cudaStream_t s);
cudaError_t prepare_warp_f32();
cudaError_t prepare_warp_f64();
// weights of each chunk of AVG_CHUNK samples and their partial knot sums (reduce.cuh)
cudaError_t launch_weights_average(const float* costs, const float* knots, int N, int E, double lambda, int normalize,
                                   double* e_out, double* zq, double* partial, DevIterInfo* info, cudaStream_t s);
// w = e / z and the iteration's lse / ESS (standalone weights entry point)
cudaError_t launch_normalize_weights(const double* e, const double* zq, int N, double* w, DevIterInfo* info,
                                     cudaStream_t s);
// weighted average with given weights: chunk partials, then chunk totals
cudaError_t launch_average_partial(const float* knots, const double* w, int N, int E, double* partial,
                                   cudaStream_t s);
cudaError_t launch_average_reduce(const double* partial, int nchunks, int E, double* out, cudaStream_t s);
struct FinalizeArgs {
    double* partial;    // [nchunks][E] chunk partial sums
    double* zq;         // [nchunks][2] chunk (z_c, q_c)
    double* gpartial;   // [ngroups][E] group totals
    double* gzq;        // [ngroups][2]
    uint32_t* gcount;   // [ngroups] chunks of the group finished (zero between iterations)
    int nchunks, ngroups, E, iter, iters, warm_from;
    const float* knots;
    const float* costs;
    DevIterInfo* info;
    DevSolve* solve;
    float* nominal;     // next iteration's nominal (and the resident warm start at the end)
    float* mean_out;    // [E]
    float* best_out;    // [E]
    mppi_result* result;
};
// chunk weights + partial sums, the group totals by the last chunk of each group and the
// finalize by the last group to finish (one launch per iteration)
cudaError_t launch_weights_finalize(const FinalizeArgs& a, int N, double lambda, int normalize, cudaStream_t s,
                                    bool pdl = false);
cudaError_t prepare_weights_kernels();   // co-residency of the cooperative finish, per device
cudaError_t launch_solve_begin(DevSolve* solve, uint32_t* gcount, int ngroups, const float* nominal, float* best_out,
                               int E, cudaStream_t s);
// sample shards (shard_kernels.cuh): one shard's cost range, and its unnormalised weights
// w [K] and their sum under a merged range (S_min, weight scale k)
struct ShardScan {
    float smin, smax;
    int best, nfinite;
};
cudaError_t launch_shard_range(const float* costs, int K, ShardScan* out, cudaStream_t s);
cudaError_t launch_shard_weights(const float* costs, int K, float smin, double k, double* w, double* wsum,
                                 cudaStream_t s);
cudaError_t launch_fast_math(int n, const float* x, const float* y, float* out, cudaStream_t s);
cudaError_t launch_widen(int n, const float* x, double* out, cudaStream_t s);
cudaError_t launch_philox_words(int n, const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, cudaStream_t s);
cudaError_t launch_dynamics_f32(const DevModel<float>* m, int n, const double* x, const double* tau, double* acc,
                                cudaStream_t s);
cudaError_t launch_dynamics_f64(const DevModel<double>* m, int n, const double* x, const double* tau, double* acc,
                                cudaStream_t s);

__host__ __device__ inline int num_chunks(int N) { return (N + AVG_CHUNK - 1) / AVG_CHUNK; }
__host__ __device__ inline int num_groups(int N) { return (num_chunks(N) + AVG_GROUP - 1) / AVG_GROUP; }

}  // namespace mppi
