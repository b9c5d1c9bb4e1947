// Definitions of the opaque C-ABI handles and host helpers shared by capi.cu,
// batch.cu, autotune.cu and server.cpp.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "internal.h"

struct mppi_model {
    int device = 0;
    int nb = 0, nj = 0, nc = 0;
    bool fixed_base = false;
    int topology = 0;
    mppi::DevModel<float> host_f;
    mppi::DevModel<double> host_d;
    void* d_f = nullptr;   // device DevModel<float>
    void* d_d = nullptr;   // device DevModel<double>
    std::vector<float> q_init;
};

struct mppi_ctx {
    const mppi_model* model = nullptr;
    uint64_t uid = 0;                            // unique per context for the life of the process
    int device = 0;
    int N = 0, H = 0, nk = 0, iters = 0, nj = 0, E = 0, nx = 0;
    double lambda = 0, dt = 0, dtk = 0, scale_q = 1, scale_v = 0;
    int normalize = 0, warm_from = 0, spline = 0;
    uint64_t seed = 0;
    uint32_t instance_id = 0;
    int mapping = 0, block = 0;
    bool auto_mapping = false;
    bool fp64_check = false;
    bool has_state = false;                      // a solve has uploaded a state
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph_exec = nullptr;
    bool profile = false;                        // event nodes around each rollout launch
    std::vector<cudaEvent_t> ev;                 // 2 per iteration when profiling
    // device buffers (one allocation)
    void* dev_block = nullptr;
    size_t dev_bytes = 0;
    double* d_x0 = nullptr;
    float* d_knots = nullptr;
    float* d_costs = nullptr;
    double* d_w = nullptr;
    double* d_partial = nullptr;
    double* d_zq = nullptr;                      // [nchunks][2] per-chunk sum e, sum e^2
    double* d_gpartial = nullptr;                // [ngroups][E] group totals of the partials
    double* d_gzq = nullptr;                     // [ngroups][2]
    uint32_t* d_gcount = nullptr;                // [ngroups] finished chunks per group
    float* d_nominal = nullptr;
    float* d_mean = nullptr;
    float* d_best = nullptr;
    float* d_sigma = nullptr;
    mppi::DevIterInfo* d_info = nullptr;
    mppi::DevSolve* d_solve = nullptr;
    mppi_result* d_result = nullptr;
    // pinned host staging
    void* host_block = nullptr;
    double* h_x0 = nullptr;
    float* h_mean = nullptr;
    float* h_best = nullptr;
    float* h_warm = nullptr;
    mppi_result* h_result = nullptr;
    std::string last_error;
};

namespace mppi {
void set_error(mppi_ctx* ctx, const std::string& msg);
mppi_status cuda_fail(mppi_ctx* ctx, cudaError_t e, const char* what);
size_t ctx_layout(mppi_ctx* c, bool assign);
// after_noise: the kernel before it in the stream is the solve's knot noise (the rollout
// may then start as its programmatic dependent)
cudaError_t enqueue_rollout(mppi_ctx* c, const double* d_x0, const float* d_knots, int N, float* d_costs,
                            double* d_finals, cudaStream_t s, bool after_noise = false);
cudaError_t enqueue_iteration(mppi_ctx* c, int it, cudaStream_t s);
cudaError_t enqueue_solve_kernels(mppi_ctx* c, cudaStream_t s);
mppi_status launch_solve(mppi_ctx* c);
void invalidate_graph(mppi_ctx* c);
int default_mapping(const mppi_model* m, int N);
int default_block(int mapping);
bool mapping_valid(const mppi_model* m, int mapping, int block);
cudaError_t prepare_kernels();
}  // namespace mppi
