// Host interface of the persistent batched kernels (batch_impl.cuh), shared with the server.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "capi_internal.h"

namespace mppi {

constexpr int BATCH_THREADS = 256;
static_assert(BATCH_THREADS >= 160, "the finalize holds up to 8 elements per thread of B - 32");
constexpr int BATCH_VARIANTS = 10;  // rollout variants, one persistent kernel each

// The instances of one rollout variant (mapping, axis plan, modular cost), which walk
// their own queue in their own persistent kernel: item counts, estimated work (tiles x
// tile cost) and the byte offsets of the group's queue header, prefill list and items.
struct BatchGroup {
    int variant = 0;
    long total = 0, nprefill = 0;
    double work = 0.0;
    size_t o_q = 0, o_pre = 0, o_items = 0;
};

// Byte layout of one batched launch (see batch_impl.cuh).
struct BatchLayout {
    int count = 0, max_E = 0;
    long total = 0, nprefill = 0;
    size_t in_bytes = 0, out_bytes = 0;
    size_t o_groups = 0, o_q = 0, o_insts = 0, o_pre = 0, o_in = 0, image_bytes = 0;
    size_t o_ctr = 0, o_items = 0, o_out = 0, dev_bytes = 0;
    std::vector<BatchGroup> groups;
};

// Auxiliary streams and events on which the groups' persistent kernels fork from the
// launching stream and join back to it (created on first use, kept by their owner).
struct BatchStreams {
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaError_t ensure(int n);
    void release();
};

int batch_tile(int mapping);
// Bounds of layout_batch(...).dev_bytes: batch_fixed_bound() + the sum of
// batch_instance_bound() over the batch's contexts.
size_t batch_fixed_bound();
size_t batch_instance_bound(const mppi_ctx* c);
size_t batch_smem_bytes(int max_E);
BatchLayout layout_batch(mppi_ctx* const* ctxs, int count);
void fill_batch_image(mppi_ctx* const* ctxs, const BatchLayout& L, const double* const* states,
                      const float* const* warm, unsigned char* img, std::vector<size_t>* in_off,
                      std::vector<size_t>* out_off);
cudaError_t prepare_batch_kernel(int max_E, size_t* smem, int* per_sm);
cudaError_t enqueue_batch(const BatchLayout& L, const unsigned char* h_img, unsigned char* d_block,
                          unsigned char* h_out, int grid, size_t smem, cudaStream_t s, BatchStreams& bs);
mppi_status unpack_batch(mppi_ctx* const* ctxs, const BatchLayout& L, const std::vector<size_t>& out_off,
                         const unsigned char* h_out, float* const* out_mean, float* const* out_best,
                         mppi_result* info);
// Validation shared by mppi_solve_batch and mppi_submit.
mppi_status check_batchable(const mppi_ctx* c, int device);

}  // namespace mppi
