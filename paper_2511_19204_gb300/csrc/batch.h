// Host interface of the persistent batched kernel (batch.cu), shared with the server.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "capi_internal.h"

namespace mppi {

constexpr int BATCH_THREADS = 256;

// Byte layout of one batched launch (see batch.cu).
struct BatchLayout {
    int count = 0, max_E = 0;
    long total = 0, nprefill = 0;
    size_t in_bytes = 0, out_bytes = 0;
    size_t o_q = 0, o_insts = 0, o_pre = 0, o_in = 0, image_bytes = 0;
    size_t o_ctr = 0, o_items = 0, o_out = 0, dev_bytes = 0;
};

int batch_tile(int mapping);
size_t batch_smem_bytes(int max_E);
BatchLayout layout_batch(mppi_ctx* const* ctxs, int count);
void fill_batch_image(mppi_ctx* const* ctxs, const BatchLayout& L, const double* const* states,
                      const float* const* warm, unsigned char* img, std::vector<size_t>* in_off,
                      std::vector<size_t>* out_off);
cudaError_t prepare_batch_kernel(int max_E, size_t* smem, int* per_sm);
cudaError_t enqueue_batch(const BatchLayout& L, const unsigned char* h_img, unsigned char* d_block,
                          unsigned char* h_out, int grid, size_t smem, cudaStream_t s);
mppi_status unpack_batch(mppi_ctx* const* ctxs, const BatchLayout& L, const std::vector<size_t>& out_off,
                         const unsigned char* h_out, float* const* out_mean, float* const* out_best,
                         mppi_result* info);
// Validation shared by mppi_solve_batch and mppi_submit.
mppi_status check_batchable(const mppi_ctx* c, int device);

}  // namespace mppi
