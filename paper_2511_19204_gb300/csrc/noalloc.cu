// Allocation-free variant of the FP64 knot average (mppi_average_noalloc).
//
// Some callers cannot call cudaMalloc at the point where they need the average: a
// real-time control loop that must not block on the allocator (cudaMalloc/cudaFree can
// synchronise the device), code that runs with a fixed, pre-reserved memory footprint,
// or a host whose allocator is owned by another framework. This entry point takes the
// caller's device inputs and output and keeps its scratch (the per-chunk FP64 partial
// sums) in a file-scope device array of fixed size instead of allocating it.
#include <cuda_runtime.h>

#include <mutex>

#include "capi_internal.h"

namespace mppi {

// Scratch for the per-chunk partial sums: ceil(K / 64) * E doubles at most.
constexpr size_t NOALLOC_SCRATCH_DOUBLES = (size_t)1 << 20;  // 8 MiB on every device that loads the library

static __device__ __align__(256) double g_avg_scratch[NOALLOC_SCRATCH_DOUBLES];

namespace {
std::mutex g_mu;
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
}  // namespace

// Device address of the scratch array on the current device. In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device (with
// that device current) and cached.
static cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_avg_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace mppi

using namespace mppi;

extern "C" mppi_status mppi_average_noalloc(int32_t K, int32_t E, const float* d_knots, const double* d_w,
                                            double* d_out, void* stream) {
    if (K < 1 || E < 1 || !d_knots || !d_w || !d_out) {
        set_error(nullptr, "mppi_average_noalloc: K and E must be positive and the pointers non-null");
        return MPPI_ERR_INVALID_ARG;
    }
    const size_t need = (size_t)num_chunks(K) * (size_t)E;
    if (need > NOALLOC_SCRATCH_DOUBLES) {
        set_error(nullptr,
                  "mppi_average_noalloc: ceil(K / 64) * E exceeds the 1048576-double scratch array; use mppi_average");
        return MPPI_ERR_INVALID_ARG;
    }
    double* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "mppi_average_noalloc: cudaGetSymbolAddress");
    // every scratch element the reduction reads is written first by this call's partial
    // pass, so nothing needs clearing
    cudaStream_t s = (cudaStream_t)stream;
    e = launch_average_partial(d_knots, d_w, K, E, scratch, s);
    if (e == cudaSuccess) e = launch_average_reduce(scratch, num_chunks(K), E, d_out, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "mppi_average_noalloc: launch");
    return MPPI_OK;
}
