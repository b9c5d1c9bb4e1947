// Allocation-free variant of the FP64 knot average (mppi_average_noalloc).
//
// Some callers cannot call cudaMalloc at the point where they need the average: a
// real-time control loop that must not block on the allocator (cudaMalloc/cudaFree can
// synchronise the device), code that runs with a fixed, pre-reserved memory footprint,
// or a host whose allocator is owned by another framework. This entry point takes the
// caller's device inputs and output and keeps its scratch (the per-chunk FP64 partial
// sums) in a file-scope device array of fixed size instead of allocating it.
#include <cuda.h>
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
// The scratch address is only valid in the context it was looked up in: a device reset
// (cudaDeviceReset, or another framework releasing and recreating the primary context)
// gives the device a new context whose copy of the array may sit elsewhere. So the cache
// is keyed on the context's process-unique id (cuCtxGetId), not on the device number.
struct ScratchEntry {
    unsigned long long ctx_id = 0;
    bool valid = false;
    double* addr = nullptr;
};
ScratchEntry g_scratch[kMaxDevices];
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_ctx_get_id_looked_up = false;

// Id of the context current on this thread; false when there is none yet or the driver
// cannot tell.
bool current_context_id(unsigned long long* id) {
    if (!g_ctx_get_id_looked_up) {
        g_ctx_get_id_looked_up = true;
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(fn);
    }
    return g_ctx_get_id && g_ctx_get_id(nullptr, id) == CUDA_SUCCESS;
}
}  // namespace

// Device address of the scratch array in the current device's context. In host code the
// array's name is only a host-side stand-in, so the address is looked up with the device
// current (cudaGetSymbolAddress) once per context and cached; a new context on the device
// (after a reset) is detected by its id and looked up again.
static cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    ScratchEntry& c = g_scratch[dev];
    if (!have_id || !c.valid || c.ctx_id != id) {
        double* p = nullptr;
        // also makes the runtime's context current when no context was current yet
        e = cudaGetSymbolAddress((void**)&p, g_avg_scratch);
        if (e != cudaSuccess) return e;
        if (!have_id) have_id = current_context_id(&id);
        c.addr = p;
        c.ctx_id = id;
        c.valid = have_id;  // without a context id every call looks the address up again
    }
    *out = c.addr;
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
