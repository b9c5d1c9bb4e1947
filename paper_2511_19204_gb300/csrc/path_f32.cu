// Every FP32 kernel of the path in one translation unit: the per-iteration kernels, the
// rollout kernels of every mapping and the persistent batched kernel call the same
// non-inlined device functions (noise, rollouts, chunk weights, finalize), so a batched
// instance and a single solve run identical machine code and produce identical bits.
#include "internal.h"
#include "rollout_warp.cuh"
#include "iter_kernels.cuh"
#include "chain_kernel.cuh"
#include "batch_impl.cuh"
#include "shard_kernels.cuh"

namespace mppi {
cudaError_t launch_rollout_warp_f32(const RolloutArgs<float>& a, int G, int block, cudaStream_t s) {
    if (G == 32) return launch_rollout_warp_t<float, 32>(a, block, s);
    if (G == 16) return launch_rollout_warp_t<float, 16>(a, block, s);
    return cudaErrorInvalidValue;
}
cudaError_t launch_dynamics_f32(const DevModel<float>* m, int n, const double* x, const double* tau, double* acc,
                                cudaStream_t s) {
    return launch_dynamics_t<float>(m, n, x, tau, acc, s);
}
cudaError_t launch_predict_f32(const DevModel<float>* m, const double* x0, const float* knots, int H, int nsteps,
                               int nk, float dt, float dtk, double* out, uint32_t* status, cudaStream_t s) {
    return launch_predict_t<float>(m, x0, knots, H, nsteps, nk, dt, dtk, out, status, s);
}
cudaError_t prepare_warp_f32() { return prepare_warp_kernels<float>(); }
}  // namespace mppi

// The check word of this translation unit, which holds every FP32 kernel of the path
// (check builds only; see MPPI_CHECK_OK in common.cuh).
extern "C" mppi_status mppi_check_word(uint32_t* h_word, int32_t reset) {
    if (!h_word) return MPPI_ERR_INVALID_ARG;
    *h_word = 0;
#ifdef MPPI_CHECK
    cudaError_t e = cudaMemcpyFromSymbol(h_word, mppi::g_check_word, sizeof(uint32_t));
    if (e == cudaSuccess && reset) {
        const uint32_t zero = 0;
        e = cudaMemcpyToSymbol(mppi::g_check_word, &zero, sizeof(uint32_t));
    }
    return e == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
#else
    (void)reset;
    return MPPI_ERR_UNSUPPORTED;
#endif
}
