// FP64 check-build instantiations of the warp-per-sample rollout and dynamics kernels
// (same source as the FP32 product, double arithmetic: separates algorithmic
// differences from FP32 rounding when compared with the FP64 oracle).
#include "internal.h"
#include "rollout_warp.cuh"

namespace mppi {
cudaError_t launch_rollout_warp_f64(const RolloutArgs<double>& a, int G, int block, cudaStream_t s) {
    if (G == 32) return launch_rollout_warp_t<double, 32>(a, block, s);
    if (G == 16) return launch_rollout_warp_t<double, 16>(a, block, s);
    return cudaErrorInvalidValue;
}
cudaError_t launch_dynamics_f64(const DevModel<double>* m, int n, const double* x, const double* tau, double* acc,
                                cudaStream_t s) {
    return launch_dynamics_t<double>(m, n, x, tau, acc, s);
}
cudaError_t launch_predict_f64(const DevModel<double>* m, const double* x0, const float* knots, int H, int nsteps,
                               int nk, double dt, double dtk, double* out, uint32_t* status, cudaStream_t s) {
    return launch_predict_t<double>(m, x0, knots, H, nsteps, nk, dt, dtk, out, status, s);
}
cudaError_t prepare_warp_f64() { return prepare_warp_kernels<double>(); }
}  // namespace mppi
