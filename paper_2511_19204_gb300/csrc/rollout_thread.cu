// Thread-per-sample rollout for specialised robot trees (filled in below when a tree
// shape has a specialisation).
#include "internal.h"

namespace mppi {
bool thread_mapping_supported(int topology) { (void)topology; return false; }
cudaError_t launch_rollout_thread_f32(const RolloutArgs<float>& a, int topology, int block, cudaStream_t s) {
    (void)a; (void)topology; (void)block; (void)s;
    return cudaErrorNotSupported;
}
cudaError_t prepare_thread_f32() { return cudaSuccess; }
}  // namespace mppi
