// Entry points whose implementation follows (batched persistent solve, serving,
// autotuning).
#include "capi_internal.h"

extern "C" {
mppi_status mppi_server_create(int32_t, size_t, int32_t, mppi_server** out) { if (out) *out = nullptr; return MPPI_ERR_UNSUPPORTED; }
void mppi_server_destroy(mppi_server*) {}
mppi_status mppi_submit(mppi_server*, mppi_ctx*, const double*, const float*, uint64_t*) { return MPPI_ERR_UNSUPPORTED; }
mppi_status mppi_poll(mppi_server*, uint64_t, float*, float*, mppi_result*, int64_t) { return MPPI_ERR_UNSUPPORTED; }
mppi_status mppi_server_stats(mppi_server*, int64_t*) { return MPPI_ERR_UNSUPPORTED; }
}
