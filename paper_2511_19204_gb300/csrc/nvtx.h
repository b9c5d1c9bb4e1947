// NVTX ranges (header-only NVTX v3 from the CUDA toolkit) around the library's host entry
// points: a profiler (Nsight Systems, ncu's NVTX filters) shows each solve, batch, server
// launch and kernel-level call as a named range. Without a profiler attached a push / pop
// pair costs a few nanoseconds.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace mppi {
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace mppi

#define MPPI_NVTX_CAT2(a, b) a##b
#define MPPI_NVTX_CAT(a, b) MPPI_NVTX_CAT2(a, b)
#define MPPI_NVTX(name) ::mppi::NvtxRange MPPI_NVTX_CAT(nvtx_range_, __LINE__)(name)
