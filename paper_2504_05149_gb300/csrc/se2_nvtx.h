// NVTX ranges around the C-ABI calls: each public entry point shows up by
// name on a profiler's timeline (nothing happens without a profiler).
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace se2 {
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace se2
#define SE2_RANGE(name) ::se2::NvtxRange se2_nvtx_range_(name)
