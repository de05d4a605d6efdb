// NVTX ranges around the library's entry points, so that a profiler timeline
// (Nsight Systems, or ncu's --nvtx filters) shows which call issued which
// kernels.  Header-only NVTX v3: when no tool is attached, a push/pop is a
// check of one function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace cdi {

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace cdi
