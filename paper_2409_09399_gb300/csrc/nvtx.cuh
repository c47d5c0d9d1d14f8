// nvtx.cuh -- NVTX ranges around the library's entry points, so that a timeline
// profiler (nsys) or ncu --nvtx shows each call by name.  NVTX v3 is header-only:
// without an attached tool a range costs one check of a function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace gint {

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace gint
