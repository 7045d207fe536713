// nvtx_range.h -- scoped NVTX ranges around the library's entry points, so profilers show
// which call a kernel belongs to. NVTX3 is header-only and inert unless a tool is attached.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace isg {
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace isg
