// jxf_nvtx.cuh -- NVTX ranges around the C entry points, so that a timeline
// profiler shows each library call (step, state copies, right-hand side,
// reverse mode, block phases, batch steps) as a named range.  NVTX v3 is
// header-only and costs a branch per call when no profiler is attached.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace jxf {

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace jxf

#define JXF_RANGE(name) ::jxf::NvtxRange jxf_nvtx_range_(name)
