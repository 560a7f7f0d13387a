// Tracing: one named NVTX range per C-ABI call, around the call's host-side validation and
// launches, so that timeline tools (Nsight Systems, ncu --nvtx) attribute the kernels each
// call enqueues.  NVTX v3 is header-only: without an attached tool a range costs one check.
#pragma once
#include <nvtx3/nvToolsExt.h>

struct EpicRange {
    explicit EpicRange(const char* name) { nvtxRangePushA(name); }
    ~EpicRange() { nvtxRangePop(); }
    EpicRange(const EpicRange&) = delete;
    EpicRange& operator=(const EpicRange&) = delete;
};
