// labs_nvtx.h -- an NVTX range around each working entry point of the C ABI, so that
// a profiler's timeline shows the library's calls (labs_walk, labs_neighbor_delta, ...)
// around the kernels they launch.  NVTX v3 is header-only: without a tool attached a
// range costs one check of an unset function pointer.  Host code only.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace labsgpu {

struct ApiRange {
    explicit ApiRange(const char* name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
    ApiRange(const ApiRange&) = delete;
    ApiRange& operator=(const ApiRange&) = delete;
};

}  // namespace labsgpu

// Opens a range named after the enclosing function for the rest of its body.
#define LABS_API_RANGE() ::labsgpu::ApiRange labs_api_range_(__func__)
