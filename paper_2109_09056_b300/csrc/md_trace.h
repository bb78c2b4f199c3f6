// md_trace.h -- NVTX ranges around the C ABI's entry points (host side).
//
// NVTX v3 is header-only: with no tool attached a range costs a load and a
// branch.  Each range is named after its entry point, so a profiler can select
// the kernels of one kind of call, e.g.
//   ncu --nvtx --nvtx-include "md_step/" ...
// captures only kernels launched inside md_step.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace mdb {
class TraceRange {
public:
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
}  // namespace mdb

#define MD_TRACE(name) const ::mdb::TraceRange md_trace_range_(name)
