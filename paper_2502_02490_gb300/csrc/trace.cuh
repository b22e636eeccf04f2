// NVTX ranges around the C-ABI entry points, so that a timeline or kernel profiler (nsys, ncu
// --nvtx) shows which library call launched which kernels.  NVTX v3 is header-only; with no
// tool attached a push/pop costs a null check.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace qxd {
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
}  // namespace qxd

#define QXD_TRACE() qxd::TraceRange qxd_trace_range_(__func__)
