// trace.h -- NVTX ranges around the host library's entry points, so that a
// profiler's timeline shows which call enqueued which kernels and copies.
// NVTX is header-only here: without a tool attached each range costs one
// check of a function pointer.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace xe {

struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace xe

#define CORR_TRACE_CAT2(a, b) a##b
#define CORR_TRACE_CAT(a, b) CORR_TRACE_CAT2(a, b)
// One range from here to the end of the enclosing scope.
#define CORR_TRACE(name) ::xe::TraceRange CORR_TRACE_CAT(corr_trace_, __LINE__)(name)
