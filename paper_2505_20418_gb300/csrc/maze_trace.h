// NVTX ranges around the public entry points: a profiler attached to the
// process (ncu --nvtx, for instance, to filter a capture to the kernels of
// one call) sees each call as a named range. NVTX v3 is header-only and inert
// unless a tool injects its library, so the ranges cost a few host
// instructions otherwise. Ranges mark the host-side call: the kernels a call
// enqueues (graph replays included) fall inside it when the call waits for
// them, as maze_step does.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace maze {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace maze
