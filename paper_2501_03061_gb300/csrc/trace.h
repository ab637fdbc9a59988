// NVTX ranges around the C entry points and the phases of a PT-IM step, for profilers that read
// them (ncu --nvtx, Nsight Systems).  NVTX 3 is header-only and costs a no-op call when no tool
// is attached; where its headers are absent the ranges compile to nothing.
#pragma once

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define PT_HAVE_NVTX 1
#endif
#endif

namespace pt {

inline void trace_push(const char* name) {
#ifdef PT_HAVE_NVTX
  nvtxRangePushA(name);
#else
  (void)name;
#endif
}

inline void trace_pop() {
#ifdef PT_HAVE_NVTX
  nvtxRangePop();
#endif
}

struct TraceRange {
  explicit TraceRange(const char* name) { trace_push(name); }
  ~TraceRange() { trace_pop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace pt
