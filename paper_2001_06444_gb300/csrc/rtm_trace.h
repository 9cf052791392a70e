// rtm_trace.h — phase markers of the library's calls (internal).
//
// Each migration call opens an NVTX range named after the call, and its
// phases (set-up, forward and backward time loops, stacking) open nested
// ranges, so a profiler can select them (ncu --nvtx --nvtx-include ...).
// With RTM_TRACE=1 in the environment the calls also print, to stderr, the
// host time since the call began at each phase boundary: where a call's host
// time goes when the device waits on it.
#pragma once
#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>

namespace rtm {

inline bool trace_enabled() {
  static const bool on = [] {
    const char *e = std::getenv("RTM_TRACE");
    return e && e[0] == '1';
  }();
  return on;
}

// The call being traced on this thread (nested calls keep the outer one).
struct CallTrace {
  const char *name;
  std::chrono::steady_clock::time_point t0;
  CallTrace *outer;
  static CallTrace *&current() {
    static thread_local CallTrace *cur = nullptr;
    return cur;
  }
  explicit CallTrace(const char *n) : name(n), t0(std::chrono::steady_clock::now()) {
    outer = current();
    current() = this;
    nvtxRangePushA(n);
  }
  ~CallTrace() {
    mark("end");
    nvtxRangePop();
    current() = outer;
  }
  CallTrace(const CallTrace &) = delete;
  CallTrace &operator=(const CallTrace &) = delete;
  void mark(const char *what) const {
    if (!trace_enabled()) return;
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    std::fprintf(stderr, "rtm-trace %s +%.3f ms %s\n", name, ms, what);
  }
};

// Mark a phase boundary of the current call (no-op outside a traced call).
inline void trace_mark(const char *what) {
  if (CallTrace *t = CallTrace::current()) t->mark(what);
}

// A nested NVTX range for one phase of a call.
struct PhaseRange {
  explicit PhaseRange(const char *n) { nvtxRangePushA(n); }
  ~PhaseRange() { nvtxRangePop(); }
  PhaseRange(const PhaseRange &) = delete;
  PhaseRange &operator=(const PhaseRange &) = delete;
};

}  // namespace rtm
