// rtm_engine.h — the native runtime behind the C ABI (internal).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <cstdarg>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/rtm.h"
#include "rtm_common.h"

struct rtm_server;

namespace rtm {
// How a migration is launched (all choices give bit-identical results).
struct RunConfig {
  int step_kernel = 2;  // 2: two-step TMA kernel where possible; 1: single-step only
  int max_items = 0;    // cap on items in flight (0 = memory budget)
  int graph = 0;        // 1: capture each phase of a batch in a CUDA graph
};
// Shape key of the autotuner cache.
struct TuneKey {
  int nx, nz, nb, nt, isnap, dtype;
  bool operator<(const TuneKey &o) const {
    const int a[6] = {nx, nz, nb, nt, isnap, dtype}, b[6] = {o.nx, o.nz, o.nb, o.nt, o.isnap, o.dtype};
    for (int i = 0; i < 6; ++i)
      if (a[i] != b[i]) return a[i] < b[i];
    return false;
  }
};
}  // namespace rtm

struct rtm_ctx {
  int device = 0;
  size_t budget = 0;        // bytes of device memory the context may hold
  size_t used = 0;          // bytes currently reserved by running work
  cudaMemPool_t pool = nullptr;
  std::mutex mu;            // guards `used` and the error text
  std::condition_variable mem_cv;
  char err[512] = "no error";
  int max_batch = 0;        // 0 = no cap beyond memory
  bool prof = false;        // time the step-kernel phases with events
  rtm::RunConfig defaults;  // launch configuration when no tuned entry matches
  std::map<rtm::TuneKey, rtm::RunConfig> tuned;  // autotuner results (guarded by mu)
  int *h_err = nullptr;     // pinned: device wait-timeout flag of the last call
  rtm_stats stats{};        // guarded by mu
  rtm_server *server = nullptr;
};

namespace rtm {

int fail(rtm_ctx *ctx, int code, const char *fmt, ...);

// Device allocation from the context pool, stream-ordered.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  cudaError_t alloc(rtm_ctx *ctx, size_t n, cudaStream_t s);
  void release();
  template <class T>
  T *as() const {
    return reinterpret_cast<T *>(p);
  }
};

bool is_device_ptr(const void *p);

Geo make_geo(const rtm_grid &gr);
int checkpoint_steps(const rtm_opts &op, const rtm_grid &gr, const Geo &g);
Coef make_coef(const rtm_grid &gr);

struct MigrationPlan {
  Geo g;
  int nsnap = 0;
  size_t item_bytes = 0;    // per in-flight item
  size_t shared_bytes = 0;  // per call
};
MigrationPlan plan_migration(const rtm_grid &gr, const rtm_acq &acq, const rtm_opts &op,
                             int nsample);

int check_grid(rtm_ctx *ctx, const rtm_grid *g);
int check_acq(rtm_ctx *ctx, const rtm_grid *g, const rtm_acq *a, bool need_rec);
int check_opts(rtm_ctx *ctx, const rtm_opts *o);

// Host seismograms whose copy to the device is issued late, on its own
// stream: they are first read by the backward phase, so their upload runs
// behind the first forward phase.  The copy goes in per-batch pieces in shot
// order, each followed by an event, so a batch's backward phase waits only
// for the shots it reads.  `alloc_done` is recorded on the main stream once
// `dst` is allocated.
struct LateCopy {
  const void *src = nullptr;
  void *dst = nullptr;
  size_t shot_bytes = 0;  // one shot's seismogram [nt][nrec]
  cudaStream_t cs = nullptr;
  cudaEvent_t alloc_done = nullptr;
  std::vector<cudaEvent_t> ready;  // one per batch, once issued
  bool issued = false;
};

// Migration of nsample models x all shots with device pointers and a fixed
// batch size B (items in flight).  Memory is allocated from the pool.
// With born_refl set, Born modelling instead: the backward phase is replaced
// by the perturbation field driven by c m S^k, recorded into born_out
// [nitems][nt][nrec]; seis_d and img_d are not used.  With `late` set, the
// copy of the seismograms into seis_d is issued after the first forward
// phase is enqueued, and the main stream waits for it before any backward
// step.
int migrate_device(rtm_ctx *ctx, const rtm_grid &gr, int nsample, const float *vel_d,
                   const rtm_acq &acq, const float *seis_d, const rtm_opts &op, float *img_d,
                   int B, cudaStream_t st, const RunConfig &cfg,
                   const float *born_refl = nullptr, float *born_out = nullptr,
                   LateCopy *late = nullptr);
RunConfig config_for(rtm_ctx *ctx, const rtm_grid &gr, const rtm_opts &op);

// Velocity range check (CFL of §3, positivity, finiteness); synchronises st.
int check_velocity(rtm_ctx *ctx, const rtm_grid &gr, const float *vel_d, long long n,
                   cudaStream_t st);

size_t reserve_wait(rtm_ctx *ctx, size_t want, size_t min_need, int timeout_ms);
void unreserve(rtm_ctx *ctx, size_t bytes);

}  // namespace rtm

// request loop (rtm_server.cu)
int rtm_server_submit(rtm_ctx *ctx, const rtm_request *req, uint64_t *ticket);
int rtm_server_poll(rtm_ctx *ctx, uint64_t ticket, int *state, int timeout_ms);
void rtm_server_shutdown(rtm_ctx *ctx);
