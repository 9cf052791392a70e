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
  int step_kernel = 2;  // 2: two-step kernel, one tile per block, where possible;
                        // 3: persistent two-step kernel with a copy ring;
                        // 4: two-step kernel, one tile per block, v^{n+1} over v^n;
                        // 1: single-step only
  int max_items = 0;    // cap on items in flight (0 = memory budget)
  int graph = 0;        // 1: capture each phase of a batch in a CUDA graph
  int tile_z = 24;      // centre rows of a two-step tile (16 with kernel 3, 32 with kernel 4)
  int l2_ahead = 0;     // step_kernel 2: each block prefetches a later block's tile into L2
  int image_input = 0;  // two-step backward launches image their input field where they can
  int pdl = 0;          // step_kernel 4: programmatic dependent launches (griddepcontrol)
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
  // Device wait-timeout flags: one pinned slot per call in flight.  A call
  // copies its kernels' flag into its own slot; a call that synchronises reads
  // it, an asynchronous one leaves it pending with an event, and the next
  // call on the context reads it once the event has completed.
  struct PendingFlag {
    int slot;
    cudaEvent_t ev;
  };
  int *h_flags = nullptr;           // pinned [kFlagSlots][2]: {code, source line}
  std::vector<int> free_flags;      // guarded by flag_mu
  std::deque<PendingFlag> pending;  // guarded by flag_mu
  int seen_code = 0, seen_line = 0;  // first raised flag among reaped pending ones (flag_mu)
  std::mutex flag_mu;
  std::atomic<int> inject_timeouts{0};  // test hook: calls that start with the flag raised
  rtm_stats stats{};        // guarded by mu
  rtm_server *server = nullptr;
  // streams on which calls given the legacy default stream run (guarded by
  // stream_mu): the legacy stream cannot be captured into graphs
  std::vector<cudaStream_t> free_streams;
  std::mutex stream_mu;
};

namespace rtm {

constexpr int kFlagSlots = 256;

int fail(rtm_ctx *ctx, int code, const char *fmt, ...);
// The message of the last fail() on the calling thread (request threads read
// their own error text here, not the context's, which other threads share).
const char *thread_error();

// Device flag slots (see rtm_ctx).  A call's kernels raise its flag with
// code 1 when a bounded wait gives up, and (debug builds) code 2 with the
// source line when an index check fails.  Acquire a zeroed slot; copy the
// call's two flag words into h_flags + 2 slot; after a synchronised call,
// read and release it (flag_take: the code, 0 if none); or leave it pending
// behind an event recorded on st.
int flag_acquire(rtm_ctx *ctx);
int flag_take(rtm_ctx *ctx, int slot, int *line);
void flag_defer(rtm_ctx *ctx, int slot, cudaStream_t st);
// The status a raised flag reports: RTM_ERR_TIMEOUT (a wait gave up) or
// RTM_ERR_STATE (a debug index check failed); `whose` names the call.
int flag_status(rtm_ctx *ctx, int code, int line, const char *whose);
// An error status if a pending flag of an earlier call came back raised.
int check_wait_flag(rtm_ctx *ctx);

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

Geo make_geo(const rtm_grid &gr, int tile_z = 24);
// Host tables of the propagation kernels: the sponge factors per memory column
// (zero outside the padded domain) and per row (Cerjan profile, §3 reading);
// the receivers of each single-step tile as CSR {row * TX + col in the tile,
// receiver index}.
void sponge_tables(const Geo &g, std::vector<float> &gx, std::vector<float> &gz);
void receiver_tiles(const Geo &g, const rtm_acq &acq, std::vector<int> &rptr,
                    std::vector<int2> &rent);
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
// The kernels' wait-timeout flag is copied into flag slot `flag_slot` (if
// >= 0) once the work is enqueued.
int migrate_device(rtm_ctx *ctx, const rtm_grid &gr, int nsample, const float *vel_d,
                   const rtm_acq &acq, const float *seis_d, const rtm_opts &op, float *img_d,
                   int B, cudaStream_t st, const RunConfig &cfg,
                   const float *born_refl = nullptr, float *born_out = nullptr,
                   LateCopy *late = nullptr, int flag_slot = -1);
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
// Cancels queued requests and waits (bounded) for running ones; false if some
// are still running after the bound (the server then stays attached).
bool rtm_server_shutdown(rtm_ctx *ctx);
// Most requests running at once and requests admitted past a waiting head,
// since the server started (or the last reset).
void rtm_server_counters(rtm_ctx *ctx, bool reset, long long *peak_running,
                         long long *backfilled);
