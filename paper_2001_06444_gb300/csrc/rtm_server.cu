// rtm_server.cu — request loop with continuous batching.
//
// Requests (one velocity model, its shots and data) queue in arrival order.
// A scheduler thread admits the head of the queue as soon as the context's
// memory budget can hold its snapshot buffers (at least one shot in flight,
// up to all of its shots), gives it its own CUDA stream and a launcher thread,
// and moves on: requests that arrive while others run join the device work as
// memory frees up, and their kernels overlap on the GPU.
//
// Backfill: while the head waits for memory, a later request that fits in
// what is free now is admitted past it, up to kMaxOvertake times per head;
// after that the head is admitted before anything else, so nothing starves.
// Every wait is bounded; a request that fails reports FAILED with its own
// error text (a device-side wait that gave up fails its own request only).
//
// The paper runs independent migrations in MPI subgroups, starting the next
// one as soon as a subgroup finishes (§3); this is the single-GPU counterpart.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "rtm_engine.h"

using namespace rtm;
using Clock = std::chrono::steady_clock;

struct rtm_req_state {
  uint64_t id = 0;
  rtm_request r;
  std::vector<int> sx, sz, rx, rz;
  std::vector<float> wav;
  MigrationPlan plan;
  size_t need1 = 0, want = 0, reserved = 0;
  int overtaken = 0;  // later requests admitted while this one headed the queue
  int state = RTM_REQ_QUEUED;
  int rc = RTM_OK;
  std::string err;
};

struct rtm_server {
  std::mutex mu;
  std::condition_variable cv;        // request state changes
  std::deque<std::shared_ptr<rtm_req_state>> queue;
  std::map<uint64_t, std::shared_ptr<rtm_req_state>> all;
  std::thread sched;
  bool stop = false;
  uint64_t next = 1;
  int running = 0;
  int peak_running = 0;  // most requests running at once
  long long backfilled = 0;  // requests admitted past a waiting head
  bool log = false;          // RTM_SERVER_LOG=1: admissions and completions to stderr
  Clock::time_point t0 = Clock::now();
  static constexpr int kMaxQueue = 4096;
  static constexpr int kMaxRunning = 32;
  static constexpr int kMaxOvertake = 16;    // backfill admissions past one waiting head
  static constexpr int kBackfillWindow = 64;  // queued requests looked at behind the head
};

static void run_request(rtm_ctx *ctx, rtm_server *S, std::shared_ptr<rtm_req_state> q, int B) {
  int rc = RTM_OK;
  cudaStream_t st = nullptr;
  std::string err;
  if (cudaSetDevice(ctx->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    rc = RTM_ERR_CUDA;
    err = "could not create a stream for the request";
  }
  // this request's own wait-timeout flag and error text (other request
  // threads share the context's)
  const int slot = rc ? -1 : flag_acquire(ctx);
  if (!rc) rc = check_velocity(ctx, q->r.grid, q->r.vel, (long long)q->r.grid.nx * q->r.grid.nz, st);
  if (!rc)
    rc = migrate_device(ctx, q->r.grid, 1, q->r.vel, q->r.acq, q->r.seis, q->r.opts, q->r.image,
                        B, st, config_for(ctx, q->r.grid, q->r.opts), nullptr, nullptr, nullptr,
                        slot);
  if (rc && err.empty()) err = thread_error();
  if (st) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (!rc && e != cudaSuccess) {
      rc = RTM_ERR_CUDA;
      err = cudaGetErrorString(e);
    }
    cudaStreamDestroy(st);
  }
  int line = 0;
  const int code = flag_take(ctx, slot, &line);
  if (code && !rc) {
    rc = flag_status(ctx, code, line, "this request (its image is incomplete)");
    err = thread_error();
  }
  unreserve(ctx, q->reserved);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    q->rc = rc;
    q->err = err;
    q->state = rc ? RTM_REQ_FAILED : RTM_REQ_DONE;
    S->running--;
    if (S->log)
      std::fprintf(stderr, "rtm-server %.3f done id=%llu rc=%d running=%d\n",
                   std::chrono::duration<double>(Clock::now() - S->t0).count(),
                   (unsigned long long)q->id, rc, S->running);
  }
  S->cv.notify_all();
}

// Start request q with `got` bytes reserved (S->mu held; q already out of
// the queue).
static void admit(rtm_ctx *ctx, rtm_server *S, const std::shared_ptr<rtm_req_state> &q, size_t got) {
  q->reserved = got;
  q->state = RTM_REQ_RUNNING;
  S->running++;
  S->peak_running = std::max(S->peak_running, S->running);
  const long long nitems = q->r.acq.nshot;
  long long B = (long long)((got - q->plan.shared_bytes) / q->plan.item_bytes);
  B = std::max<long long>(1, std::min<long long>(B, nitems));
  if (S->log)
    std::fprintf(stderr,
                 "rtm-server %.3f admit id=%llu grid=%dx%d shots=%d nt=%d B=%lld got=%.2fGB "
                 "want=%.2fGB running=%d queued=%zu\n",
                 std::chrono::duration<double>(Clock::now() - S->t0).count(),
                 (unsigned long long)q->id, q->r.grid.nx, q->r.grid.nz, q->r.acq.nshot,
                 q->r.grid.nt, B, got / 1e9, q->want / 1e9, S->running, S->queue.size());
  std::thread(run_request, ctx, S, q, (int)B).detach();
  S->cv.notify_all();
}

// Remove q from the queue if it is still there (S->mu held).
static bool take_from_queue(rtm_server *S, const std::shared_ptr<rtm_req_state> &q) {
  for (auto it = S->queue.begin(); it != S->queue.end(); ++it)
    if (*it == q) {
      S->queue.erase(it);
      return true;
    }
  return false;
}

static void scheduler(rtm_ctx *ctx, rtm_server *S) {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (!S->stop) {
    if (S->queue.empty() || S->running >= rtm_server::kMaxRunning) {
      S->cv.wait_for(lk, std::chrono::milliseconds(50));
      continue;
    }
    auto q = S->queue.front();
    lk.unlock();
    const size_t got = reserve_wait(ctx, q->want, q->need1, 20);
    lk.lock();
    if (got) {
      if (take_from_queue(S, q))
        admit(ctx, S, q, got);
      else
        unreserve(ctx, got);  // cancelled by a shutdown meanwhile
      continue;
    }
    // the head waits for memory: backfill with a later request that fits in
    // what is free now, a bounded number of times per head
    if (q->overtaken >= rtm_server::kMaxOvertake) continue;
    std::vector<std::shared_ptr<rtm_req_state>> behind;
    for (size_t i = 1; i < S->queue.size() && (int)i <= rtm_server::kBackfillWindow; ++i)
      behind.push_back(S->queue[i]);
    for (auto &c : behind) {
      if (S->stop || S->running >= rtm_server::kMaxRunning) break;
      lk.unlock();
      const size_t g2 = reserve_wait(ctx, c->want, c->need1, 0);
      lk.lock();
      if (!g2) continue;
      if (take_from_queue(S, c)) {
        q->overtaken++;
        S->backfilled++;
        admit(ctx, S, c, g2);
        break;
      }
      unreserve(ctx, g2);
    }
  }
}

static rtm_server *ensure_server(rtm_ctx *ctx) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!ctx->server) {
    ctx->server = new rtm_server();
    const char *lg = std::getenv("RTM_SERVER_LOG");
    ctx->server->log = lg && lg[0] == '1';
    ctx->server->sched = std::thread(scheduler, ctx, ctx->server);
  }
  return ctx->server;
}

int rtm_server_submit(rtm_ctx *ctx, const rtm_request *req, uint64_t *ticket) {
  if (!req || !ticket) return fail(ctx, RTM_ERR_ARG, "request and ticket must not be NULL");
  int rc;
  if ((rc = check_grid(ctx, &req->grid)) || (rc = check_acq(ctx, &req->grid, &req->acq, true)) ||
      (rc = check_opts(ctx, &req->opts)))
    return rc;
  if (!req->vel || !req->seis || !req->image)
    return fail(ctx, RTM_ERR_ARG, "request arrays must not be NULL");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, RTM_ERR_CUDA, "cudaSetDevice");
  if (!is_device_ptr(req->vel) || !is_device_ptr(req->seis) || !is_device_ptr(req->image))
    return fail(ctx, RTM_ERR_ARG, "request arrays must be device memory");
  auto q = std::make_shared<rtm_req_state>();
  q->r = *req;
  const rtm_acq &a = req->acq;
  q->sx.assign(a.src_ix, a.src_ix + a.nshot);
  q->sz.assign(a.src_iz, a.src_iz + a.nshot);
  q->rx.assign(a.rec_ix, a.rec_ix + a.nrec);
  q->rz.assign(a.rec_iz, a.rec_iz + a.nrec);
  q->wav.assign(a.wavelet, a.wavelet + req->grid.nt);
  q->r.acq.src_ix = q->sx.data();
  q->r.acq.src_iz = q->sz.data();
  q->r.acq.rec_ix = q->rx.data();
  q->r.acq.rec_iz = q->rz.data();
  q->r.acq.wavelet = q->wav.data();
  q->plan = plan_migration(req->grid, req->acq, req->opts, 1);
  q->need1 = q->plan.shared_bytes + q->plan.item_bytes;
  long long nb = a.nshot;
  const RunConfig cfg = config_for(ctx, req->grid, req->opts);
  const int cap = ctx->max_batch > 0 ? ctx->max_batch : cfg.max_items;
  if (cap > 0 && nb > cap) nb = cap;
  q->want = q->plan.shared_bytes + (size_t)nb * q->plan.item_bytes;
  if (q->need1 > ctx->budget)
    return fail(ctx, RTM_ERR_NOMEM, "request needs %.3f GB, budget is %.3f GB", q->need1 / 1e9,
                ctx->budget / 1e9);
  rtm_server *S = ensure_server(ctx);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(ctx, RTM_ERR_STATE, "the context is being destroyed");
    if ((int)S->queue.size() >= rtm_server::kMaxQueue)
      return fail(ctx, RTM_ERR_BUSY, "request queue is full (%d)", rtm_server::kMaxQueue);
    q->id = S->next++;
    S->queue.push_back(q);
    S->all[q->id] = q;
    *ticket = q->id;
  }
  S->cv.notify_all();
  return RTM_OK;
}

int rtm_server_poll(rtm_ctx *ctx, uint64_t ticket, int *state, int timeout_ms) {
  if (!state) return fail(ctx, RTM_ERR_ARG, "state must not be NULL");
  rtm_server *S = ctx->server;
  if (!S) return fail(ctx, RTM_ERR_STATE, "unknown ticket %llu", (unsigned long long)ticket);
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end())
    return fail(ctx, RTM_ERR_STATE, "unknown ticket %llu", (unsigned long long)ticket);
  auto q = it->second;
  auto done = [&]() { return q->state == RTM_REQ_DONE || q->state == RTM_REQ_FAILED; };
  if (timeout_ms > 0) S->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
  *state = q->state;
  if (!done()) return RTM_ERR_TIMEOUT;
  S->all.erase(it);
  if (q->state == RTM_REQ_FAILED) {
    std::string e = q->err;
    lk.unlock();
    fail(ctx, q->rc, "request %llu failed: %s", (unsigned long long)ticket, e.c_str());
  }
  return RTM_OK;
}

bool rtm_server_shutdown(rtm_ctx *ctx) {
  rtm_server *S = ctx->server;
  if (!S) return true;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    // cancel what never started; wait (bounded) for running requests
    for (auto &q : S->queue) {
      q->state = RTM_REQ_FAILED;
      q->rc = RTM_ERR_STATE;
      q->err = "context destroyed before the request started";
    }
    S->queue.clear();
    S->cv.wait_for(lk, std::chrono::seconds(600), [&]() { return S->running == 0; });
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->sched.joinable()) S->sched.join();
  bool idle;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    idle = S->running == 0;
  }
  if (!idle) return false;  // requests still running after the bound keep S (and ctx) alive
  ctx->server = nullptr;
  delete S;
  return true;
}

void rtm_server_counters(rtm_ctx *ctx, bool reset, long long *peak_running,
                         long long *backfilled) {
  *peak_running = *backfilled = 0;
  rtm_server *S = ctx->server;
  if (!S) return;
  std::lock_guard<std::mutex> lk(S->mu);
  *peak_running = S->peak_running;
  *backfilled = S->backfilled;
  if (reset) {
    S->peak_running = S->running;
    S->backfilled = 0;
  }
}
