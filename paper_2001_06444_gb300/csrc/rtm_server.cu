// rtm_server.cu — request loop with continuous batching.
//
// Requests (one velocity model, its shots and data) queue in arrival order.
// A scheduler thread admits the head of the queue as soon as the context's
// memory budget can hold its snapshot buffers (at least one shot in flight,
// up to all of its shots), gives it its own CUDA stream and a launcher thread,
// and moves on: requests that arrive while others run join the device work as
// memory frees up, and their kernels overlap on the GPU.  Admission is strictly
// in order (no request overtakes an earlier one), so nothing starves.  Every
// wait is bounded; a request that fails reports FAILED with its error text.
//
// The paper runs independent migrations in MPI subgroups, starting the next
// one as soon as a subgroup finishes (§3); this is the single-GPU counterpart.
#include <cuda_runtime.h>

#include <chrono>
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
  static constexpr int kMaxQueue = 4096;
  static constexpr int kMaxRunning = 32;
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
  if (!rc) rc = check_velocity(ctx, q->r.grid, q->r.vel, (long long)q->r.grid.nx * q->r.grid.nz, st);
  if (!rc)
    rc = migrate_device(ctx, q->r.grid, 1, q->r.vel, q->r.acq, q->r.seis, q->r.opts, q->r.image,
                        B, st, config_for(ctx, q->r.grid, q->r.opts));
  if (st) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (!rc && e != cudaSuccess) {
      rc = RTM_ERR_CUDA;
      err = cudaGetErrorString(e);
    }
    cudaStreamDestroy(st);
  }
  if (rc && err.empty()) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    err = ctx->err;
  }
  unreserve(ctx, q->reserved);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    q->rc = rc;
    q->err = err;
    q->state = rc ? RTM_REQ_FAILED : RTM_REQ_DONE;
    S->running--;
  }
  S->cv.notify_all();
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
    if (!got) continue;  // head of the queue waits for memory; retry
    S->queue.pop_front();
    q->reserved = got;
    q->state = RTM_REQ_RUNNING;
    S->running++;
    const long long nitems = q->r.acq.nshot;
    long long B = (long long)((got - q->plan.shared_bytes) / q->plan.item_bytes);
    B = std::max<long long>(1, std::min<long long>(B, nitems));
    std::thread(run_request, ctx, S, q, (int)B).detach();
    S->cv.notify_all();
  }
}

static rtm_server *ensure_server(rtm_ctx *ctx) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!ctx->server) {
    ctx->server = new rtm_server();
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

void rtm_server_shutdown(rtm_ctx *ctx) {
  rtm_server *S = ctx->server;
  if (!S) return;
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
  const bool idle = S->running == 0;
  ctx->server = nullptr;
  if (idle) delete S;  // a request still running after the bound keeps S alive
}
