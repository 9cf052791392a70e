// rtm_api.cu — C ABI entry points and the migration engine (host side).
//
// The engine schedules (velocity sample, shot) migrations as independent work
// items, B of them in flight at a time (B sized by the memory budget), each
// launch of the step kernel advancing all B grids by one time step:
//   forward   n = 0 .. nt-1: u^{n+1} from u^n, u^{n-1}; source c f^n;
//             snapshot S^n stored when n is in K (scale reduced one launch
//             earlier);
//   backward  k = nt .. 1:   w^k from w^{k+1}, w^{k+2}; data c R^T d[k-1];
//             imaging num += S^k w^k, den += (S^k)^2 when k is in K;
//   per item: I = num / (den + eps max den), Kahan-added in shot order to
//             its sample's stack;
//   per call: Laplacian filter of each stack (§3).
// This is Listing 1's shot loop (forward modelling, then adjoint modelling
// with imaging) with the shots and the Monte Carlo samples of §3 run side by
// side on one GPU instead of in MPI subgroups.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rtm_engine.h"
#include "rtm_launch.h"
#include "rtm_trace.h"

namespace rtm {

static thread_local char t_err[512] = "no error";

int fail(rtm_ctx *ctx, int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_err, sizeof(t_err), fmt, ap);
  va_end(ap);
  if (ctx) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::memcpy(ctx->err, t_err, sizeof(ctx->err));
  }
  return code;
}

const char *thread_error() { return t_err; }

// ------------------------------------------------ wait-timeout flag slots --

// Reap pending slots whose copies have landed (with `wait_oldest`, wait for
// the oldest first); a raised one sets timeout_seen.  flag_mu held.
static void reap_flags(rtm_ctx *ctx, bool wait_oldest) {
  for (auto it = ctx->pending.begin(); it != ctx->pending.end();) {
    const bool first = it == ctx->pending.begin();
    const cudaError_t q =
        (wait_oldest && first) ? cudaEventSynchronize(it->ev) : cudaEventQuery(it->ev);
    if (q == cudaErrorNotReady) {
      ++it;
      continue;
    }
    if (q != cudaSuccess) cudaGetLastError();
    const volatile int *f = ctx->h_flags + 2 * it->slot;
    if (f[0] && !ctx->seen_code) {
      ctx->seen_code = f[0];
      ctx->seen_line = f[1];
    }
    cudaEventDestroy(it->ev);
    ctx->free_flags.push_back(it->slot);
    it = ctx->pending.erase(it);
  }
}

int flag_acquire(rtm_ctx *ctx) {
  std::lock_guard<std::mutex> lk(ctx->flag_mu);
  if (ctx->free_flags.empty()) reap_flags(ctx, false);
  while (ctx->free_flags.empty() && !ctx->pending.empty()) reap_flags(ctx, true);
  if (ctx->free_flags.empty()) return -1;  // more calls in flight than slots
  const int s = ctx->free_flags.back();
  ctx->free_flags.pop_back();
  volatile int *f = ctx->h_flags + 2 * s;
  f[0] = f[1] = 0;
  return s;
}

int flag_take(rtm_ctx *ctx, int slot, int *line) {
  *line = 0;
  if (slot < 0) return 0;
  std::lock_guard<std::mutex> lk(ctx->flag_mu);
  const volatile int *f = ctx->h_flags + 2 * slot;
  const int code = f[0];
  *line = f[1];
  ctx->free_flags.push_back(slot);
  return code;
}

int flag_status(rtm_ctx *ctx, int code, int line, const char *whose) {
  if (!code) return RTM_OK;
  if (code == 2)
    return fail(ctx, RTM_ERR_STATE,
                "a device index check failed in %s (kernel source line %d, debug build); the "
                "access was skipped",
                whose, line);
  return fail(ctx, RTM_ERR_TIMEOUT, "a device-side wait gave up in %s", whose);
}

void flag_defer(rtm_ctx *ctx, int slot, cudaStream_t st) {
  if (slot < 0) return;
  cudaEvent_t ev = nullptr;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(ev, st) != cudaSuccess) {
    // no event: wait for the stream here so the slot can be read now
    cudaGetLastError();
    if (ev) cudaEventDestroy(ev);
    cudaStreamSynchronize(st);
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(ctx->flag_mu);
    const volatile int *f = ctx->h_flags + 2 * slot;
    if (f[0] && !ctx->seen_code) {
      ctx->seen_code = f[0];
      ctx->seen_line = f[1];
    }
    ctx->free_flags.push_back(slot);
    return;
  }
  std::lock_guard<std::mutex> lk(ctx->flag_mu);
  ctx->pending.push_back(rtm_ctx::PendingFlag{slot, ev});
}

// A kernel whose bounded wait gave up raises its call's flag; a call that
// synchronises reports it itself, an asynchronous call's flag is reported by
// the first call on the context that finds it complete.
int check_wait_flag(rtm_ctx *ctx) {
  int code, line;
  {
    std::lock_guard<std::mutex> lk(ctx->flag_mu);
    reap_flags(ctx, false);
    code = ctx->seen_code;
    line = ctx->seen_line;
    ctx->seen_code = ctx->seen_line = 0;
  }
  return flag_status(ctx, code, line, "an earlier call");
}

#define CU(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(ctx, RTM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

cudaError_t DevBuf::alloc(rtm_ctx *ctx, size_t n, cudaStream_t s) {
  release();
  st = s;
  bytes = n;
  if (n == 0) return cudaSuccess;
  return cudaMallocFromPoolAsync(&p, n, ctx->pool, s);
}

void DevBuf::release() {
  if (p) cudaFreeAsync(p, st);
  p = nullptr;
  bytes = 0;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static long long round_up(long long a, long long m) { return (a + m - 1) / m * m; }

Geo make_geo(const rtm_grid &gr, int tile_z) {
  Geo g;
  g.nb = gr.nb;
  g.nz = gr.nz;
  g.nx = gr.nx;
  g.NZ = gr.nz + 2 * gr.nb;
  g.NX = gr.nx + 2 * gr.nb;
  g.X0 = (4 - gr.nb % 4) % 4;
  g.CP = g.X0 + gr.nb;
  g.SX = (int)round_up(gr.nx, 4);
  // the pitch covers the padded domain and the 4-aligned physical window
  g.P = (int)round_up(std::max(g.X0 + g.NX, g.CP + g.SX), 32);
  g.ntx = (g.P + TX - 1) / TX;
  g.ntz = (g.NZ + TZ - 1) / TZ;
  g.ntx2 = (g.P + step2_tile_x() - 1) / step2_tile_x();
  g.tz2 = tile_z;
  g.ntz2 = (g.NZ + tile_z - 1) / tile_z;
  g.plane = (long long)g.NZ * g.P;
  g.pplane = (long long)g.nz * g.SX;
  return g;
}

// 8th-order central second-derivative weights (§3: eighth order in space).
static const double kA8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

Coef make_coef(const rtm_grid &gr) {
  Coef k;
  const double rx = 1.0 / (gr.dx * gr.dx), rz = 1.0 / (gr.dz * gr.dz);
  k.c0 = (float)(kA8[0] * (rx + rz));
  k.iso = 1;
  for (int m = 1; m <= 4; ++m) {
    k.ax[m - 1] = (float)(kA8[m] * rx);
    k.az[m - 1] = (float)(kA8[m] * rz);
    k.iso &= k.ax[m - 1] == k.az[m - 1];
  }
  return k;
}

static size_t snap_elem_bytes(int dtype) { return dtype == RTM_SNAP_F32 ? 4 : 2; }

// Segment length of checkpoint mode (0 = keep every snapshot).  Even, so
// two-step launches never straddle a checkpoint; -1 picks the length that
// minimises checkpoints (2 planes each) plus the snapshot ring.
int checkpoint_steps(const rtm_opts &op, const rtm_grid &gr, const Geo &g) {
  if (op.checkpoint == 0) return 0;
  long long c = op.checkpoint;
  if (c < 0) {
    const double esz = op.snap_dtype == RTM_SNAP_F32 ? 4.0 : 2.0;
    c = (long long)std::llround(
        std::sqrt(2.0 * (double)g.plane * gr.nt * op.isnap / ((double)g.pplane * esz)));
  }
  c += c & 1;
  if (c < 2) c = 2;
  return c >= gr.nt ? 0 : (int)c;
}

MigrationPlan plan_migration(const rtm_grid &gr, const rtm_acq &acq, const rtm_opts &op,
                             int nsample) {
  MigrationPlan p;
  p.g = make_geo(gr, 16);  // the shorter tile: the larger per-tile tables
  p.nsnap = gr.nt / op.isnap;
  const Geo &g = p.g;
  const int cpC = checkpoint_steps(op, gr, g);
  if (!cpC) {
    p.item_bytes = 4 * (size_t)g.plane * 4 +
                   (size_t)p.nsnap * g.pplane * snap_elem_bytes(op.snap_dtype) +
                   2 * (size_t)g.pplane * 4 + (size_t)(p.nsnap + 1) * 4 + 256 * 6;
  } else {  // two field sets, the checkpoints, the snapshot ring
    const size_t nseg = (gr.nt + cpC - 1) / cpC, ring = cpC / op.isnap + 1;
    p.item_bytes = 8 * (size_t)g.plane * 4 + nseg * 2 * (size_t)g.plane * 4 +
                   ring * g.pplane * snap_elem_bytes(op.snap_dtype) + 2 * (size_t)g.pplane * 4 +
                   (ring + 1) * 4 + 256 * 10;
  }
  p.shared_bytes = (size_t)nsample * g.plane * 4 + (size_t)g.P * 4 + (size_t)g.NZ * 4 +
                   (size_t)acq.nshot * 8 + (size_t)(g.ntx * g.ntz + 1) * 4 +
                   (size_t)acq.nrec * 40 + (size_t)(g.ntx2 * g.ntz2 + 1) * 8 + (size_t)gr.nt * 4 +
                   2 * (size_t)nsample * g.pplane * 4 +
                   (size_t)acq.nshot * (size_t)nsample * 8 + 4096;
  return p;
}

// -------------------------------------------------------------- checks --

int check_grid(rtm_ctx *ctx, const rtm_grid *g) {
  if (!g) return fail(ctx, RTM_ERR_ARG, "grid is NULL");
  if (g->nx < 1 || g->nz < 1 || g->nb < 0 || g->nt < 1)
    return fail(ctx, RTM_ERR_ARG, "bad grid sizes nx=%d nz=%d nb=%d nt=%d", g->nx, g->nz, g->nb,
                g->nt);
  if (!(g->dx > 0 && g->dz > 0 && g->dt > 0) || !std::isfinite(g->dx) || !std::isfinite(g->dz) ||
      !std::isfinite(g->dt))
    return fail(ctx, RTM_ERR_ARG, "bad spacing dx=%g dz=%g dt=%g", g->dx, g->dz, g->dt);
  const long long NZ = (long long)g->nz + 2LL * g->nb, NX = (long long)g->nx + 2LL * g->nb;
  if (NZ * (NX + 64) >= (1LL << 31) || NZ > 65535LL * TZ)
    return fail(ctx, RTM_ERR_ARG, "grid too large (%lld x %lld padded)", NZ, NX);
  return RTM_OK;
}

int check_acq(rtm_ctx *ctx, const rtm_grid *g, const rtm_acq *a, bool need_rec) {
  if (!a) return fail(ctx, RTM_ERR_ARG, "acquisition is NULL");
  if (a->nshot < 1 || !a->src_ix || !a->src_iz)
    return fail(ctx, RTM_ERR_ARG, "need at least one source (nshot=%d)", a->nshot);
  if (a->nrec < (need_rec ? 1 : 0) || (a->nrec > 0 && (!a->rec_ix || !a->rec_iz)))
    return fail(ctx, RTM_ERR_ARG, "bad receiver set (nrec=%d)", a->nrec);
  if (!a->wavelet) return fail(ctx, RTM_ERR_ARG, "wavelet is NULL");
  for (int s = 0; s < a->nshot; ++s)
    if (a->src_ix[s] < 0 || a->src_ix[s] >= g->nx || a->src_iz[s] < 0 || a->src_iz[s] >= g->nz)
      return fail(ctx, RTM_ERR_ARG, "source %d at (ix=%d, iz=%d) is outside the %dx%d grid", s,
                  a->src_ix[s], a->src_iz[s], g->nx, g->nz);
  for (int r = 0; r < a->nrec; ++r)
    if (a->rec_ix[r] < 0 || a->rec_ix[r] >= g->nx || a->rec_iz[r] < 0 || a->rec_iz[r] >= g->nz)
      return fail(ctx, RTM_ERR_ARG, "receiver %d at (ix=%d, iz=%d) is outside the %dx%d grid", r,
                  a->rec_ix[r], a->rec_iz[r], g->nx, g->nz);
  for (int n = 0; n < g->nt; ++n)
    if (!std::isfinite(a->wavelet[n]))
      return fail(ctx, RTM_ERR_ARG, "wavelet sample %d is not finite", n);
  return RTM_OK;
}

int check_opts(rtm_ctx *ctx, const rtm_opts *o) {
  if (!o) return fail(ctx, RTM_ERR_ARG, "options are NULL");
  if (o->isnap < 1) return fail(ctx, RTM_ERR_ARG, "isnap must be >= 1 (got %d)", o->isnap);
  if (o->snap_dtype < 0 || o->snap_dtype > 2)
    return fail(ctx, RTM_ERR_ARG, "snap_dtype must be 0, 1 or 2 (got %d)", o->snap_dtype);
  if (!(o->eps >= 0) || !std::isfinite(o->eps))
    return fail(ctx, RTM_ERR_ARG, "eps must be finite and >= 0");
  if (o->checkpoint < -1) return fail(ctx, RTM_ERR_ARG, "checkpoint must be >= -1");
  return RTM_OK;
}

// Closed form of the stability bound of leapfrog with the 8th-order stencil:
// v dt sqrt((1/dx^2 + 1/dz^2) * 2048/315) <= 2, 2048/315 being minus the
// symbol of the 1D weights at the Nyquist wavenumber.
static double courant_number(double vmax, const rtm_grid &gr) {
  return vmax * gr.dt * std::sqrt((1.0 / (gr.dx * gr.dx) + 1.0 / (gr.dz * gr.dz)) * 2048.0 / 315.0) /
         2.0;
}

int check_velocity(rtm_ctx *ctx, const rtm_grid &gr, const float *vel_d, long long n,
                   cudaStream_t st) {
  DevBuf r;
  CU(r.alloc(ctx, 16, st));
  // pageable copies: the H2D is staged before the call returns and the D2H
  // completes before it returns, so stack arrays are safe here
  const unsigned init[4] = {0u, 0x7f7fffffu, 0u, 0u};
  CU(cudaMemcpyAsync(r.p, init, 16, cudaMemcpyHostToDevice, st));
  CU(launch_vrange(vel_d, n, r.as<unsigned>(), st));
  unsigned out[4];
  CU(cudaMemcpyAsync(out, r.p, 16, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (out[2]) return fail(ctx, RTM_ERR_ARG, "%u velocity values are non-positive or not finite", out[2]);
  float vmax;
  std::memcpy(&vmax, &out[0], 4);
  const double cn = courant_number(vmax, gr);
  if (cn > 1.0)
    return fail(ctx, RTM_ERR_CFL,
                "CFL violated: v_max dt sqrt((1/dx^2+1/dz^2) 2048/315)/2 = %.6f > 1 (v_max=%g)", cn,
                (double)vmax);
  return RTM_OK;
}

// ---------------------------------------------------- memory admission --

size_t reserve_wait(rtm_ctx *ctx, size_t want, size_t min_need, int timeout_ms) {
  std::unique_lock<std::mutex> lk(ctx->mu);
  auto avail = [&]() { return ctx->budget > ctx->used ? ctx->budget - ctx->used : 0; };
  if (timeout_ms > 0)
    ctx->mem_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                         [&]() { return avail() >= min_need; });
  const size_t a = avail();
  if (a < min_need) return 0;
  const size_t got = std::min(want, a);
  ctx->used += got;
  return got;
}

void unreserve(rtm_ctx *ctx, size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->used = ctx->used > bytes ? ctx->used - bytes : 0;
  }
  ctx->mem_cv.notify_all();
}

// ------------------------------------------------------------- engine --

static void sponge_profile(int N, int nb, std::vector<double> &out) {
  out.resize(N);
  for (int I = 0; I < N; ++I) {
    const int k = std::min(I, N - 1 - I);
    if (k >= nb) {
      out[I] = 1.0;
    } else {
      const double a = 0.015 * (double)(nb - k);
      out[I] = std::exp(-a * a);
    }
  }
}

void sponge_tables(const Geo &g, std::vector<float> &gx, std::vector<float> &gz) {
  std::vector<double> pz, px;
  sponge_profile(g.NZ, g.nb, pz);
  sponge_profile(g.NX, g.nb, px);
  gz.assign(g.NZ, 0.f);
  gx.assign(g.P, 0.f);
  for (int I = 0; I < g.NZ; ++I) gz[I] = (float)pz[I];
  for (int J = 0; J < g.NX; ++J) gx[g.X0 + J] = (float)px[J];
}

void receiver_tiles(const Geo &g, const rtm_acq &acq, std::vector<int> &rptr,
                    std::vector<int2> &rent) {
  const int ntiles = g.ntx * g.ntz;
  rptr.assign(ntiles + 1, 0);
  std::vector<int> rtile(acq.nrec);
  for (int r = 0; r < acq.nrec; ++r) {
    const int row = acq.rec_iz[r] + g.nb, col = acq.rec_ix[r] + g.CP;
    rtile[r] = (row / TZ) * g.ntx + col / TX;
    rptr[rtile[r] + 1]++;
  }
  for (int t = 0; t < ntiles; ++t) rptr[t + 1] += rptr[t];
  rent.assign(std::max(acq.nrec, 1), make_int2(0, 0));
  std::vector<int> fill(rptr.begin(), rptr.end() - 1);
  for (int r = 0; r < acq.nrec; ++r) {
    const int row = acq.rec_iz[r] + g.nb, col = acq.rec_ix[r] + g.CP;
    const int t = rtile[r];
    const int lr = row - (t / g.ntx) * TZ, lc = col - (t % g.ntx) * TX;
    rent[fill[t]++] = make_int2(lr * TX + lc, r);
  }
}

// ------------------------------------------------------- tensor maps --

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    cudaGetLastError();
  });
  return fn;
}

// 3D map over [depth][NZ][P] floats with a (bx, bz, 1) box; out-of-range
// elements of a box read as zero.
static int make_map(rtm_ctx *ctx, CUtensorMap *m, const float *base, const Geo &g, int depth,
                    int bx, int bz) {
  auto fn = encode_fn();
  if (!fn) return fail(ctx, RTM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[3] = {(cuuint64_t)g.P, (cuuint64_t)g.NZ, (cuuint64_t)depth};
  const cuuint64_t strides[2] = {(cuuint64_t)g.P * 4, (cuuint64_t)g.plane * 4};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)bz, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, RTM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return RTM_OK;
}

// ---------------------------------------------------------------- engine --

struct Common {
  Geo g;
  Coef k;
  int nsample = 1;
  int kernel = 2;  // RunConfig::step_kernel of the call
  int l2_ahead = 0;  // RunConfig::l2_ahead of the call
  int pdl = 0;       // RunConfig::pdl of the call
  long long n_rent = 0, n_rext = 0, n_rcen = 0;  // receiver-table entries (debug index checks)
  DevBuf c_all, gx, gz, src_rc, rptr, rent, rext_ptr, rext_ent, rcen_ptr, rcen_ent, wav, items, err;
  CUtensorMap mc;
};

// Receiver lists of the two-step tiles: every tile whose extended region
// (tile plus a 4-point ring) holds the receiver, and the one tile whose centre
// does; offsets are r * EX + c within the extended region.
static void step2_receiver_lists(const Geo &g, const rtm_acq &acq, std::vector<int> &eptr,
                                 std::vector<int2> &eent, std::vector<int> &cptr,
                                 std::vector<int2> &cent) {
  const int TXc = step2_tile_x(), TZc = g.tz2, H = step2_ext(), EXw = TXc + 2 * H;
  const int nt2 = g.ntx2 * g.ntz2;
  std::vector<std::vector<int2>> e(nt2), c(nt2);
  for (int r = 0; r < acq.nrec; ++r) {
    const int row = acq.rec_iz[r] + g.nb, col = acq.rec_ix[r] + g.CP;
    const int bx = col / TXc, bz = row / TZc;
    for (int tz = std::max(0, bz - 1); tz <= std::min(g.ntz2 - 1, bz + 1); ++tz)
      for (int tx = std::max(0, bx - 1); tx <= std::min(g.ntx2 - 1, bx + 1); ++tx) {
        const int er = row - (tz * TZc - H), ec = col - (tx * TXc - H);
        if (er < 0 || er >= TZc + 2 * H || ec < 0 || ec >= EXw) continue;
        const int2 en = make_int2(er * EXw + ec, r);
        e[tz * g.ntx2 + tx].push_back(en);
        if (er >= H && er < H + TZc && ec >= H && ec < H + TXc) c[tz * g.ntx2 + tx].push_back(en);
      }
  }
  eptr.assign(nt2 + 1, 0);
  cptr.assign(nt2 + 1, 0);
  eent.clear();
  cent.clear();
  for (int t = 0; t < nt2; ++t) {
    eent.insert(eent.end(), e[t].begin(), e[t].end());
    cent.insert(cent.end(), c[t].begin(), c[t].end());
    eptr[t + 1] = (int)eent.size();
    cptr[t + 1] = (int)cent.size();
  }
  if (eent.empty()) eent.push_back(make_int2(0, 0));
  if (cent.empty()) cent.push_back(make_int2(0, 0));
}

// Upload the per-call tables shared by all items.
static int setup_common(rtm_ctx *ctx, Common &C, const rtm_grid &gr, const rtm_acq &acq,
                        int nsample, const float *vel_d, cudaStream_t st, int step_kernel,
                        int tile_z, int l2_ahead, int pdl) {
  C.g = make_geo(gr, step_kernel >= 3 ? tile_z : 24);
  C.kernel = step_kernel;
  C.l2_ahead = l2_ahead;
  C.pdl = pdl;
  C.k = make_coef(gr);
  C.nsample = nsample;
  const Geo &g = C.g;
  std::vector<float> gz, gx;
  sponge_tables(g, gx, gz);
  // sources: memory (row, col); receivers: CSR over single-step tiles
  std::vector<int> src(2 * acq.nshot);
  for (int s = 0; s < acq.nshot; ++s) {
    src[s] = acq.src_iz[s] + g.nb;
    src[acq.nshot + s] = acq.src_ix[s] + g.CP;
  }
  std::vector<int> rptr;
  std::vector<int2> rent;
  receiver_tiles(g, acq, rptr, rent);
  std::vector<int> eptr, cptr;
  std::vector<int2> eent, cent;
  step2_receiver_lists(g, acq, eptr, eent, cptr, cent);
  C.n_rent = (long long)rent.size();
  C.n_rext = (long long)eent.size();
  C.n_rcen = (long long)cent.size();
  CU(C.c_all.alloc(ctx, (size_t)nsample * g.plane * 4, st));
  CU(C.gx.alloc(ctx, gx.size() * 4, st));
  CU(C.gz.alloc(ctx, gz.size() * 4, st));
  CU(C.src_rc.alloc(ctx, src.size() * 4, st));
  CU(C.rptr.alloc(ctx, rptr.size() * 4, st));
  CU(C.rent.alloc(ctx, rent.size() * sizeof(int2), st));
  CU(C.rext_ptr.alloc(ctx, eptr.size() * 4, st));
  CU(C.rext_ent.alloc(ctx, eent.size() * sizeof(int2), st));
  CU(C.rcen_ptr.alloc(ctx, cptr.size() * 4, st));
  CU(C.rcen_ent.alloc(ctx, cent.size() * sizeof(int2), st));
  CU(C.wav.alloc(ctx, (size_t)gr.nt * 4, st));
  CU(C.err.alloc(ctx, 16, st));
  CU(cudaMemcpyAsync(C.gx.p, gx.data(), gx.size() * 4, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(C.gz.p, gz.data(), gz.size() * 4, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(C.src_rc.p, src.data(), src.size() * 4, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(C.rptr.p, rptr.data(), rptr.size() * 4, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(C.rent.p, rent.data(), rent.size() * sizeof(int2), cudaMemcpyHostToDevice,
                     st));
  CU(cudaMemcpyAsync(C.rext_ptr.p, eptr.data(), eptr.size() * 4, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(C.rext_ent.p, eent.data(), eent.size() * sizeof(int2),
                     cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(C.rcen_ptr.p, cptr.data(), cptr.size() * 4, cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(C.rcen_ent.p, cent.data(), cent.size() * sizeof(int2),
                     cudaMemcpyHostToDevice, st));
  CU(cudaMemcpyAsync(C.wav.p, acq.wavelet, (size_t)gr.nt * 4, cudaMemcpyHostToDevice, st));
  CU(cudaMemsetAsync(C.err.p, 0, 16, st));
  CU(launch_prep_c(vel_d, C.c_all.as<float>(), g, gr.dt, nsample, st));
  if (step_kernel >= 2) {
    const int H = step2_ext();
    int rc = make_map(ctx, &C.mc, C.c_all.as<float>(), g, nsample, step2_tile_x() + 2 * H,
                      g.tz2 + 2 * H);
    if (rc) return rc;
  }
  // the host vectors above go out of scope: make the copies complete first
  CU(cudaStreamSynchronize(st));
  return RTM_OK;
}

// Field buffers of B items: v ping-pong, d ping-pong (the two-step kernel
// reads d in a halo, so it cannot update it in place; the single-step kernel
// does, in whichever buffer is current).
struct Fields {
  DevBuf v[2], d[2];
  CUtensorMap mv[2], md[2];
  int cv = 0, cd = 0;  // index of the current v and d buffer
  int n2 = 0;          // two-step launches since the fields were zeroed (snake order parity)
};

static int alloc_fields(rtm_ctx *ctx, Fields &F, const Geo &g, int B, cudaStream_t st,
                        int step_kernel) {
  for (int i = 0; i < 2; ++i) {
    CU(F.v[i].alloc(ctx, (size_t)B * g.plane * 4, st));
    CU(F.d[i].alloc(ctx, (size_t)B * g.plane * 4, st));
    if (step_kernel >= 2) {
      const int H = step2_ext();
      int rc = make_map(ctx, &F.mv[i], F.v[i].as<float>(), g, B, step2_tile_x() + 4 * H,
                        g.tz2 + 4 * H);
      if (!rc)
        rc = make_map(ctx, &F.md[i], F.d[i].as<float>(), g, B, step2_tile_x() + 2 * H,
                      g.tz2 + 2 * H);
      if (rc) return rc;
    }
  }
  return RTM_OK;
}

static int zero_fields(rtm_ctx *ctx, Fields &F, const Geo &g, int nb, cudaStream_t st) {
  for (int i = 0; i < 2; ++i) {
    CU(cudaMemsetAsync(F.v[i].p, 0, (size_t)nb * g.plane * 4, st));
    CU(cudaMemsetAsync(F.d[i].p, 0, (size_t)nb * g.plane * 4, st));
  }
  F.cv = F.cd = F.n2 = 0;
  return RTM_OK;
}

static void fill_args(StepArgs &A, const Common &C, const rtm_grid &gr, const rtm_acq &acq) {
  std::memset(&A, 0, sizeof(A));
  A.g = C.g;
  A.k = C.k;
  A.gx = C.gx.as<float>();
  A.gz = C.gz.as<float>();
  A.c_all = C.c_all.as<float>();
  A.src_row = C.src_rc.as<int>();
  A.src_col = C.src_rc.as<int>() + acq.nshot;
  A.wav = C.wav.as<float>();
  A.src_scale = (float)(1.0 / (gr.dx * gr.dz));
  A.rtile_ptr = C.rptr.as<int>();
  A.rtile_ent = C.rent.as<int2>();
  A.nrec = acq.nrec;
  A.nt = gr.nt;
  A.err = C.err.as<int>();
  A.len.nshot = acq.nshot;
  A.len.nsample = C.nsample;
  A.len.rent = C.n_rent;
  A.len.rcen = C.n_rcen;
}

static void fill_args2(Step2Args &A2, const StepArgs &A, const Common &C) {
  std::memset(&A2, 0, sizeof(A2));
  A2.g = A.g;
  A2.k = A.k;
  A2.gx = A.gx;
  A2.gz = A.gz;
  A2.c_all = A.c_all;
  A2.item_sample = A.item_sample;
  A2.item_shot = A.item_shot;
  A2.one_sample = C.nsample == 1;
  A2.src_row = A.src_row;
  A2.src_col = A.src_col;
  A2.wav = A.wav;
  A2.src_scale = A.src_scale;
  A2.rext_ptr = C.rext_ptr.as<int>();
  A2.rext_ent = C.rext_ent.as<int2>();
  A2.rcen_ptr = C.rcen_ptr.as<int>();
  A2.rcen_ent = C.rcen_ent.as<int2>();
  A2.nrec = A.nrec;
  A2.nt = A.nt;
  A2.seis = A.seis;
  A2.rec_out = A.rec_out;
  A2.snap = A.snap;
  A2.snap_dtype = A.snap_dtype;
  A2.nsnap = A.nsnap;
  A2.smax = A.smax;
  A2.num = A.num;
  A2.den = A.den;
  A2.dmax = A.dmax;
  A2.err = C.err.as<int>();
  A2.refl = A.refl;
  A2.len = A.len;
  A2.len.rent = C.n_rext;
}

// Test hook: if injections are pending, take one and raise this call's flag.
static int maybe_inject_timeout(rtm_ctx *ctx, const Common &C, cudaStream_t st) {
  int n = ctx->inject_timeouts.load();
  while (n > 0 && !ctx->inject_timeouts.compare_exchange_weak(n, n - 1)) {
  }
  static const int kRaised = 1;  // (a pageable copy is staged before the call returns)
  if (n > 0) CU(cudaMemcpyAsync(C.err.p, &kRaised, 4, cudaMemcpyHostToDevice, st));
  return RTM_OK;
}

// One single-step launch: v from the current buffer into the other, d in place.
static int step1(rtm_ctx *ctx, int mode, StepArgs &A, Fields &F, const StepRT &rt, int nb,
                 cudaStream_t st) {
  A.fa = F.v[F.cv].as<float>();
  A.fb = F.v[1 - F.cv].as<float>();
  A.fd = F.d[F.cd].as<float>();
  CU(launch_step(mode, A, rt, nb, st));
  F.cv = 1 - F.cv;
  return RTM_OK;
}

// One two-step launch: both v and d into the other buffers.  The persistent
// kernel walks its tiles in snake order: every other launch from the end of
// the tile list, so it starts on the grids the previous launch wrote last.
static int step2(rtm_ctx *ctx, int mode, Step2Args &A2, const Common &C, Fields &F,
                 const Step2RT &rt, int nb, cudaStream_t st) {
  A2.v_out = F.v[1 - F.cv].as<float>();
  A2.d_out = F.d[1 - F.cd].as<float>();
  A2.v_in = F.v[F.cv].as<float>();
  A2.d_in = F.d[F.cd].as<float>();
  Step2RT r = rt;
  r.reverse = F.n2 & 1;
  r.ahead = C.l2_ahead;
  // (programmatic dependent launches are built for the migration's phases)
  r.pdl = C.kernel == 4 && C.pdl && (mode == MODE_FWD || mode == MODE_BWD);
  if (C.kernel == 3)
    CU(launch_step2p(mode, C.g.tz2, F.mv[F.cv], F.md[F.cd], C.mc, A2, r, nb, st));
  else if (C.kernel == 4)
    CU(launch_step2a(mode, C.g.tz2, F.mv[F.cv], F.md[F.cd], C.mc, A2, r, nb, st));
  else
    CU(launch_step2(mode, F.mv[F.cv], F.md[F.cd], C.mc, A2, r, nb, st));
  F.cv = 1 - F.cv;
  F.cd = 1 - F.cd;
  F.n2 += 1;
  return RTM_OK;
}

RunConfig config_for(rtm_ctx *ctx, const rtm_grid &gr, const rtm_opts &op) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->tuned.find(TuneKey{gr.nx, gr.nz, gr.nb, gr.nt, op.isnap, op.snap_dtype});
  return it != ctx->tuned.end() ? it->second : ctx->defaults;
}

// Issue `issue()` on st, either directly or captured once into a CUDA graph
// that is then launched (one launch for a whole phase of a batch).
template <class F>
static int run_phase(rtm_ctx *ctx, bool graph, cudaStream_t st, F issue) {
  // the legacy default stream cannot be captured: launch directly there
  if (!graph || st == nullptr || st == cudaStreamLegacy) return issue();
  CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const int rc = issue();
  cudaGraph_t gph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &gph);
  trace_mark("  graph captured");
  if (rc) {
    if (gph) cudaGraphDestroy(gph);
    return rc;
  }
  if (e != cudaSuccess) return fail(ctx, RTM_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&ex, gph, 0);
  cudaGraphDestroy(gph);
  trace_mark("  graph instantiated");
  if (ei != cudaSuccess) return fail(ctx, RTM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
  const cudaError_t el = cudaGraphLaunch(ex, st);
  trace_mark("  graph launched");
  cudaGraphExecDestroy(ex);  // released once the launch completes
  trace_mark("  graph released");
  if (el != cudaSuccess) return fail(ctx, RTM_ERR_CUDA, "graph launch failed: %s", cudaGetErrorString(el));
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->stats.graph_launches += 1;
  }
  return RTM_OK;
}

int migrate_device(rtm_ctx *ctx, const rtm_grid &gr, int nsample, const float *vel_d,
                   const rtm_acq &acq, const float *seis_d, const rtm_opts &op, float *img_d,
                   int B, cudaStream_t st, const RunConfig &cfg, const float *born_refl,
                   float *born_out, LateCopy *late, int flag_slot) {
  Common C;
  int rc;
  {
    PhaseRange ph("setup");
    rc = setup_common(ctx, C, gr, acq, nsample, vel_d, st, cfg.step_kernel, cfg.tile_z,
                      cfg.l2_ahead, cfg.pdl);
  }
  if (!rc) rc = maybe_inject_timeout(ctx, C, st);
  if (rc) return rc;
  trace_mark("tables and model set up");
  const Geo &g = C.g;
  const int nsnap = gr.nt / op.isnap;
  const long long nitems = (long long)nsample * acq.nshot;
  if (B > nitems) B = (int)nitems;
  if (B < 1) B = 1;
  // items in (sample, shot) order
  std::vector<int> items(2 * nitems);
  for (long long q = 0; q < nitems; ++q) {
    items[q] = (int)(q / acq.nshot);
    items[nitems + q] = (int)(q % acq.nshot);
  }
  CU(C.items.alloc(ctx, items.size() * 4, st));
  CU(cudaMemcpyAsync(C.items.p, items.data(), items.size() * 4, cudaMemcpyHostToDevice, st));
  const size_t esz = snap_elem_bytes(op.snap_dtype);
  // checkpoint mode: the state every cpC steps instead of every snapshot;
  // each segment's snapshots are recomputed into a ring of `ring` slots
  const int cpC = checkpoint_steps(op, gr, g);
  const int nseg = cpC ? (gr.nt + cpC - 1) / cpC : 0;
  const int ring = cpC ? cpC / op.isnap + 1 : nsnap;
  Fields F, U;  // F: forward fields, then the receiver wavefield; U: recomputed forward
  if ((rc = alloc_fields(ctx, F, g, B, st, cfg.step_kernel))) return rc;
  if (cpC && (rc = alloc_fields(ctx, U, g, B, st, cfg.step_kernel))) return rc;
  DevBuf snap, smax, num, den, dmax, stack, comp, cps;
  CU(snap.alloc(ctx, std::max<size_t>((size_t)B * ring * g.pplane * esz, 16), st));
  CU(smax.alloc(ctx, (size_t)B * std::max(ring, 1) * 4, st));
  if (cpC) CU(cps.alloc(ctx, (size_t)nseg * 2 * B * g.plane * 4, st));
  CU(num.alloc(ctx, (size_t)B * g.pplane * 4, st));
  CU(den.alloc(ctx, (size_t)B * g.pplane * 4, st));
  CU(dmax.alloc(ctx, (size_t)B * 4, st));
  CU(stack.alloc(ctx, (size_t)nsample * g.pplane * 4, st));
  CU(comp.alloc(ctx, (size_t)nsample * g.pplane * 4, st));
  CU(cudaMemsetAsync(num.p, 0, num.bytes, st));
  CU(cudaMemsetAsync(den.p, 0, den.bytes, st));
  CU(cudaMemsetAsync(stack.p, 0, stack.bytes, st));
  CU(cudaMemsetAsync(comp.p, 0, comp.bytes, st));

  // algorithmic bytes per item (16 B per padded update; b per physical pixel
  // per snapshot written or read; 16 B per physical pixel per imaging step);
  // recomputation in checkpoint mode is overhead, not counted
  const double upd = (double)g.NZ * g.NX, pix = (double)g.nz * g.nx;
  const double fwd_bytes = gr.nt * 16.0 * upd + nsnap * (double)esz * pix;
  // (Born modelling's second phase reads a snapshot and the reflectivity per
  // pixel on imaging steps instead of updating num and den)
  const double bwd_bytes = gr.nt * 16.0 * upd +
                           nsnap * ((double)esz + (born_refl ? 4.0 : 16.0)) * pix;
  long long launches = 0, step_launches = 0;
  struct Events {  // phase-timing events (profiling), destroyed on every path
    std::vector<cudaEvent_t> v;
    ~Events() {
      for (cudaEvent_t e : v) cudaEventDestroy(e);
    }
  } ev;
  auto mark = [&]() -> int {
    if (!ctx->prof) return RTM_OK;
    cudaEvent_t e;
    CU(cudaEventCreate(&e));
    ev.v.push_back(e);
    CU(cudaEventRecord(e, st));
    return RTM_OK;
  };

  // the late seismogram upload: issued once, behind the first forward phase
  // (outside any graph capture), in per-batch pieces in shot order; batch bi
  // waits for its piece, and so for every earlier one, before backward steps
  auto issue_late = [&](long long bi) -> int {
    if (!late) return RTM_OK;
    if (!late->issued) {
      late->issued = true;
      CU(cudaStreamWaitEvent(late->cs, late->alloc_done, 0));
      const char *src = static_cast<const char *>(late->src);
      char *dst = static_cast<char *>(late->dst);
      int done = 0;  // shots uploaded so far
      for (long long q0 = 0; q0 < nitems; q0 += B) {
        const long long q1 = std::min<long long>(nitems, q0 + B);
        // shots this batch reads (items in (sample, shot) order; a batch
        // that crosses a sample boundary may read any shot)
        const int hi = (q1 - 1) / acq.nshot > q0 / acq.nshot ? acq.nshot
                                                            : (int)((q1 - 1) % acq.nshot) + 1;
        if (hi > done) {
          CU(cudaMemcpyAsync(dst + done * late->shot_bytes, src + done * late->shot_bytes,
                             (size_t)(hi - done) * late->shot_bytes, cudaMemcpyHostToDevice,
                             late->cs));
          done = hi;
        }
        cudaEvent_t e;
        CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        late->ready.push_back(e);
        CU(cudaEventRecord(e, late->cs));
      }
    }
    CU(cudaStreamWaitEvent(st, late->ready[(size_t)bi], 0));
    return RTM_OK;
  };

  StepArgs A;
  fill_args(A, C, gr, acq);
  A.seis = seis_d;
  A.snap = snap.p;
  A.snap_dtype = op.snap_dtype;
  A.nsnap = ring;
  A.smax = smax.as<unsigned>();
  A.num = num.as<float>();
  A.den = den.as<float>();
  A.dmax = dmax.as<unsigned>();
  A.len.items = B;
  A.len.snap = (long long)B * ring * g.pplane;
  A.len.smax = (long long)B * std::max(ring, 1);
  A.len.refl = born_refl ? (long long)g.nz * g.nx : 0;
  A.refl = born_refl;
  const int isnap = op.isnap, nt = gr.nt;
  const bool half = op.snap_dtype != RTM_SNAP_F32;
  const bool two = cfg.step_kernel >= 2;
  const bool graph = cfg.graph != 0;
  auto inK = [&](int m) { return m >= 1 && m <= nt && m % isnap == 0; };
  int nb = 0;
  Step2Args A2;

  // Forward steps n0 .. n1-1 on Fs.  store: keep S^k, k in K and n0 < k <= n1,
  // in slot k/isnap - 1 - kbase.  save: copy the state into checkpoint n/cpC
  // before every step n that is a multiple of cpC.
  auto fwd_range = [&](Fields &Fs, int n0, int n1, int kbase, bool store, bool save) -> int {
    int r2;
    auto idx = [&](int k) { return k / isnap - 1 - kbase; };
    bool stored = true;  // the range's input field is not the range's to store
    for (int n = n0; n < n1;) {
      if (save && n % cpC == 0) {
        const size_t bytes = (size_t)nb * g.plane * 4;
        float *dst = cps.as<float>() + (size_t)(n / cpC) * 2 * B * g.plane;
        CU(cudaMemcpyAsync(dst, Fs.v[Fs.cv].p, bytes, cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpyAsync(dst + (size_t)B * g.plane, Fs.d[Fs.cd].p, bytes,
                           cudaMemcpyDeviceToDevice, st));
      }
      if (two && n + 2 <= n1 && (!half || isnap % 2 == 0)) {
        Step2RT r;
        r.t1 = n;
        r.t2 = n + 1;
        r.snap_in_idx = (store && inK(n) && !stored) ? idx(n) : -1;
        r.snap_mid_idx = (store && !half && inK(n + 1)) ? idx(n + 1) : -1;
        r.snap_out_idx = (store && !half && inK(n + 2)) ? idx(n + 2) : -1;
        r.max_out_idx = (store && half && inK(n + 2)) ? idx(n + 2) : -1;
        r.img_mid_idx = r.img_out_idx = -1;
        r.img_in_idx = -1;
        r.dmax_flag = 0;
        if ((r2 = step2(ctx, MODE_FWD, A2, C, Fs, r, nb, st))) return r2;
        stored = !half;
        n += 2;
      } else {
        StepRT r{};
        r.n = n;
        r.snap_idx = (store && inK(n) && !stored) ? idx(n) : -1;
        r.max_idx = (store && half && inK(n + 1)) ? idx(n + 1) : -1;
        r.img_idx = -1;
        r.dmax_flag = 0;
        if ((r2 = step1(ctx, MODE_FWD, A, Fs, r, nb, st))) return r2;
        stored = false;
        n += 1;
      }
      ++step_launches;
    }
    if (store && inK(n1) && !stored) {
      CU(launch_snap_store(A, Fs.v[Fs.cv].as<float>(), idx(n1), nb, st));
      ++launches;
    }
    return RTM_OK;
  };
  // Backward steps k = k1 .. k0+1 on Ws, imaging with slot k/isnap - 1 - kbase.
  // A two-step launch images its INPUT field where it can (img_in): the loads
  // of its imaging operands then start before its tile copies land.  With an
  // even isnap the steps are paired so that the imaging fields are launch
  // inputs: one single step comes first when k1 is even.  A field is imaged
  // as an output only when no two-step launch takes it as input.  Every field
  // is imaged once, in the same order, so images do not change.
  auto bwd_range = [&](Fields &Ws, int k1, int k0, int kbase) -> int {
    int r2;
    auto idx = [&](int k) { return k / isnap - 1 - kbase; };
    auto single = [&](int k) -> int {  // w^k from w^{k+1}; images w^k
      StepRT r{};
      r.n = k;
      r.snap_idx = r.max_idx = -1;
      r.img_idx = inK(k) ? idx(k) : -1;
      r.dmax_flag = (k == isnap) ? 1 : 0;
      ++step_launches;
      return step1(ctx, MODE_BWD, A, Ws, r, nb, st);
    };
    int k = k1;
    bool in_done = true;  // the next launch's input needs no imaging here
    const bool use_in = cfg.image_input != 0;
    if (use_in && two && isnap % 2 == 0 && k1 % 2 == 0 && k1 - 2 > k0) {
      if ((r2 = single(k))) return r2;
      k -= 1;
    }
    while (k > k0) {
      if (two && k - 1 > k0) {
        Step2RT r;
        r.t1 = k - 1;
        r.t2 = k - 2;
        r.snap_in_idx = r.snap_mid_idx = r.snap_out_idx = r.max_out_idx = -1;
        r.img_in_idx = (!in_done && inK(k + 1)) ? idx(k + 1) : -1;
        r.img_mid_idx = inK(k) ? idx(k) : -1;
        // the launch at k - 2 takes w^{k-1} as input (and images it there)
        const bool next_two = use_in && k - 3 > k0;
        r.img_out_idx = (inK(k - 1) && !next_two) ? idx(k - 1) : -1;
        r.dmax_flag = (r.img_in_idx >= 0 && k + 1 == isnap)    ? 3
                      : (r.img_mid_idx >= 0 && k == isnap)     ? 1
                      : (r.img_out_idx >= 0 && k - 1 == isnap) ? 2
                                                               : 0;
        if ((r2 = step2(ctx, MODE_BWD, A2, C, Ws, r, nb, st))) return r2;
        ++step_launches;
        in_done = !next_two;
        k -= 2;
      } else {
        if ((r2 = single(k))) return r2;
        in_done = true;
        k -= 1;
      }
    }
    return RTM_OK;
  };

  for (long long q0 = 0; q0 < nitems; q0 += B) {
    nb = (int)std::min<long long>(B, nitems - q0);
    A.item_sample = C.items.as<int>() + q0;
    A.item_shot = C.items.as<int>() + nitems + q0;
    fill_args2(A2, A, C);
    if ((rc = zero_fields(ctx, F, g, nb, st))) return rc;
    CU(cudaMemsetAsync(smax.p, 0, smax.bytes, st));
    CU(cudaMemsetAsync(dmax.p, 0, dmax.bytes, st));
    if (!cpC) {
      // forward with every snapshot S^k, k in K; then backward with imaging
      if ((rc = mark())) return rc;
      {
        PhaseRange ph("forward");
        rc = run_phase(ctx, graph, st, [&]() { return fwd_range(F, 0, nt, 0, true, false); });
      }
      if (rc) return rc;
      trace_mark("forward phase enqueued");
      if ((rc = mark())) return rc;
      if (born_refl) {
        // Born modelling: the perturbation field starts at rest; each step
        // adds c m S^{n+1} on imaging steps and records the receivers
        if ((rc = zero_fields(ctx, F, g, nb, st))) return rc;
        A.refl = A2.refl = born_refl;
        A.rec_out = A2.rec_out = born_out + (size_t)q0 * nt * acq.nrec;
        A.len.rec_out = A2.len.rec_out = (nitems - q0) * (long long)nt * acq.nrec;
        if ((rc = mark())) return rc;
        rc = run_phase(ctx, graph, st, [&]() -> int {
          auto slot = [&](int k) { return inK(k) ? k / isnap - 1 : -1; };
          for (int n = 0; n < nt;) {
            int r2;
            if (two && n + 2 <= nt) {
              Step2RT r;
              r.t1 = n;
              r.t2 = n + 1;
              r.snap_in_idx = r.snap_mid_idx = r.snap_out_idx = r.max_out_idx = -1;
              r.img_mid_idx = slot(n + 1);
              r.img_out_idx = slot(n + 2);
              r.img_in_idx = -1;
              r.dmax_flag = 0;
              r2 = step2(ctx, MODE_BORN, A2, C, F, r, nb, st);
              n += 2;
            } else {
              StepRT r{};
              r.n = n;
              r.snap_idx = r.max_idx = -1;
              r.img_idx = slot(n + 1);
              r2 = step1(ctx, MODE_BORN, A, F, r, nb, st);
              n += 1;
            }
            if (r2) return r2;
            ++step_launches;
          }
          return RTM_OK;
        });
        if (rc) return rc;
        if ((rc = mark())) return rc;
        continue;
      }
      if ((rc = zero_fields(ctx, F, g, nb, st))) return rc;
      if ((rc = issue_late(q0 / B))) return rc;
      if ((rc = mark())) return rc;
      {
        PhaseRange ph("backward");
        rc = run_phase(ctx, graph, st, [&]() { return bwd_range(F, nt, 0, 0); });
      }
      if (rc) return rc;
      trace_mark("backward phase enqueued");
      if ((rc = mark())) return rc;
    } else {
      // forward keeping the state every cpC steps; then, segment by segment
      // from the last, recompute the segment's snapshots from its checkpoint
      // and run its backward steps (F carries the receiver wavefield across)
      if ((rc = mark())) return rc;
      rc = run_phase(ctx, graph, st, [&]() { return fwd_range(F, 0, nt, 0, false, true); });
      if (rc) return rc;
      if ((rc = zero_fields(ctx, F, g, nb, st))) return rc;
      if ((rc = issue_late(q0 / B))) return rc;
      for (int sgi = nseg - 1; sgi >= 0 && !rc; --sgi) {
        const int n0 = sgi * cpC, n1 = std::min(nt, n0 + cpC), kbase = n0 / isnap;
        rc = run_phase(ctx, graph, st, [&]() -> int {
          const size_t bytes = (size_t)nb * g.plane * 4;
          const float *src = cps.as<float>() + (size_t)sgi * 2 * B * g.plane;
          CU(cudaMemcpyAsync(U.v[0].p, src, bytes, cudaMemcpyDeviceToDevice, st));
          CU(cudaMemcpyAsync(U.d[0].p, src + (size_t)B * g.plane, bytes, cudaMemcpyDeviceToDevice,
                             st));
          U.cv = U.cd = 0;
          if (half) CU(cudaMemsetAsync(smax.p, 0, smax.bytes, st));
          int r2 = fwd_range(U, n0, n1, kbase, true, false);
          if (!r2) r2 = bwd_range(F, n1, n0, kbase);
          return r2;
        });
      }
      if (rc) return rc;
      if ((rc = mark())) return rc;
    }
    CU(launch_norm_stack(A.num, A.den, A.dmax, A.item_sample, nb, (float)op.eps, g.pplane,
                         stack.as<float>(), comp.as<float>(), nsample, C.err.as<int>(), st));
    launches += 1;
  }
  launches += step_launches;
  if (!born_refl) {
    CU(launch_filter(stack.as<float>(), comp.as<float>(), nsample, g.nz, g.nx, g.SX,
                     (float)(1.0 / (gr.dz * gr.dz)), (float)(1.0 / (gr.dx * gr.dx)),
                     op.laplacian, img_d, st));
    launches += 1;
  }
  launches += 1;  // prep_c
  if (flag_slot >= 0)
    CU(cudaMemcpyAsync(ctx->h_flags + 2 * flag_slot, C.err.p, 8, cudaMemcpyDeviceToHost, st));
  double ms_total = 0.0;
  if (ctx->prof) {
    CU(cudaStreamSynchronize(st));
    for (size_t i = 0; i + 1 < ev.v.size(); i += 2) {
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, ev.v[i], ev.v[i + 1]));
      ms_total += ms;
    }
  }
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->stats.launches += launches;
    if (ctx->prof) {
      ctx->stats.step_launches += step_launches;
      ctx->stats.step_ms += ms_total;
      ctx->stats.step_bytes += (double)nitems * (fwd_bytes + bwd_bytes);
      ctx->stats.point_updates += (double)nitems * 2.0 * gr.nt * upd;
    }
    ctx->stats.migrations += nitems;
  }
  return RTM_OK;
}

// Forward modelling of shots [s0, s0 + ns) into seis_d [ns][nt][nrec]
// (device), B shots advanced per launch.
static int model_device(rtm_ctx *ctx, const rtm_grid &gr, const float *vel_d,
                        const rtm_acq &acq, int s0, int ns, float *seis_d, int B,
                        cudaStream_t st, int flag_slot) {
  const int sk = ctx->defaults.step_kernel;
  Common C;
  int rc = setup_common(ctx, C, gr, acq, 1, vel_d, st, sk, ctx->defaults.tile_z,
                        ctx->defaults.l2_ahead, ctx->defaults.pdl);
  if (!rc) rc = maybe_inject_timeout(ctx, C, st);
  if (rc) return rc;
  const Geo &g = C.g;
  if (B > ns) B = ns;
  if (B < 1) B = 1;
  std::vector<int> items(2 * (size_t)ns);
  for (int q = 0; q < ns; ++q) {
    items[q] = 0;
    items[ns + q] = s0 + q;
  }
  CU(C.items.alloc(ctx, items.size() * 4, st));
  CU(cudaMemcpyAsync(C.items.p, items.data(), items.size() * 4, cudaMemcpyHostToDevice, st));
  Fields F;
  if ((rc = alloc_fields(ctx, F, g, B, st, sk))) return rc;
  StepArgs A;
  fill_args(A, C, gr, acq);
  A.len.items = B;
  const bool two = sk >= 2;
  long long launches = 0;
  for (int q0 = 0; q0 < ns; q0 += B) {
    const int nb = std::min(B, ns - q0);
    if ((rc = zero_fields(ctx, F, g, nb, st))) return rc;
    A.item_sample = C.items.as<int>() + q0;
    A.item_shot = C.items.as<int>() + ns + q0;
    A.rec_out = seis_d + (size_t)q0 * gr.nt * acq.nrec;
    A.len.rec_out = (long long)(ns - q0) * gr.nt * acq.nrec;
    Step2Args A2;
    fill_args2(A2, A, C);
    for (int n = 0; n < gr.nt;) {
      if (two && n + 2 <= gr.nt) {
        Step2RT r;
        r.t1 = n;
        r.t2 = n + 1;
        r.snap_in_idx = r.snap_mid_idx = r.snap_out_idx = r.max_out_idx = -1;
        r.img_mid_idx = r.img_out_idx = r.img_in_idx = -1;
        r.dmax_flag = 0;
        if ((rc = step2(ctx, MODE_MODEL, A2, C, F, r, nb, st))) return rc;
        n += 2;
      } else {
        StepRT r{};
        r.n = n;
        r.snap_idx = r.max_idx = r.img_idx = -1;
        if ((rc = step1(ctx, MODE_MODEL, A, F, r, nb, st))) return rc;
        n += 1;
      }
      ++launches;
    }
  }
  if (flag_slot >= 0)
    CU(cudaMemcpyAsync(ctx->h_flags + 2 * flag_slot, C.err.p, 8, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));  // `items` lives on this stack frame
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->stats.launches += launches + 1;
  return RTM_OK;
}

// Device view of a caller array: the pointer itself, or a staged copy.
struct View {
  DevBuf buf;
  float *d = nullptr;
  bool staged = false;
};

static int view_in(rtm_ctx *ctx, View &v, const float *p, size_t bytes, cudaStream_t st) {
  if (is_device_ptr(p)) {
    v.d = const_cast<float *>(p);
    return RTM_OK;
  }
  CU(v.buf.alloc(ctx, bytes, st));
  CU(cudaMemcpyAsync(v.buf.p, p, bytes, cudaMemcpyHostToDevice, st));
  v.d = v.buf.as<float>();
  v.staged = true;
  return RTM_OK;
}

static int view_out(rtm_ctx *ctx, View &v, float *p, size_t bytes, cudaStream_t st) {
  if (is_device_ptr(p)) {
    v.d = p;
    return RTM_OK;
  }
  CU(v.buf.alloc(ctx, bytes, st));
  v.d = v.buf.as<float>();
  v.staged = true;
  return RTM_OK;
}

static int view_finish(rtm_ctx *ctx, View &v, float *p, size_t bytes, cudaStream_t st) {
  if (!v.staged) return RTM_OK;
  CU(cudaMemcpyAsync(p, v.d, bytes, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return RTM_OK;
}

static int late_begin(rtm_ctx *ctx, LateCopy &l, const void *src, void *dst, size_t shot_bytes,
                      cudaStream_t st) {
  l.src = src;
  l.dst = dst;
  l.shot_bytes = shot_bytes;
  CU(cudaStreamCreateWithFlags(&l.cs, cudaStreamNonBlocking));
  CU(cudaEventCreateWithFlags(&l.alloc_done, cudaEventDisableTiming));
  CU(cudaEventRecord(l.alloc_done, st));
  return RTM_OK;
}

// Waits on the host for whatever the upload issued (on every path, so the
// staging buffer is never released under a copy in flight; on success the
// copies ended before the backward phases that waited for them), then
// releases the stream and events.
static void late_end(LateCopy &l) {
  if (l.issued) cudaStreamSynchronize(l.cs);
  for (cudaEvent_t e : l.ready) cudaEventDestroy(e);
  if (l.alloc_done) cudaEventDestroy(l.alloc_done);
  if (l.cs) cudaStreamDestroy(l.cs);
  l = LateCopy{};
}

static int set_device(rtm_ctx *ctx) {
  CU(cudaSetDevice(ctx->device));
  return RTM_OK;
}

// A call that synchronised its stream reads its own flag slot.
static int own_wait_flag(rtm_ctx *ctx, int slot) {
  int line = 0;
  const int code = flag_take(ctx, slot, &line);
  return flag_status(ctx, code, line, "this call");
}

}  // namespace rtm

using namespace rtm;

// ------------------------------------------------------------------ ABI --

extern "C" {

double rtm_cfl_limit(void) { return 2.0 / std::sqrt(2.0 * 2048.0 / 315.0); }

int rtm_ctx_create(rtm_ctx **out, int device, size_t hbm_budget_bytes) {
  if (!out) return RTM_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return RTM_ERR_ARG;
  }
  rtm_ctx *ctx = new rtm_ctx();
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return RTM_ERR_CUDA;
  }
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    delete ctx;
    return RTM_ERR_CUDA;
  }
  ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.85 * (double)fr);
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess) {
    delete ctx;
    return RTM_ERR_CUDA;
  }
  uint64_t thr = UINT64_MAX;
  cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr);
  if (cudaMallocHost(&ctx->h_flags, 2 * kFlagSlots * sizeof(int)) != cudaSuccess) {
    cudaMemPoolDestroy(ctx->pool);
    delete ctx;
    return RTM_ERR_CUDA;
  }
  for (int i = kFlagSlots - 1; i >= 0; --i) {
    ctx->h_flags[2 * i] = ctx->h_flags[2 * i + 1] = 0;
    ctx->free_flags.push_back(i);
  }
  // RTM_STEP_KERNEL picks the context's default propagation kernel: 1 the
  // single-step kernel, 2 (default) the two-step kernel with one tile per
  // block (RTM_L2_AHEAD=1 turns on its L2 prefetch of later tiles), 3 the
  // persistent two-step kernel (RTM_TILE_Z=16 for 16-row tiles), 4 the
  // two-step kernel with v^{n+1} over v^n (RTM_TILE_Z=32 for 32-row tiles)
  const char *sk = std::getenv("RTM_STEP_KERNEL");
  const int k = sk ? std::atoi(sk) : 0;
  ctx->defaults.step_kernel = (k >= 1 && k <= 4) ? k : 2;
  const char *tz = std::getenv("RTM_TILE_Z");
  const int z = tz ? std::atoi(tz) : 24;
  ctx->defaults.tile_z = ((z == 16 && k == 3) || (z == 32 && k == 4)) ? z : 24;
  const char *la = std::getenv("RTM_L2_AHEAD");
  ctx->defaults.l2_ahead = (la && la[0] == '1') ? 1 : 0;
  // RTM_IMAGE_INPUT=1: backward launches image their input field where they can
  const char *ii = std::getenv("RTM_IMAGE_INPUT");
  ctx->defaults.image_input = (ii && ii[0] == '1') ? 1 : 0;
  // RTM_PDL=1: the kernel-4 launches are programmatic dependents of the previous one
  const char *pd = std::getenv("RTM_PDL");
  ctx->defaults.pdl = (pd && pd[0] == '1') ? 1 : 0;
  // RTM_GRAPHS=1 captures each phase of a batch in a CUDA graph by default
  const char *gr = std::getenv("RTM_GRAPHS");
  ctx->defaults.graph = (gr && gr[0] == '1') ? 1 : 0;
  *out = ctx;
  return RTM_OK;
}

int rtm_ctx_destroy(rtm_ctx *ctx) {
  if (!ctx) return RTM_OK;
  cudaSetDevice(ctx->device);
  // requests still running after the shutdown bound keep using the context:
  // leave it alive (the caller may try again) rather than free it under them
  if (!rtm_server_shutdown(ctx))
    return fail(ctx, RTM_ERR_BUSY, "requests are still running; the context was not destroyed");
  cudaDeviceSynchronize();
  {
    std::lock_guard<std::mutex> lk(ctx->flag_mu);
    for (auto &p : ctx->pending) cudaEventDestroy(p.ev);
    ctx->pending.clear();
  }
  for (cudaStream_t s : ctx->free_streams) cudaStreamDestroy(s);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
  delete ctx;
  return RTM_OK;
}

int rtm_ctx_set_batch(rtm_ctx *ctx, int max_items) {
  if (!ctx) return RTM_ERR_ARG;
  if (max_items < 0) return fail(ctx, RTM_ERR_ARG, "max_items must be >= 0");
  ctx->max_batch = max_items;
  return RTM_OK;
}

int rtm_autotune(rtm_ctx *ctx, const rtm_grid *grid, const rtm_acq *acq, const rtm_opts *opts,
                 int trial_steps, int *choice, void *stream) {
  if (!ctx) return RTM_ERR_ARG;
  int rc;
  if ((rc = check_grid(ctx, grid)) || (rc = check_acq(ctx, grid, acq, true)) ||
      (rc = check_opts(ctx, opts)))
    return rc;
  if ((rc = set_device(ctx)) || (rc = check_wait_flag(ctx))) return rc;
  // trials run on a private stream (capturable), after the caller's work
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
    return fail(ctx, RTM_ERR_CUDA, "could not synchronise the caller's stream");
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
    return fail(ctx, RTM_ERR_CUDA, "could not create a stream for the trials");
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  };
  StreamGuard guard{st};
  // trial: the same grid and acquisition over fewer steps, synthetic inputs
  rtm_grid tg = *grid;
  tg.nt = trial_steps > 0 ? trial_steps : 64;
  tg.nt = std::max(2, std::min(tg.nt, grid->nt));
  rtm_opts to = *opts;
  const long long nitems = acq->nshot;
  const MigrationPlan plan = plan_migration(tg, *acq, to, 1);
  const size_t vbytes = (size_t)grid->nx * grid->nz * 4;
  const size_t sbytes = (size_t)acq->nshot * tg.nt * acq->nrec * 4;
  const size_t io = 2 * vbytes + sbytes;
  const size_t need1 = plan.shared_bytes + plan.item_bytes + io;
  const size_t want = plan.shared_bytes + io + (size_t)nitems * plan.item_bytes;
  if (need1 > ctx->budget) return fail(ctx, RTM_ERR_NOMEM, "trial does not fit the budget");
  const size_t got = reserve_wait(ctx, want, need1, 600000);
  if (!got) return fail(ctx, RTM_ERR_TIMEOUT, "waited 600 s for device memory");
  const long long bmax = std::max<long long>(
      1, std::min<long long>(nitems, (long long)((got - plan.shared_bytes - io) / plan.item_bytes)));
  DevBuf vel, seis, img;
  int best = -1;
  double best_t = 1e300;
  std::vector<RunConfig> cand;
  // (kernel, tile height, L2 prefetch of later tiles): one tile per block
  // without and with the prefetch, one tile per block with v^{n+1} over v^n
  // (24 and 32 rows), persistent (24 and 16 rows), single step
  const int kinds[7][3] = {{2, 24, 0}, {2, 24, 1}, {4, 24, 0}, {4, 32, 0},
                           {3, 24, 0}, {3, 16, 0}, {1, 24, 0}};
  for (const auto &kd : kinds)
    for (int graph : {0, 1})
      for (long long items : {bmax, (bmax + 1) / 2}) {
        RunConfig c;
        c.step_kernel = kd[0];
        c.tile_z = kd[1];
        c.l2_ahead = kd[2];
        c.graph = graph;
        c.max_items = items >= nitems ? 0 : (int)items;
        bool dup = false;
        for (auto &o : cand)
          dup |= o.step_kernel == c.step_kernel && o.tile_z == c.tile_z &&
                 o.l2_ahead == c.l2_ahead && o.graph == c.graph && o.max_items == c.max_items;
        if (!dup) cand.push_back(c);
      }
  rc = RTM_OK;
  do {
    if ((rc = vel.alloc(ctx, vbytes, st)) || (rc = seis.alloc(ctx, sbytes, st)) ||
        (rc = img.alloc(ctx, vbytes, st))) {
      rc = fail(ctx, RTM_ERR_CUDA, "trial buffers");
      break;
    }
    // constant velocity at half the stability limit; zero data
    const double vt = 0.5 * 2.0 /
                      (grid->dt * std::sqrt((1.0 / (grid->dx * grid->dx) + 1.0 / (grid->dz * grid->dz)) *
                                            2048.0 / 315.0));
    std::vector<float> hv((size_t)grid->nx * grid->nz, (float)vt);
    if (cudaMemcpyAsync(vel.p, hv.data(), vbytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(seis.p, 0, sbytes, st) != cudaSuccess) {
      rc = fail(ctx, RTM_ERR_CUDA, "trial inputs");
      break;
    }
    struct Pair {  // trial timing events, released on every path
      cudaEvent_t a = nullptr, b = nullptr;
      ~Pair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
      }
    } ev2;
    if (cudaEventCreate(&ev2.a) != cudaSuccess || cudaEventCreate(&ev2.b) != cudaSuccess) {
      rc = fail(ctx, RTM_ERR_CUDA, "trial events");
      break;
    }
    const cudaEvent_t e0 = ev2.a, e1 = ev2.b;
    for (size_t i = 0; i < cand.size() && !rc; ++i) {
      const RunConfig &c = cand[i];
      const long long cap = c.max_items > 0 ? c.max_items : bmax;
      const long long nbatch = (nitems + cap - 1) / cap;
      const int B = (int)((nitems + nbatch - 1) / nbatch);
      float ms = 0.f, best_ms = 1e30f;
      for (int rep = 0; rep < 3 && !rc; ++rep) {  // first run warms up
        const int slot = flag_acquire(ctx);
        cudaEventRecord(e0, st);
        rc = migrate_device(ctx, tg, 1, vel.as<float>(), *acq, seis.as<float>(), to,
                            img.as<float>(), B, st, c, nullptr, nullptr, nullptr, slot);
        cudaEventRecord(e1, st);
        if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(ctx, RTM_ERR_CUDA, "trial sync");
        if (rc) {
          flag_defer(ctx, slot, st);
        } else {
          rc = own_wait_flag(ctx, slot);
        }
        if (!rc && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
          best_ms = std::min(best_ms, ms);
      }
      if (!rc && best_ms < best_t) {
        best_t = best_ms;
        best = (int)i;
      }
    }
  } while (0);
  vel.release();
  seis.release();
  img.release();
  if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(ctx, RTM_ERR_CUDA, "sync");
  unreserve(ctx, got);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->tuned[TuneKey{grid->nx, grid->nz, grid->nb, grid->nt, opts->isnap, opts->snap_dtype}] = cand[best];
  }
  if (choice) {
    choice[0] = cand[best].step_kernel;
    choice[1] = cand[best].max_items;
    choice[2] = cand[best].graph;
    choice[3] = cand[best].tile_z;
    choice[4] = cand[best].l2_ahead;
  }
  return RTM_OK;
}

int rtm_selftest_wait(rtm_ctx *ctx, int wait_ms, int *raised, void *stream) {
  if (!ctx || !raised || wait_ms < 1 || wait_ms > 10000) return RTM_ERR_ARG;
  int rc;
  if ((rc = set_device(ctx))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf f;
  CU(f.alloc(ctx, 16, st));
  CU(cudaMemsetAsync(f.p, 0, 16, st));
  CU(launch_wait_probe(f.as<int>(), (unsigned long long)wait_ms * 1000000ull, st));
  int h = 0;
  CU(cudaMemcpyAsync(&h, f.p, 4, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  *raised = h;
  return RTM_OK;
}

int rtm_ctx_inject_wait_timeout(rtm_ctx *ctx, int count) {
  if (!ctx || count < 0) return RTM_ERR_ARG;
  ctx->inject_timeouts.store(count);
  return RTM_OK;
}

int rtm_plan_bytes(const rtm_grid *grid, const rtm_acq *acq, const rtm_opts *opts, int nsample,
                   size_t *call_bytes, size_t *item_bytes) {
  if (!call_bytes || !item_bytes || nsample < 1) return RTM_ERR_ARG;
  int rc;
  if ((rc = check_grid(nullptr, grid)) || (rc = check_acq(nullptr, grid, acq, true)) ||
      (rc = check_opts(nullptr, opts)))
    return rc;
  const MigrationPlan p = plan_migration(*grid, *acq, *opts, nsample);
  *call_bytes = p.shared_bytes;
  *item_bytes = p.item_bytes;
  return RTM_OK;
}

int rtm_ctx_set_profiling(rtm_ctx *ctx, int on) {
  if (!ctx) return RTM_ERR_ARG;
  ctx->prof = on != 0;
  return RTM_OK;
}

int rtm_ctx_stats(rtm_ctx *ctx, rtm_stats *out, int reset) {
  if (!ctx || !out) return RTM_ERR_ARG;
  long long peak = 0, backfilled = 0;
  rtm_server_counters(ctx, reset != 0, &peak, &backfilled);
  std::lock_guard<std::mutex> lk(ctx->mu);
  *out = ctx->stats;
  out->requests_peak_running = peak;
  out->requests_backfilled = backfilled;
  if (reset) ctx->stats = rtm_stats{};
  return RTM_OK;
}

const char *rtm_last_error(rtm_ctx *ctx) { return ctx ? ctx->err : "no context"; }

int rtm_model(rtm_ctx *ctx, const rtm_grid *grid, const float *vel, const rtm_acq *acq, int shot,
              float *seis, void *stream) {
  if (!ctx) return RTM_ERR_ARG;
  int rc;
  if ((rc = check_grid(ctx, grid)) || (rc = check_acq(ctx, grid, acq, true))) return rc;
  if (!vel || !seis) return fail(ctx, RTM_ERR_ARG, "vel and seis must not be NULL");
  if (shot < -1 || shot >= acq->nshot)
    return fail(ctx, RTM_ERR_ARG, "shot %d outside [-1, %d)", shot, acq->nshot);
  if ((rc = set_device(ctx)) || (rc = check_wait_flag(ctx))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int s0 = shot < 0 ? 0 : shot, ns = shot < 0 ? acq->nshot : 1;
  const size_t vbytes = (size_t)grid->nx * grid->nz * 4;
  const size_t sbytes = (size_t)ns * grid->nt * acq->nrec * 4;
  const Geo g = make_geo(*grid);
  const size_t item = 3 * (size_t)g.plane * 4;
  const size_t io = (is_device_ptr(vel) ? 0 : vbytes) + (is_device_ptr(seis) ? 0 : sbytes);
  const size_t base = (size_t)g.plane * 4 + (size_t)(g.P + g.NZ) * 4 + (size_t)acq->nrec * 12 +
                      (size_t)acq->nshot * 16 + (size_t)grid->nt * 4 + (size_t)(g.ntx * g.ntz + 1) * 4 +
                      io + 4096;
  if (base + item > ctx->budget)
    return fail(ctx, RTM_ERR_NOMEM, "modelling needs %.3f GB, budget is %.3f GB", (base + item) / 1e9,
                ctx->budget / 1e9);
  size_t want = base + (size_t)ns * item;
  if (ctx->max_batch > 0) want = std::min(want, base + (size_t)ctx->max_batch * item);
  const size_t got = reserve_wait(ctx, want, base + item, 600000);
  if (!got) return fail(ctx, RTM_ERR_TIMEOUT, "waited 600 s for device memory");
  const int B = (int)std::max<size_t>(1, std::min<size_t>(ns, (got - base) / item));
  View v, s;
  const int slot = flag_acquire(ctx);
  rc = view_in(ctx, v, vel, vbytes, st);
  if (!rc) rc = check_velocity(ctx, *grid, v.d, (long long)grid->nx * grid->nz, st);
  if (!rc) rc = view_out(ctx, s, seis, sbytes, st);
  if (!rc) rc = model_device(ctx, *grid, v.d, *acq, s0, ns, s.d, B, st, slot);
  if (!rc) rc = view_finish(ctx, s, seis, sbytes, st);
  if (!rc)
    rc = own_wait_flag(ctx, slot);  // model_device synchronised its stream
  else
    flag_defer(ctx, slot, st);
  unreserve(ctx, got);
  return rc;
}

// raw: the stacked imaging numerator (no illumination normalisation, no
// filter), the adjoint of Born modelling.
// A call given the legacy default stream, whose launch configuration
// captures phases into graphs, runs on a context-owned stream instead: after
// the caller's earlier work on the legacy stream, and before its later work
// (events join the two).  The legacy stream cannot be captured.
struct CallStream {
  rtm_ctx *ctx = nullptr;
  cudaStream_t user = nullptr, st = nullptr;
  bool own = false;
  CallStream() = default;
  CallStream(const CallStream &) = delete;
  CallStream &operator=(const CallStream &) = delete;
  ~CallStream() { end(); }
  void begin(rtm_ctx *c, cudaStream_t u, bool graph) {
    ctx = c;
    user = st = u;
    if (!graph || (u != nullptr && u != cudaStreamLegacy)) return;
    cudaStream_t s = nullptr;
    {
      std::lock_guard<std::mutex> lk(ctx->stream_mu);
      if (!ctx->free_streams.empty()) {
        s = ctx->free_streams.back();
        ctx->free_streams.pop_back();
      }
    }
    if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
    if (!join(u, s)) {  // (stay on the caller's stream)
      park(s);
      return;
    }
    st = s;
    own = true;
  }
  void end() {
    if (!own) return;
    own = false;
    join(st, user);
    park(st);
  }

 private:
  static bool join(cudaStream_t from, cudaStream_t to) {  // `to` waits for `from`'s work so far
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return false;
    const bool ok = cudaEventRecord(ev, from) == cudaSuccess && cudaStreamWaitEvent(to, ev, 0) == cudaSuccess;
    cudaEventDestroy(ev);  // (released once it completes)
    return ok;
  }
  void park(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(ctx->stream_mu);
    ctx->free_streams.push_back(s);
  }
};

static int migrate_common(rtm_ctx *ctx, const rtm_grid *grid, int nsample, const float *vels,
                          const rtm_acq *acq, const float *seis, const rtm_opts *opts,
                          float *images, void *stream, bool raw = false) {
  if (!ctx) return RTM_ERR_ARG;
  CallTrace trace(raw ? "rtm_migrate_adjoint" : (nsample > 1 ? "rtm_migrate_ensemble" : "rtm_migrate"));
  int rc;
  if ((rc = check_grid(ctx, grid)) || (rc = check_acq(ctx, grid, acq, true)) ||
      (rc = check_opts(ctx, opts)))
    return rc;
  if (nsample < 1) return fail(ctx, RTM_ERR_ARG, "nsample must be >= 1");
  if (!vels || !seis || !images) return fail(ctx, RTM_ERR_ARG, "NULL array argument");
  if ((rc = set_device(ctx)) || (rc = check_wait_flag(ctx))) return rc;
  const size_t vbytes = (size_t)nsample * grid->nx * grid->nz * 4;
  const size_t sbytes = (size_t)acq->nshot * grid->nt * acq->nrec * 4;
  rtm_opts op = *opts;
  if (raw) {
    op.eps = -1.0;  // the stacking kernel adds num as it is
    op.laplacian = 0;
  }
  const MigrationPlan plan = plan_migration(*grid, *acq, op, nsample);
  const size_t io = (is_device_ptr(vels) ? 0 : vbytes) + (is_device_ptr(seis) ? 0 : sbytes) +
                    (is_device_ptr(images) ? 0 : vbytes);
  const size_t need1 = plan.shared_bytes + plan.item_bytes + io;
  const long long nitems = (long long)nsample * acq->nshot;
  const RunConfig cfg = config_for(ctx, *grid, op);
  CallStream cs;  // (declared before the staging buffers: their frees come before the join)
  cs.begin(ctx, (cudaStream_t)stream, cfg.graph != 0);
  const cudaStream_t st = cs.st;
  size_t want = plan.shared_bytes + io + (size_t)nitems * plan.item_bytes;
  const int cap = ctx->max_batch > 0 ? ctx->max_batch : cfg.max_items;
  if (cap > 0) want = std::min(want, plan.shared_bytes + io + (size_t)cap * plan.item_bytes);
  if (need1 > ctx->budget)
    return fail(ctx, RTM_ERR_NOMEM, "one migration needs %.3f GB, budget is %.3f GB",
                need1 / 1e9, ctx->budget / 1e9);
  const size_t got = reserve_wait(ctx, want, need1, 600000);
  if (!got) return fail(ctx, RTM_ERR_TIMEOUT, "waited 600 s for %.3f GB of the budget", need1 / 1e9);
  // items in flight: what the reservation holds, balanced over the batches
  long long bmax = std::max<long long>(
      1, std::min<long long>(nitems, (long long)((got - plan.shared_bytes - io) / plan.item_bytes)));
  const long long nbatch = (nitems + bmax - 1) / bmax;
  const int B = (int)((nitems + nbatch - 1) / nbatch);
  View v, s, im;
  LateCopy late;
  const int slot = flag_acquire(ctx);
  rc = view_in(ctx, v, vels, vbytes, st);
  if (!rc) rc = check_velocity(ctx, *grid, v.d, (long long)nsample * grid->nx * grid->nz, st);
  trace_mark("velocity staged and checked");
  // host seismograms: allocate now, upload behind the first forward phase
  if (!rc) rc = view_out(ctx, s, const_cast<float *>(seis), sbytes, st);
  if (!rc && s.staged)
    rc = late_begin(ctx, late, seis, s.d, (size_t)grid->nt * acq->nrec * 4, st);
  if (!rc) rc = view_out(ctx, im, images, vbytes, st);
  trace_mark("buffers ready");
  if (!rc)
    rc = migrate_device(ctx, *grid, nsample, v.d, *acq, s.d, op, im.d, B, st, cfg, nullptr,
                        nullptr, s.staged ? &late : nullptr, slot);
  trace_mark("migration enqueued");
  late_end(late);
  if (!rc) rc = view_finish(ctx, im, images, vbytes, st);
  trace_mark("image returned");
  if (!rc && (im.staged || ctx->prof))
    rc = own_wait_flag(ctx, slot);  // the stream was synchronised
  else
    flag_defer(ctx, slot, st);
  unreserve(ctx, got);
  return rc;
}

int rtm_migrate(rtm_ctx *ctx, const rtm_grid *grid, const float *vel, const rtm_acq *acq,
                const float *seis, const rtm_opts *opts, float *image, void *stream) {
  return migrate_common(ctx, grid, 1, vel, acq, seis, opts, image, stream);
}

int rtm_migrate_ensemble(rtm_ctx *ctx, const rtm_grid *grid, int nsample, const float *vels,
                         const rtm_acq *acq, const float *seis, const rtm_opts *opts,
                         float *images, void *stream) {
  return migrate_common(ctx, grid, nsample, vels, acq, seis, opts, images, stream);
}

int rtm_migrate_adjoint(rtm_ctx *ctx, const rtm_grid *grid, const float *vel,
                        const rtm_acq *acq, const float *seis, const rtm_opts *opts, float *image,
                        void *stream) {
  return migrate_common(ctx, grid, 1, vel, acq, seis, opts, image, stream, true);
}

int rtm_born(rtm_ctx *ctx, const rtm_grid *grid, const float *vel, const rtm_acq *acq,
             const float *refl, const rtm_opts *opts, float *seis, void *stream) {
  if (!ctx) return RTM_ERR_ARG;
  int rc;
  if ((rc = check_grid(ctx, grid)) || (rc = check_acq(ctx, grid, acq, true)) ||
      (rc = check_opts(ctx, opts)))
    return rc;
  if (!vel || !refl || !seis) return fail(ctx, RTM_ERR_ARG, "NULL array argument");
  if (opts->checkpoint)
    return fail(ctx, RTM_ERR_ARG, "Born modelling keeps every snapshot (checkpoint must be 0)");
  if ((rc = set_device(ctx)) || (rc = check_wait_flag(ctx))) return rc;
  const size_t vbytes = (size_t)grid->nx * grid->nz * 4;
  const size_t sbytes = (size_t)acq->nshot * grid->nt * acq->nrec * 4;
  const MigrationPlan plan = plan_migration(*grid, *acq, *opts, 1);
  const size_t io = (is_device_ptr(vel) ? 0 : vbytes) + (is_device_ptr(refl) ? 0 : vbytes) +
                    (is_device_ptr(seis) ? 0 : sbytes);
  const size_t need1 = plan.shared_bytes + plan.item_bytes + io;
  const RunConfig cfg = config_for(ctx, *grid, *opts);
  CallStream cs;  // (declared before the staging buffers: their frees come before the join)
  cs.begin(ctx, (cudaStream_t)stream, cfg.graph != 0);
  const cudaStream_t st = cs.st;
  size_t want = plan.shared_bytes + io + (size_t)acq->nshot * plan.item_bytes;
  const int cap = ctx->max_batch > 0 ? ctx->max_batch : cfg.max_items;
  if (cap > 0) want = std::min(want, plan.shared_bytes + io + (size_t)cap * plan.item_bytes);
  if (need1 > ctx->budget)
    return fail(ctx, RTM_ERR_NOMEM, "one Born modelling needs %.3f GB, budget is %.3f GB",
                need1 / 1e9, ctx->budget / 1e9);
  const size_t got = reserve_wait(ctx, want, need1, 600000);
  if (!got) return fail(ctx, RTM_ERR_TIMEOUT, "waited 600 s for %.3f GB of the budget", need1 / 1e9);
  const long long nitems = acq->nshot;
  long long bmax = std::max<long long>(
      1, std::min<long long>(nitems, (long long)((got - plan.shared_bytes - io) / plan.item_bytes)));
  const long long nbatch = (nitems + bmax - 1) / bmax;
  const int B = (int)((nitems + nbatch - 1) / nbatch);
  View v, m, out;
  const int slot = flag_acquire(ctx);
  rc = view_in(ctx, v, vel, vbytes, st);
  if (!rc) rc = check_velocity(ctx, *grid, v.d, (long long)grid->nx * grid->nz, st);
  if (!rc) rc = view_in(ctx, m, refl, vbytes, st);
  if (!rc) rc = view_out(ctx, out, seis, sbytes, st);
  if (!rc)
    rc = migrate_device(ctx, *grid, 1, v.d, *acq, nullptr, *opts, nullptr, B, st, cfg, m.d,
                        out.d, nullptr, slot);
  if (!rc) rc = view_finish(ctx, out, seis, sbytes, st);
  if (!rc && (out.staged || ctx->prof))
    rc = own_wait_flag(ctx, slot);
  else
    flag_defer(ctx, slot, st);
  unreserve(ctx, got);
  return rc;
}

int rtm_ensemble_stats(rtm_ctx *ctx, const float *images, int n, long npix, double *mean,
                       double *std_, float *q05, float *q95, void *stream) {
  if (!ctx) return RTM_ERR_ARG;
  if (!images || !mean || !std_ || !q05 || !q95) return fail(ctx, RTM_ERR_ARG, "NULL array argument");
  if (n < 1 || n > ens_stats_max_n() || npix < 1)
    return fail(ctx, RTM_ERR_ARG, "need 1 <= n <= %d and npix >= 1 (n=%d npix=%ld)",
                ens_stats_max_n(), n, npix);
  int rc;
  if ((rc = set_device(ctx))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = is_device_ptr(images) && is_device_ptr(mean) && is_device_ptr(std_) &&
                   is_device_ptr(q05) && is_device_ptr(q95);
  if (dev) {
    CU(launch_ens_stats(images, n, npix, mean, std_, q05, q95, st));
    return RTM_OK;
  }
  DevBuf bi, bm, bs, b5, b9;
  CU(bi.alloc(ctx, (size_t)n * npix * 4, st));
  CU(bm.alloc(ctx, (size_t)npix * 8, st));
  CU(bs.alloc(ctx, (size_t)npix * 8, st));
  CU(b5.alloc(ctx, (size_t)npix * 4, st));
  CU(b9.alloc(ctx, (size_t)npix * 4, st));
  CU(cudaMemcpyAsync(bi.p, images, bi.bytes, cudaMemcpyDefault, st));
  CU(launch_ens_stats(bi.as<float>(), n, npix, bm.as<double>(), bs.as<double>(), b5.as<float>(),
                      b9.as<float>(), st));
  CU(cudaMemcpyAsync(mean, bm.p, bm.bytes, cudaMemcpyDefault, st));
  CU(cudaMemcpyAsync(std_, bs.p, bs.bytes, cudaMemcpyDefault, st));
  CU(cudaMemcpyAsync(q05, b5.p, b5.bytes, cudaMemcpyDefault, st));
  CU(cudaMemcpyAsync(q95, b9.p, b9.bytes, cudaMemcpyDefault, st));
  CU(cudaStreamSynchronize(st));
  return RTM_OK;
}

int rtm_uncertainty_maps(rtm_ctx *ctx, const double *mean, const double *std_, long npix,
                         double *conf, double *ratio, void *stream) {
  if (!ctx) return RTM_ERR_ARG;
  if (!mean || !std_ || !conf || !ratio || npix < 1) return fail(ctx, RTM_ERR_ARG, "bad arguments");
  int rc;
  if ((rc = set_device(ctx))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf scratch;
  CU(scratch.alloc(ctx, 16, st));
  const bool dev = is_device_ptr(mean) && is_device_ptr(std_) && is_device_ptr(conf) &&
                   is_device_ptr(ratio);
  if (dev) {
    CU(launch_unc_maps(mean, std_, npix, conf, ratio, scratch.as<unsigned long long>(), st));
    return RTM_OK;
  }
  DevBuf bm, bs, bc, br;
  CU(bm.alloc(ctx, (size_t)npix * 8, st));
  CU(bs.alloc(ctx, (size_t)npix * 8, st));
  CU(bc.alloc(ctx, (size_t)npix * 8, st));
  CU(br.alloc(ctx, (size_t)npix * 8, st));
  CU(cudaMemcpyAsync(bm.p, mean, bm.bytes, cudaMemcpyDefault, st));
  CU(cudaMemcpyAsync(bs.p, std_, bs.bytes, cudaMemcpyDefault, st));
  CU(launch_unc_maps(bm.as<double>(), bs.as<double>(), npix, bc.as<double>(), br.as<double>(),
                     scratch.as<unsigned long long>(), st));
  CU(cudaMemcpyAsync(conf, bc.p, bc.bytes, cudaMemcpyDefault, st));
  CU(cudaMemcpyAsync(ratio, br.p, br.bytes, cudaMemcpyDefault, st));
  CU(cudaStreamSynchronize(st));
  return RTM_OK;
}

int rtm_submit(rtm_ctx *ctx, const rtm_request *req, uint64_t *ticket) {
  if (!ctx) return RTM_ERR_ARG;
  return rtm_server_submit(ctx, req, ticket);
}

int rtm_poll(rtm_ctx *ctx, uint64_t ticket, int *state, int timeout_ms) {
  if (!ctx) return RTM_ERR_ARG;
  return rtm_server_poll(ctx, ticket, state, timeout_ms);
}

}  // extern "C"
