// rtm_eikonal.cu — first-arrival traveltimes on the device: the forward
// operator of the tomography stage (§2.1 Eq. 1: traveltimes from the eikonal
// equation |grad T| = 1/v; §3: one solve per source for every proposed
// velocity model, which dominates that stage's cost).
//
// Discretisation: the first-order upwind scheme on an nz x nx grid (spacings
// dz, dx): with a, b the smaller vertical and horizontal neighbour times,
//     ((T - a)^+ / dz)^2 + ((T - b)^+ / dx)^2 = s^2,  s = 1/v,
// and T = 0 at the source node.  Its discrete solution is unique; fast
// marching reaches it in one ordered pass, and Gauss-Seidel sweeps in the four
// diagonal directions reach it by iterating to a fixed point (Zhao 2005).
//
// The solver sweeps level by level: in the sweep towards (+z, +x) the nodes
// with i + j = l depend only on level l - 1 (already updated in this sweep)
// and on level l + 1 (from the previous sweep), exactly as in the sequential
// row-by-row sweep, so each level is updated in parallel and the result is
// that of the sequential sweep (Detrixhe, Gibou and Min 2013).  One CTA solves
// one (velocity sample, source) problem: its traveltime field lives in shared
// memory when it fits (about 56 K nodes), else in an L2-resident buffer.
// Iterations (four sweeps each) stop when one changes no node, or at a cap.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "rtm_engine.h"
#include "rtm_launch.h"

namespace {

using u32 = uint32_t;
constexpr float kInf = __builtin_huge_valf();

struct EikArgs {
  const float *slow;     // [nsample][nz][nx] slowness (s/m)
  int nz, nx, nsrc, nrec;
  float dz, dx, wz, wx, wsum, wprod, inv_wsum;  // spacings, 1/dz^2, 1/dx^2, sum, product, 1/sum
  const int *src;        // [nsrc][2] (iz, ix)
  const int *rec;        // [nrec][2]
  float *times;          // [nsample][nsrc][nrec] or null
  float *fields;         // [nsample][nsrc][nz][nx]: output, and the work field off-chip
  int max_iter;
  int *iters;            // [nsample * nsrc] iterations to the fixed point, -1 at the cap
};

// The upwind update from the smaller vertical (a) and horizontal (b)
// neighbour times: one-sided from the smaller one if that does not exceed
// the other, else the larger root of the two-term quadratic.  The root takes
// the hardware reciprocal square root and a multiply by 1/(wz + wx): a few
// ulps per update, far inside the FP32 error of a path of updates.
__device__ __forceinline__ float update(float a, float b, float s, const EikArgs &A) {
  const bool vz = a <= b;
  const float u1 = vz ? a : b, u2 = vz ? b : a;
  const float h1 = vz ? A.dz : A.dx, w1 = vz ? A.wz : A.wx, w2 = vz ? A.wx : A.wz;
  const float t1 = u1 + s * h1;
  if (t1 <= u2) return t1;  // also both neighbours unknown: inf
  const float d = u1 - u2;
  const float disc = fmaxf(A.wsum * (s * s) - A.wprod * (d * d), 1e-30f);
  return (w1 * u1 + w2 * u2 + disc * rsqrtf(disc)) * A.inv_wsum;
}

// One tile of TZ x TX nodes, updated in the sweep's order by one thread: the
// tile and its halo are loaded into registers, the nodes are updated one
// after the other, and the changed values are stored.  Tiles on one tile
// diagonal run in parallel; every node sees each neighbour in the same state
// (updated in this sweep, or from the previous one) as in the sequential
// sweep, so the result is the sequential sweep's, bit for bit.
template <int TZ, int TX, bool FZ, bool FX>
__device__ __forceinline__ bool sweep_tile(float *T, const float *s, int i0, int j0, int nz, int nx,
                                           const EikArgs &A) {
  float t[TZ][TX], sl[TZ][TX], up[TX], dn[TX], lf[TZ], rt[TZ];
#pragma unroll
  for (int r = 0; r < TZ; ++r) {
    const int i = i0 + r;
#pragma unroll
    for (int c = 0; c < TX; ++c) {
      const int j = j0 + c;
      const bool in = i < nz && j < nx;
      const long long k = (long long)i * nx + j;
      t[r][c] = in ? T[k] : kInf;
      sl[r][c] = in ? __ldg(s + k) : 0.f;
    }
    lf[r] = i < nz && j0 > 0 ? T[(long long)i * nx + j0 - 1] : kInf;
    rt[r] = i < nz && j0 + TX < nx ? T[(long long)i * nx + j0 + TX] : kInf;
  }
#pragma unroll
  for (int c = 0; c < TX; ++c) {
    const int j = j0 + c;
    up[c] = j < nx && i0 > 0 ? T[(long long)(i0 - 1) * nx + j] : kInf;
    dn[c] = j < nx && i0 + TZ < nz ? T[(long long)(i0 + TZ) * nx + j] : kInf;
  }
  u32 changed = 0;
#pragma unroll
  for (int rr = 0; rr < TZ; ++rr) {
    const int r = FZ ? rr : TZ - 1 - rr;
#pragma unroll
    for (int cc = 0; cc < TX; ++cc) {
      const int c = FX ? cc : TX - 1 - cc;
      if (i0 + r >= nz || j0 + c >= nx) continue;  // outside the grid: stays infinite
      const float a = fminf(r > 0 ? t[r - 1][c] : up[c], r < TZ - 1 ? t[r + 1][c] : dn[c]);
      const float b = fminf(c > 0 ? t[r][c - 1] : lf[r], c < TX - 1 ? t[r][c + 1] : rt[r]);
      const float v = update(a, b, sl[r][c], A);
      if (v < t[r][c]) {
        t[r][c] = v;
        changed |= 1u << (r * TX + c);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < TZ; ++r)
#pragma unroll
    for (int c = 0; c < TX; ++c)
      if ((changed >> (r * TX + c)) & 1u) T[(long long)(i0 + r) * nx + j0 + c] = t[r][c];
  return changed != 0;
}

template <int TZ, int TX, bool FZ, bool FX>
__device__ __forceinline__ int sweep(float *T, const float *s, const EikArgs &A) {
  const int nz = A.nz, nx = A.nx;
  const int ntz = (nz + TZ - 1) / TZ, ntx = (nx + TX - 1) / TX;
  int changed = 0;
  for (int l = 0; l < ntz + ntx - 1; ++l) {
    const int lo = max(0, l - (ntx - 1)), hi = min(ntz - 1, l);
    for (int ip = lo + (int)threadIdx.x; ip <= hi; ip += blockDim.x) {
      const int jp = l - ip;
      const int ti = FZ ? ip : ntz - 1 - ip, tj = FX ? jp : ntx - 1 - jp;
      changed |= sweep_tile<TZ, TX, FZ, FX>(T, s, ti * TZ, tj * TX, nz, nx, A);
    }
    __syncthreads();
  }
  return changed;
}

template <int TZ, int TX, bool RESIDENT>
__global__ void __launch_bounds__(256, 4) k_eik_sweep(const __grid_constant__ EikArgs A) {
  extern __shared__ float s_T[];
  const int p = blockIdx.x;  // sample * nsrc + source
  const int sample = p / A.nsrc, src = p % A.nsrc;
  const int nz = A.nz, nx = A.nx;
  const long long N = (long long)nz * nx;
  const float *s = A.slow + (long long)sample * N;
  float *T = RESIDENT ? s_T : A.fields + (long long)p * N;
  for (long long k = threadIdx.x; k < N; k += blockDim.x) T[k] = kInf;
  __syncthreads();
  if (threadIdx.x == 0) T[(long long)A.src[2 * src] * nx + A.src[2 * src + 1]] = 0.0f;
  __syncthreads();
  int it = 0;
  bool converged = false;
  for (; it < A.max_iter; ++it) {
    // the four diagonal directions: (+z, +x), (+z, -x), (-z, -x), (-z, +x)
    int changed = sweep<TZ, TX, true, true>(T, s, A);
    changed |= sweep<TZ, TX, true, false>(T, s, A);
    changed |= sweep<TZ, TX, false, false>(T, s, A);
    changed |= sweep<TZ, TX, false, true>(T, s, A);
    if (!__syncthreads_or(changed)) {
      converged = true;
      break;
    }
  }
  if (threadIdx.x == 0) A.iters[p] = converged ? it + 1 : -1;
  if (A.times) {
    float *out = A.times + (long long)p * A.nrec;
    for (int r = threadIdx.x; r < A.nrec; r += blockDim.x)
      out[r] = T[(long long)A.rec[2 * r] * nx + A.rec[2 * r + 1]];
  }
  if (RESIDENT && A.fields) {
    float *out = A.fields + (long long)p * N;
    for (long long k = threadIdx.x; k < N; k += blockDim.x) out[k] = T[k];
  }
}

__global__ void k_eik_slowness(const float *vel, long long n, float *slow) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    slow[k] = __frcp_rn(vel[k]);
}

}  // namespace

namespace rtm {

// Largest field kept in shared memory (bytes).
size_t eik_resident_limit() {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return (size_t)std::max(0, optin - 1024);
}

cudaError_t launch_eikonal(const float *slow, int nsample, int nz, int nx, double dz, double dx,
                           int nsrc, const int *src, int nrec, const int *rec, int max_iter,
                           float *times, float *fields, int *iters, bool resident,
                           cudaStream_t st) {
  EikArgs A{};
  A.slow = slow;
  A.nz = nz;
  A.nx = nx;
  A.nsrc = nsrc;
  A.nrec = nrec;
  A.dz = (float)dz;
  A.dx = (float)dx;
  A.wz = (float)(1.0 / (dz * dz));
  A.wx = (float)(1.0 / (dx * dx));
  A.wsum = (float)(1.0 / (dz * dz) + 1.0 / (dx * dx));
  A.wprod = (float)(1.0 / (dz * dz * dx * dx));
  A.inv_wsum = (float)(1.0 / (1.0 / (dz * dz) + 1.0 / (dx * dx)));
  A.src = src;
  A.rec = rec;
  A.times = times;
  A.fields = fields;
  A.max_iter = max_iter;
  A.iters = iters;
  const long long problems = (long long)nsample * nsrc;
  if (problems > 0x7fffffffll) return cudaErrorInvalidValue;
  // tile shape: 2 x 2 (a short chain of dependent updates per thread, half
  // the diagonals of single nodes); RTM_EIK_TILE=TZxTX overrides it (one of
  // 1x1 2x2 2x4 4x2), for measurements
  const int shapes[4][2] = {{2, 2}, {1, 1}, {2, 4}, {4, 2}};
  int best = 0;
  if (const char *env = getenv("RTM_EIK_TILE")) {
    for (int q = 0; q < 4; ++q) {
      char name[8];
      snprintf(name, sizeof name, "%dx%d", shapes[q][0], shapes[q][1]);
      if (!strcmp(env, name)) best = q;
    }
  }
  const int tz = shapes[best][0], tx = shapes[best][1];
  const int level = std::min((nz + tz - 1) / tz, (nx + tx - 1) / tx);  // tiles per diagonal
  const int threads = std::min(256, std::max(32, (level + 31) / 32 * 32));
  const size_t smem = resident ? (size_t)nz * nx * 4 : 0;
  auto go = [&](auto kernel) -> cudaError_t {
    if (resident) {
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
    }
    kernel<<<(unsigned)problems, threads, smem, st>>>(A);
    return cudaGetLastError();
  };
  switch (best) {
    case 1: return resident ? go(k_eik_sweep<1, 1, true>) : go(k_eik_sweep<1, 1, false>);
    case 2: return resident ? go(k_eik_sweep<2, 4, true>) : go(k_eik_sweep<2, 4, false>);
    case 3: return resident ? go(k_eik_sweep<4, 2, true>) : go(k_eik_sweep<4, 2, false>);
    default: return resident ? go(k_eik_sweep<2, 2, true>) : go(k_eik_sweep<2, 2, false>);
  }
}

cudaError_t launch_eik_slowness(const float *vel, long long n, float *slow, cudaStream_t st) {
  const long long blocks = std::min<long long>((n + 255) / 256, 152 * 32);
  k_eik_slowness<<<(unsigned)std::max<long long>(1, blocks), 256, 0, st>>>(vel, n, slow);
  return cudaGetLastError();
}

}  // namespace rtm

// ------------------------------------------------------------------ ABI --

using namespace rtm;

#define EIK_CU(x)                                                                      \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) return fail(ctx, RTM_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

extern "C" int rtm_eikonal(rtm_ctx *ctx, int nz, int nx, double dz, double dx, int nsample,
                           const float *vel, int nsrc, const int *src_iz, const int *src_ix,
                           int nrec, const int *rec_iz, const int *rec_ix, int max_iter,
                           int flags, float *times, float *fields, int *iters, void *stream) {
  if (!ctx) return RTM_ERR_ARG;
  if (nz < 1 || nx < 1 || !(dz > 0) || !(dx > 0) || !std::isfinite(dz) || !std::isfinite(dx) ||
      nsample < 1 || nsrc < 1 || nrec < 0 || (nrec > 0 && (!rec_iz || !rec_ix)))
    return fail(ctx, RTM_ERR_ARG, "bad eikonal grid or acquisition arguments");
  if (!vel || !src_iz || !src_ix || (!times && !fields))
    return fail(ctx, RTM_ERR_ARG, "vel, sources and one of times / fields are required");
  if (nrec == 0 && times) return fail(ctx, RTM_ERR_ARG, "times needs receivers");
  if ((long long)nz * nx > (1ll << 31) / 4) return fail(ctx, RTM_ERR_ARG, "grid too large");
  for (int k = 0; k < nsrc; ++k)
    if (src_iz[k] < 0 || src_iz[k] >= nz || src_ix[k] < 0 || src_ix[k] >= nx)
      return fail(ctx, RTM_ERR_ARG, "source %d at (%d, %d) is outside the grid", k, src_iz[k],
                  src_ix[k]);
  for (int r = 0; r < nrec; ++r)
    if (rec_iz[r] < 0 || rec_iz[r] >= nz || rec_ix[r] < 0 || rec_ix[r] >= nx)
      return fail(ctx, RTM_ERR_ARG, "receiver %d at (%d, %d) is outside the grid", r, rec_iz[r],
                  rec_ix[r]);
  if (max_iter <= 0) max_iter = 64;
  if ((flags & ~(RTM_EIK_OFFCHIP | RTM_EIK_SHARED)) || flags == (RTM_EIK_OFFCHIP | RTM_EIK_SHARED))
    return fail(ctx, RTM_ERR_ARG, "bad flags %d", flags);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, RTM_ERR_CUDA, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const long long N = (long long)nz * nx, problems = (long long)nsample * nsrc;
  const size_t vbytes = (size_t)nsample * N * 4;
  DevBuf dvel, dslow, dtab, dtimes, dfields, diters, drng;
  const float *v = vel;
  if (!is_device_ptr(vel)) {
    EIK_CU(dvel.alloc(ctx, vbytes, st));
    EIK_CU(cudaMemcpyAsync(dvel.p, vel, vbytes, cudaMemcpyHostToDevice, st));
    v = dvel.as<float>();
  }
  // velocities must be positive and finite (one synchronisation)
  {
    EIK_CU(drng.alloc(ctx, 16, st));
    const unsigned init[4] = {0u, 0x7f7fffffu, 0u, 0u};
    EIK_CU(cudaMemcpyAsync(drng.p, init, 16, cudaMemcpyHostToDevice, st));
    EIK_CU(launch_vrange(v, (long long)nsample * N, drng.as<unsigned>(), st));
    unsigned out[4];
    EIK_CU(cudaMemcpyAsync(out, drng.p, 16, cudaMemcpyDeviceToHost, st));
    EIK_CU(cudaStreamSynchronize(st));
    if (out[2])
      return fail(ctx, RTM_ERR_ARG, "%u velocity values are non-positive or not finite", out[2]);
  }
  EIK_CU(dslow.alloc(ctx, vbytes, st));
  EIK_CU(launch_eik_slowness(v, (long long)nsample * N, dslow.as<float>(), st));
  std::vector<int> tab(2 * (size_t)(nsrc + nrec));
  for (int k = 0; k < nsrc; ++k) {
    tab[2 * k] = src_iz[k];
    tab[2 * k + 1] = src_ix[k];
  }
  for (int r = 0; r < nrec; ++r) {
    tab[2 * (nsrc + r)] = rec_iz[r];
    tab[2 * (nsrc + r) + 1] = rec_ix[r];
  }
  EIK_CU(dtab.alloc(ctx, tab.size() * 4, st));
  EIK_CU(cudaMemcpyAsync(dtab.p, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, st));
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const bool fits = (size_t)N * 4 <= eik_resident_limit();
  const bool resident = fits && !(flags & RTM_EIK_OFFCHIP) &&
                        ((flags & RTM_EIK_SHARED) || problems <= (long long)sms);
  const size_t tbytes = (size_t)problems * nrec * 4, fbytes = (size_t)problems * N * 4;
  float *dt = times;
  if (times && !is_device_ptr(times)) {
    EIK_CU(dtimes.alloc(ctx, tbytes, st));
    dt = dtimes.as<float>();
  }
  float *df = fields;
  if ((fields && !is_device_ptr(fields)) || (!fields && !resident)) {
    EIK_CU(dfields.alloc(ctx, fbytes, st));  // output staging, or the off-chip work fields
    df = dfields.as<float>();
  }
  EIK_CU(diters.alloc(ctx, (size_t)problems * 4, st));
  struct Timer {  // the solver's device time (profiling), released on every path
    cudaEvent_t a = nullptr, b = nullptr;
    ~Timer() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } tm;
  if (ctx->prof && cudaEventCreate(&tm.a) == cudaSuccess && cudaEventCreate(&tm.b) == cudaSuccess)
    cudaEventRecord(tm.a, st);
  const cudaEvent_t e0 = tm.b ? tm.a : nullptr, e1 = tm.b;
  EIK_CU(launch_eikonal(dslow.as<float>(), nsample, nz, nx, dz, dx, nsrc, dtab.as<int>(), nrec,
                        dtab.as<int>() + 2 * nsrc, max_iter, dt, df, diters.as<int>(), resident,
                        st));
  if (e1) cudaEventRecord(e1, st);
  std::vector<int> it((size_t)problems);
  EIK_CU(cudaMemcpyAsync(it.data(), diters.p, (size_t)problems * 4, cudaMemcpyDeviceToHost, st));
  if (times && dt != times) EIK_CU(cudaMemcpyAsync(times, dt, tbytes, cudaMemcpyDeviceToHost, st));
  if (fields && df != fields) EIK_CU(cudaMemcpyAsync(fields, df, fbytes, cudaMemcpyDeviceToHost, st));
  EIK_CU(cudaStreamSynchronize(st));
  long long sweeps = 0, stuck = 0;
  for (int x : it) {
    sweeps += x > 0 ? x : max_iter;
    stuck += x < 0;
  }
  {
    float ms = 0.f;
    if (e0 && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = 0.f;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->stats.launches += 3;
    if (e0) {
      ctx->stats.eik_launches += 1;
      ctx->stats.eik_ms += ms;
      ctx->stats.eik_updates += 4.0 * (double)sweeps * (double)N;
    }
  }
  if (iters) std::copy(it.begin(), it.end(), iters);
  if (stuck)
    return fail(ctx, RTM_ERR_STATE, "%lld problem(s) did not reach the fixed point in %d iterations",
                stuck, max_iter);
  return RTM_OK;
}
