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
#include <vector>

#include "rtm_engine.h"
#include "rtm_launch.h"

namespace {

constexpr float kInf = __builtin_huge_valf();

struct EikArgs {
  const float *slow;     // [nsample][nz][nx] slowness (s/m)
  int nz, nx, nsrc, nrec;
  float dz, dx, wz, wx, wsum, wprod;  // spacings, 1/dz^2, 1/dx^2, their sum and product
  const int *src;        // [nsrc][2] (iz, ix)
  const int *rec;        // [nrec][2]
  float *times;          // [nsample][nsrc][nrec] or null
  float *fields;         // [nsample][nsrc][nz][nx]: output, and the work field off-chip
  int max_iter;
  int *iters;            // [nsample * nsrc] iterations to the fixed point, -1 at the cap
};

// The upwind update from the smaller vertical (a) and horizontal (b)
// neighbour times: one-sided from the smaller one if that does not exceed
// the other, else the larger root of the two-term quadratic.
__device__ __forceinline__ float update(float a, float b, float s, const EikArgs &A) {
  const bool vz = a <= b;
  const float u1 = vz ? a : b, u2 = vz ? b : a;
  const float h1 = vz ? A.dz : A.dx, w1 = vz ? A.wz : A.wx, w2 = vz ? A.wx : A.wz;
  const float t1 = __fadd_rn(u1, __fmul_rn(s, h1));
  if (t1 <= u2) return t1;  // also both neighbours unknown: inf
  const float d = __fsub_rn(u1, u2);
  const float disc = __fsub_rn(__fmul_rn(A.wsum, __fmul_rn(s, s)), __fmul_rn(A.wprod, __fmul_rn(d, d)));
  const float num = __fadd_rn(__fadd_rn(__fmul_rn(w1, u1), __fmul_rn(w2, u2)), __fsqrt_rn(fmaxf(disc, 0.f)));
  return __fdiv_rn(num, A.wsum);
}

template <bool RESIDENT>
__global__ void __launch_bounds__(1024) k_eik_sweep(const __grid_constant__ EikArgs A) {
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
    int changed = 0;
#pragma unroll 1
    for (int d = 0; d < 4; ++d) {
      const bool fz = d == 0 || d == 3, fx = d < 2;  // (+,+), (+,-), (-,-), (-,+) in (z, x)
      for (int l = 0; l < nz + nx - 1; ++l) {
        const int lo = max(0, l - (nx - 1)), hi = min(nz - 1, l);
        for (int ip = lo + (int)threadIdx.x; ip <= hi; ip += blockDim.x) {
          const int jp = l - ip;
          const int i = fz ? ip : nz - 1 - ip, j = fx ? jp : nx - 1 - jp;
          const long long k = (long long)i * nx + j;
          const float a = fminf(i > 0 ? T[k - nx] : kInf, i < nz - 1 ? T[k + nx] : kInf);
          const float b = fminf(j > 0 ? T[k - 1] : kInf, j < nx - 1 ? T[k + 1] : kInf);
          const float t = update(a, b, __ldg(s + k), A);
          if (t < T[k]) {
            T[k] = t;
            changed = 1;
          }
        }
        __syncthreads();
      }
    }
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
  A.src = src;
  A.rec = rec;
  A.times = times;
  A.fields = fields;
  A.max_iter = max_iter;
  A.iters = iters;
  const int level = std::min(nz, nx);
  const int threads = std::min(1024, std::max(32, (level + 31) / 32 * 32));
  const long long problems = (long long)nsample * nsrc;
  if (problems > 0x7fffffffll) return cudaErrorInvalidValue;
  if (resident) {
    const size_t smem = (size_t)nz * nx * 4;
    cudaError_t e = cudaFuncSetAttribute(k_eik_sweep<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_eik_sweep<true><<<(unsigned)problems, threads, smem, st>>>(A);
  } else {
    k_eik_sweep<false><<<(unsigned)problems, threads, 0, st>>>(A);
  }
  return cudaGetLastError();
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
  if (flags & ~RTM_EIK_OFFCHIP) return fail(ctx, RTM_ERR_ARG, "unknown flags %d", flags);
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
  const bool resident = !(flags & RTM_EIK_OFFCHIP) && (size_t)N * 4 <= eik_resident_limit();
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
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ctx->prof) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
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
  if (e0) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  if (iters) std::copy(it.begin(), it.end(), iters);
  if (stuck)
    return fail(ctx, RTM_ERR_STATE, "%lld problem(s) did not reach the fixed point in %d iterations",
                stuck, max_iter);
  return RTM_OK;
}
