// rtm_lsrtm.cu — least-squares migration: the reflectivity m that minimises
// ||B m - d||^2, B being Born modelling (rtm_born) and B^T its adjoint
// (rtm_migrate_adjoint), by conjugate gradients on the normal equations
// (CGLS, Hestenes and Stiefel 1952; Paige and Saunders 1982).  Each
// iteration applies B once and B^T once; the vector updates and the inner
// products (FP64 accumulation, a fixed reduction order, so results repeat
// bit for bit) are the kernels below.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rtm_engine.h"

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1024;

// partial[b] = sum over this block's grid-stride share of x[i] y[i]
__global__ void __launch_bounds__(kRedThreads) k_dot_partial(const float *x, const float *y,
                                                             long long n, double *partial) {
  __shared__ double red[kRedThreads / 32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)kRedThreads + threadIdx.x; i < n;
       i += (long long)gridDim.x * kRedThreads)
    acc += (double)x[i] * (double)y[i];
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_dot_final(const double *partial, int n, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += partial[b];
    *out = s;
  }
}

// y = y + a x
__global__ void k_axpy(float *y, const float *x, double a, long long n) {
  const float af = (float)a;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = fmaf(af, x[i], y[i]);
}

// p = s + b p
__global__ void k_xpby(float *p, const float *s, double b, long long n) {
  const float bf = (float)b;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = fmaf(bf, p[i], s[i]);
}

unsigned grid_for(long long n) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 16));
}

}  // namespace

using namespace rtm;

#define LS_CU(x)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) return fail(ctx, RTM_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

extern "C" int rtm_lsrtm(rtm_ctx *ctx, const rtm_grid *grid, const float *vel, const rtm_acq *acq,
                         const float *seis, const rtm_opts *opts, int niter, float *refl,
                         double *misfit, void *stream) {
  if (!ctx) return RTM_ERR_ARG;
  int rc;
  if ((rc = check_grid(ctx, grid)) || (rc = check_acq(ctx, grid, acq, true)) ||
      (rc = check_opts(ctx, opts)))
    return rc;
  if (!vel || !seis || !refl) return fail(ctx, RTM_ERR_ARG, "NULL array argument");
  if (niter < 0 || niter > 10000) return fail(ctx, RTM_ERR_ARG, "need 0 <= niter <= 10000");
  if (opts->checkpoint)
    return fail(ctx, RTM_ERR_ARG, "least-squares migration keeps every snapshot (checkpoint 0)");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, RTM_ERR_CUDA, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const long long npix = (long long)grid->nx * grid->nz;
  const long long ndat = (long long)acq->nshot * grid->nt * acq->nrec;
  DevBuf dv, dm, dp, ds, dr, dq, dpart;
  const float *v = vel;
  if (!is_device_ptr(vel)) {
    LS_CU(dv.alloc(ctx, (size_t)npix * 4, st));
    LS_CU(cudaMemcpyAsync(dv.p, vel, (size_t)npix * 4, cudaMemcpyHostToDevice, st));
    v = dv.as<float>();
  }
  LS_CU(dm.alloc(ctx, (size_t)npix * 4, st));
  LS_CU(dp.alloc(ctx, (size_t)npix * 4, st));
  LS_CU(ds.alloc(ctx, (size_t)npix * 4, st));
  LS_CU(dr.alloc(ctx, (size_t)ndat * 4, st));
  LS_CU(dq.alloc(ctx, (size_t)ndat * 4, st));
  LS_CU(dpart.alloc(ctx, (kRedBlocks + 1) * sizeof(double), st));
  // r = d (m = 0), s = B^T r, p = s
  LS_CU(cudaMemsetAsync(dm.p, 0, dm.bytes, st));
  LS_CU(cudaMemcpyAsync(dr.p, seis, (size_t)ndat * 4, cudaMemcpyDefault, st));
  double *partial = dpart.as<double>(), *dres = partial + kRedBlocks;
  auto dot = [&](const float *x, const float *y, long long n, double *out) -> int {
    const unsigned b = (unsigned)std::min<long long>(kRedBlocks, (n + kRedThreads - 1) / kRedThreads);
    k_dot_partial<<<b, kRedThreads, 0, st>>>(x, y, n, partial);
    k_dot_final<<<1, 32, 0, st>>>(partial, (int)b, dres);
    LS_CU(cudaGetLastError());
    LS_CU(cudaMemcpyAsync(out, dres, sizeof(double), cudaMemcpyDeviceToHost, st));
    LS_CU(cudaStreamSynchronize(st));
    return RTM_OK;
  };
  float *m = dm.as<float>(), *p = dp.as<float>(), *s = ds.as<float>(), *r = dr.as<float>(),
        *q = dq.as<float>();
  double rr = 0.0, gamma = 0.0, qq = 0.0, g2 = 0.0;
  if ((rc = dot(r, r, ndat, &rr))) return rc;
  if (misfit) misfit[0] = rr;
  if ((rc = rtm_migrate_adjoint(ctx, grid, v, acq, r, opts, s, st))) return rc;
  LS_CU(cudaMemcpyAsync(p, s, (size_t)npix * 4, cudaMemcpyDeviceToDevice, st));
  if ((rc = dot(s, s, npix, &gamma))) return rc;
  long long launches = 2 * 2;
  for (int it = 0; it < niter; ++it) {
    if (!(gamma > 0.0)) {  // the gradient vanished: m is the solution
      if (misfit) std::fill(misfit + it + 1, misfit + niter + 1, rr);
      break;
    }
    if ((rc = rtm_born(ctx, grid, v, acq, p, opts, q, st))) return rc;  // q = B p
    if ((rc = dot(q, q, ndat, &qq))) return rc;
    if (!(qq > 0.0)) {
      if (misfit) std::fill(misfit + it + 1, misfit + niter + 1, rr);
      break;
    }
    const double alpha = gamma / qq;
    k_axpy<<<grid_for(npix), 256, 0, st>>>(m, p, alpha, npix);    // m += alpha p
    k_axpy<<<grid_for(ndat), 256, 0, st>>>(r, q, -alpha, ndat);   // r -= alpha q
    LS_CU(cudaGetLastError());
    if ((rc = dot(r, r, ndat, &rr))) return rc;
    if (misfit) misfit[it + 1] = rr;
    if ((rc = rtm_migrate_adjoint(ctx, grid, v, acq, r, opts, s, st))) return rc;  // s = B^T r
    if ((rc = dot(s, s, npix, &g2))) return rc;
    k_xpby<<<grid_for(npix), 256, 0, st>>>(p, s, g2 / gamma, npix);  // p = s + beta p
    LS_CU(cudaGetLastError());
    gamma = g2;
    launches += 3 + 3 * 2;  // axpy, axpy, xpby; three inner products of two kernels
  }
  LS_CU(cudaMemcpyAsync(refl, m, (size_t)npix * 4, cudaMemcpyDefault, st));
  LS_CU(cudaStreamSynchronize(st));
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->stats.launches += launches;
  }
  return RTM_OK;
}
