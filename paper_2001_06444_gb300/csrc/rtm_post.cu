// rtm_post.cu — per-shot normalisation and stacking, the Laplacian filter of
// the brute stack, and the ensemble statistics of stage 3 (sm_103a).
#include <cuda_runtime.h>

#include <cmath>

#include "rtm_common.h"
#include "rtm_launch.h"

namespace rtm {

// Source-normalised image of each item (Eq. 5; eps max(den) keeps the
// division finite, a pixel with zero illumination contributes 0), added in
// item order to its sample's stack with Kahan compensation; num and den are
// cleared for the next batch.  One thread per 4 consecutive pixels.
__global__ void k_norm_stack(float *num, float *den, const unsigned *dmax,
                             const int *item_sample, int B, float eps, long long pplane,
                             float *stack_all, float *comp_all, int nsample, int *err) {
  const long long e = 4 * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
  if (e >= pplane) return;
  (void)nsample;
  (void)err;
  int cur = -1;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f), cmp = acc;
  for (int b = 0; b < B; ++b) {
    const int smp = item_sample[b];
    if (!RTM_IN(smp, nsample, err) || !RTM_IN(e + 3, pplane, err)) continue;
    if (smp != cur) {
      if (cur >= 0) {
        *reinterpret_cast<float4 *>(stack_all + cur * pplane + e) = acc;
        *reinterpret_cast<float4 *>(comp_all + cur * pplane + e) = cmp;
      }
      acc = *reinterpret_cast<const float4 *>(stack_all + smp * pplane + e);
      cmp = *reinterpret_cast<const float4 *>(comp_all + smp * pplane + e);
      cur = smp;
    }
    const float add = eps * __uint_as_float(dmax[b]);
    float4 *pn = reinterpret_cast<float4 *>(num + b * pplane + e);
    float4 *pd = reinterpret_cast<float4 *>(den + b * pplane + e);
    const float4 nu = *pn, de = *pd;
    const float nv[4] = {nu.x, nu.y, nu.z, nu.w};
    const float dv[4] = {de.x, de.y, de.z, de.w};
    float a[4] = {acc.x, acc.y, acc.z, acc.w};
    float c[4] = {cmp.x, cmp.y, cmp.z, cmp.w};
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const float dd = dv[l] + add;
      // eps < 0: the numerator as it is (the adjoint of Born modelling)
      const float img = eps < 0.f ? nv[l] : (dd > 0.f ? nv[l] / dd : 0.f);
      const float y = img - c[l];
      const float t = a[l] + y;
      c[l] = (t - a[l]) - y;
      a[l] = t;
    }
    acc = make_float4(a[0], a[1], a[2], a[3]);
    cmp = make_float4(c[0], c[1], c[2], c[3]);
    *pn = make_float4(0.f, 0.f, 0.f, 0.f);
    *pd = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (cur >= 0) {
    *reinterpret_cast<float4 *>(stack_all + cur * pplane + e) = acc;
    *reinterpret_cast<float4 *>(comp_all + cur * pplane + e) = cmp;
  }
}

// Laplacian filter of §3 on the stack: -(D_zz + D_xx) with 3-point second
// differences and the border value repeated outside; out is compact [nz][nx].
__global__ void k_filter(const float *stack_all, const float *comp_all, int nz, int nx, int SX,
                         float rdz2, float rdx2, int laplacian, float *out) {
  const int smp = blockIdx.z, i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nx) return;
  const long long base = (long long)smp * nz * SX;
  auto at = [&](int ii, int jj) {
    ii = min(max(ii, 0), nz - 1);
    jj = min(max(jj, 0), nx - 1);
    const long long o = base + (long long)ii * SX + jj;
    return stack_all[o] - comp_all[o];
  };
  const float c = at(i, j);
  float r = c;
  if (laplacian) {
    const float dzz = (at(i - 1, j) - 2.f * c) + at(i + 1, j);
    const float dxx = (at(i, j - 1) - 2.f * c) + at(i, j + 1);
    r = -(dzz * rdz2 + dxx * rdx2);
  }
  out[(long long)smp * nz * nx + (long long)i * nx + j] = r;
}

// Per-pixel statistics over n images: FP64 two-pass mean and standard
// deviation (divisor n-1), then a bitonic sort of each pixel's column in
// shared memory for the 5% / 95% quantiles (linear interpolation at
// h = (n-1) p).  A block stages PB pixels x npad values, pixel-fastest so
// global loads are coalesced and shared accesses are conflict-free.
__global__ void k_ens_stats(const float *images, int n, int npad, int PB, long long npix,
                            double *mean, double *std_, float *q05, float *q95) {
  extern __shared__ float sv[];  // [npad][PB]
  const long long p0 = (long long)blockIdx.x * PB;
  for (int idx = threadIdx.x; idx < npad * PB; idx += blockDim.x) {
    const int k = idx / PB, p = idx - k * PB;
    float x = INFINITY;
    if (k < n) x = (p0 + p < npix) ? images[(long long)k * npix + p0 + p] : 0.f;
    sv[idx] = x;
  }
  __syncthreads();
  double mu[2] = {0.0, 0.0}, sd[2] = {0.0, 0.0};
  for (int p = threadIdx.x, t = 0; p < PB && t < 2; p += blockDim.x, ++t) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += (double)sv[k * PB + p];
    const double m = s / n;
    double q = 0.0;
    for (int k = 0; k < n; ++k) {
      const double d = (double)sv[k * PB + p] - m;
      q += d * d;
    }
    mu[t] = m;
    sd[t] = n > 1 ? sqrt(q / (n - 1)) : 0.0;
  }
  __syncthreads();
  const int half = npad / 2;
  for (int k = 2; k <= npad; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < PB * half; t += blockDim.x) {
        const int p = t % PB, q = t / PB;
        const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));
        const int l = i | j;
        const float a = sv[i * PB + p], c = sv[l * PB + p];
        const bool up = (i & k) == 0;
        if ((a > c) == up) {
          sv[i * PB + p] = c;
          sv[l * PB + p] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int p = threadIdx.x, t = 0; p < PB && t < 2; p += blockDim.x, ++t) {
    const long long pix = p0 + p;
    if (pix >= npix) continue;
    mean[pix] = mu[t];
    std_[pix] = sd[t];
    const double ps[2] = {0.05, 0.95};
    float qo[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const double h = (double)(n - 1) * ps[u];
      const int lo = (int)floor(h);
      const int hi = min(lo + 1, n - 1);
      const double xl = sv[lo * PB + p], xh = sv[hi * PB + p];
      // separately rounded multiply and add (no FMA contraction), so the
      // FP64 value, and hence its float rounding, is the textbook formula's
      qo[u] = (float)__dadd_rn(xl, __dmul_rn(h - lo, __dsub_rn(xh, xl)));
    }
    q05[pix] = qo[0];
    q95[pix] = qo[1];
  }
}

__global__ void k_init_range(unsigned long long *mm) {
  mm[0] = 0ull;                    // max of a non-negative map
  mm[1] = 0x7FF0000000000000ull;  // +inf: min
}

__global__ void k_std_range(const double *std_, long long npix, unsigned long long *mm) {
  double mx = 0.0, mn = INFINITY;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < npix;
       e += (long long)gridDim.x * blockDim.x) {
    mx = fmax(mx, std_[e]);
    mn = fmin(mn, std_[e]);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&mm[0], (unsigned long long)__double_as_longlong(mx));
    atomicMin(&mm[1], (unsigned long long)__double_as_longlong(mn));
  }
}

// Eq. 6: c = (s_max - s) / (s_max - s_min), 1 if the map is flat;
// Eq. 7: r = s / mean, 0 where the mean is 0.
__global__ void k_unc_maps(const double *mean, const double *std_, long long npix,
                           const unsigned long long *mm, double *conf, double *ratio) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= npix) return;
  const double smax = __longlong_as_double((long long)mm[0]);
  const double smin = __longlong_as_double((long long)mm[1]);
  const double s = std_[e], m = mean[e];
  conf[e] = smax > smin ? (smax - s) / (smax - smin) : 1.0;
  ratio[e] = m != 0.0 ? s / m : 0.0;
}

// ------------------------------------------------------------ launchers --

cudaError_t launch_norm_stack(float *num, float *den, const unsigned *dmax,
                              const int *item_sample, int B, float eps, long long pplane,
                              float *stack_all, float *comp_all, int nsample, int *err,
                              cudaStream_t st) {
  const long long n4 = pplane / 4;
  k_norm_stack<<<(unsigned)((n4 + 255) / 256), 256, 0, st>>>(
      num, den, dmax, item_sample, B, eps, pplane, stack_all, comp_all, nsample, err);
  return cudaGetLastError();
}

cudaError_t launch_filter(const float *stack_all, const float *comp_all, int nsample, int nz,
                          int nx, int SX, float rdz2, float rdx2, int laplacian, float *out,
                          cudaStream_t st) {
  dim3 grid((nx + 127) / 128, nz, nsample);
  k_filter<<<grid, 128, 0, st>>>(stack_all, comp_all, nz, nx, SX, rdz2, rdx2, laplacian, out);
  return cudaGetLastError();
}

int ens_stats_max_n() { return 32768; }

cudaError_t launch_ens_stats(const float *images, int n, long long npix, double *mean,
                             double *std_, float *q05, float *q95, cudaStream_t st) {
  int npad = 1;
  while (npad < n) npad <<= 1;
  if (npad < 2) npad = 2;
  int PB = (48 * 1024) / (4 * npad);
  if (PB > 256) PB = 256;
  if (PB < 1) PB = 1;
  const size_t smem = (size_t)PB * npad * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_ens_stats, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = (npix + PB - 1) / PB;
  k_ens_stats<<<(unsigned)blocks, 256, smem, st>>>(images, n, npad, PB, npix, mean, std_, q05,
                                                   q95);
  return cudaGetLastError();
}

cudaError_t launch_unc_maps(const double *mean, const double *std_, long long npix,
                            double *conf, double *ratio, unsigned long long *scratch,
                            cudaStream_t st) {
  k_init_range<<<1, 1, 0, st>>>(scratch);
  long long blocks = (npix + 255) / 256;
  const unsigned rb = (unsigned)(blocks > 2048 ? 2048 : (blocks < 1 ? 1 : blocks));
  k_std_range<<<rb, 256, 0, st>>>(std_, npix, scratch);
  k_unc_maps<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, 0, st>>>(mean, std_, npix, scratch,
                                                                  conf, ratio);
  return cudaGetLastError();
}

}  // namespace rtm
