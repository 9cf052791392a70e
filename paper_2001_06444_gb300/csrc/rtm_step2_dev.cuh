// rtm_step2_dev.cuh — device helpers shared by the two-step propagation
// kernels (rtm_prop2.cu: one tile per block; rtm_prop2p.cu: persistent blocks
// with a two-stage copy ring).  Both kernels evaluate the scheme of §2.2
// Eq. 4 / §3 in the difference form described in rtm_prop.cu, with the same
// per-point arithmetic, so their fields agree bit for bit with each other and
// with the single-step kernel.
#pragma once
#include <cuda.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "rtm_common.h"

namespace rtm {
namespace s2 {

constexpr int C2X = 120;                      // centre tile width (memory columns)
constexpr int EX = C2X + 8;                   // extended region width (halo 4)
constexpr int VX = C2X + 16;                  // v^n tile width (halo 8)
constexpr int NTH = 256;                      // 32 x 8 threads
constexpr unsigned long long kWaitNs = 1000000000ull;  // bound of a device-side wait: 1 s

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float lane4(const float4 &v, int l) {
  return l == 0 ? v.x : (l == 1 ? v.y : (l == 2 ? v.z : v.w));
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Wait for the mbarrier phase to complete, for at most `ns` nanoseconds.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned phase,
                                                  unsigned long long ns) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, phase))
    if (global_ns() - t0 > ns) return false;
  return true;
}

// Quantised store / load of 4 consecutive physical values (same encoding as
// the single-step kernel).
__device__ __forceinline__ void snap_store4(void *base, long long off, int dtype, float4 v,
                                            float inv_s) {
  if (dtype == 0) {
    *reinterpret_cast<float4 *>(reinterpret_cast<float *>(base) + off) = v;
  } else if (dtype == 2) {
    __half2 a = __floats2half2_rn(v.x * inv_s, v.y * inv_s);
    __half2 b = __floats2half2_rn(v.z * inv_s, v.w * inv_s);
    uint2 u;
    u.x = *reinterpret_cast<unsigned *>(&a);
    u.y = *reinterpret_cast<unsigned *>(&b);
    *reinterpret_cast<uint2 *>(reinterpret_cast<__half *>(base) + off) = u;
  } else {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x * inv_s, v.y * inv_s);
    __nv_bfloat162 b = __floats2bfloat162_rn(v.z * inv_s, v.w * inv_s);
    uint2 u;
    u.x = *reinterpret_cast<unsigned *>(&a);
    u.y = *reinterpret_cast<unsigned *>(&b);
    *reinterpret_cast<uint2 *>(reinterpret_cast<__nv_bfloat16 *>(base) + off) = u;
  }
}

__device__ __forceinline__ float4 snap_load4(const void *base, long long off, int dtype, float s) {
  if (dtype == 0) return *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(base) + off);
  uint2 u;
  if (dtype == 2) {
    u = *reinterpret_cast<const uint2 *>(reinterpret_cast<const __half *>(base) + off);
    const float2 a = __half22float2(*reinterpret_cast<__half2 *>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<__half2 *>(&u.y));
    return make_float4(a.x * s, a.y * s, b.x * s, b.y * s);
  }
  u = *reinterpret_cast<const uint2 *>(reinterpret_cast<const __nv_bfloat16 *>(base) + off);
  const float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.y));
  return make_float4(a.x * s, a.y * s, b.x * s, b.y * s);
}

__device__ __forceinline__ void snap_scale(int dtype, unsigned mbits, float &s, float &inv) {
  if (dtype == 0) {
    s = inv = 1.f;
    return;
  }
  const float m = __uint_as_float(mbits);
  if (!(m > 0.f)) {
    s = inv = 0.f;
    return;
  }
  if (dtype == 2) {
    s = m * (1.f / 32768.f);
    inv = 32768.f / m;
  } else {
    s = m;
    inv = 1.f / m;
  }
}

__device__ __forceinline__ void block_max_atomic(float v, unsigned *dst, float *red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (threadIdx.x == 0) red[threadIdx.y] = v;
  __syncthreads();
  if (threadIdx.y == 0) {
    v = threadIdx.x < (NTH / 32) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 4; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0 && v > 0.f) atomicMax(dst, __float_as_uint(v));
  }
}

// Paired FP32 arithmetic (__fadd2_rn, __ffma2_rn, __fmul2_rn: two lanes per
// instruction).  Each lane rounds exactly like the scalar operation, so
// results equal the scalar kernel's.

// One leapfrog update of 4 consecutive points.
//   zc[0..8]: the 9 rows (centre row zc[4]) of the 4-column strip,
//   xl, xr:   the 4 columns left and right of the strip in the centre row,
//   dv, cv:   d^n and c at the strip,
//   SPONGE:   the block's region reaches the sponge: every point takes the
//             sponge form (which gives the interior formula's bits where
//             g = 1), with gzr the row's factor and gxs the strip's four (in
//             shared memory).  Blocks clear of the sponge compile in the
//             interior formula alone.  (Choosing between the two forms per
//             row measured slower.)
//   ISO:      dx == dz.  The Laplacian is summed ring by ring, m = 4..1: the
//             ring's neighbours are added first, then the centre is taken
//             off with one rounding, t_m = fma(v0, -4, (v_-m + v_+m) +
//             (w_-m + w_+m)) along x (v) and z (w), lap = fma(a_m/h^2, t_m,
//             lap).  Otherwise each direction alone, fma(v0, -2, v_-m +
//             v_+m) scaled by its own a_m/dx^2 or a_m/dz^2.  Taking the
//             centre off per ring keeps FP32 cancellation small (the
//             17-term sum of the plain form does not).
// Returns d^{n+1} (before injection); v^{n+1} = v^n + d^{n+1}.  Lanes are
// processed in pairs (0,1) and (2,3); each lane rounds as the scalar form of
// the single-step kernel.
template <bool SPONGE, bool ISO>
__device__ __forceinline__ float4 update4(const float4 *zc, const float4 &xl, const float4 &xr,
                                          const float4 &dv, const float4 &cv, const Coef &k,
                                          float gzr, const float *gxs) {
  const float4 xc = zc[4];
  const float v[12] = {xl.x, xl.y, xl.z, xl.w, xc.x, xc.y, xc.z, xc.w, xr.x, xr.y, xr.z, xr.w};
  float out[4];
#pragma unroll
  for (int l = 0; l < 4; l += 2) {
    const float2 ce = make_float2(v[4 + l], v[5 + l]);
    float2 lap = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 4; m >= 1; --m) {
      const float2 xm = make_float2(v[4 + l - m], v[5 + l - m]);
      const float2 xp = make_float2(v[4 + l + m], v[5 + l + m]);
      const float2 zm = l == 0 ? make_float2(zc[4 - m].x, zc[4 - m].y)
                               : make_float2(zc[4 - m].z, zc[4 - m].w);
      const float2 zp = l == 0 ? make_float2(zc[4 + m].x, zc[4 + m].y)
                               : make_float2(zc[4 + m].z, zc[4 + m].w);
      if (ISO) {
        const float2 s = __fadd2_rn(__fadd2_rn(xm, xp), __fadd2_rn(zm, zp));
        const float2 t = __ffma2_rn(ce, make_float2(-4.f, -4.f), s);
        lap = __ffma2_rn(make_float2(k.ax[m - 1], k.ax[m - 1]), t, lap);
      } else {
        const float2 tx = __ffma2_rn(ce, make_float2(-2.f, -2.f), __fadd2_rn(xm, xp));
        lap = __ffma2_rn(make_float2(k.ax[m - 1], k.ax[m - 1]), tx, lap);
        const float2 tz = __ffma2_rn(ce, make_float2(-2.f, -2.f), __fadd2_rn(zm, zp));
        lap = __ffma2_rn(make_float2(k.az[m - 1], k.az[m - 1]), tz, lap);
      }
    }
    const float2 c = l == 0 ? make_float2(cv.x, cv.y) : make_float2(cv.z, cv.w);
    const float2 p = l == 0 ? make_float2(dv.x, dv.y) : make_float2(dv.z, dv.w);
    const float2 nd = __ffma2_rn(c, lap, p);
    if (!SPONGE) {
      out[l] = nd.x;
      out[l + 1] = nd.y;
    } else {
      // g^2 d + g c L v - (1-g)^2 v, each lane rounded as the scalar form
      // fmaf(g g, d, fmaf(g c, L v, (-(1-g)(1-g)) v)) of the single-step
      // kernel; points with g == 1 take the interior formula
      const float2 gg = __fmul2_rn(make_float2(gzr, gzr),
                                   *reinterpret_cast<const float2 *>(gxs + l));
      const float2 om = __ffma2_rn(gg, make_float2(-1.f, -1.f), make_float2(1.f, 1.f));
      const float2 mo = __ffma2_rn(gg, make_float2(1.f, 1.f), make_float2(-1.f, -1.f));
      const float2 w = __fmul2_rn(__fmul2_rn(om, mo), ce);
      const float2 sp = __ffma2_rn(__fmul2_rn(gg, gg), p, __ffma2_rn(__fmul2_rn(gg, c), lap, w));
      out[l] = gg.x == 1.f ? nd.x : sp.x;
      out[l + 1] = gg.y == 1.f ? nd.y : sp.y;
    }
  }
  return make_float4(out[0], out[1], out[2], out[3]);
}

// Born modelling: d += (c m) S at the physical pixels of a 4-column strip
// (row i, columns j0..j0+3; j0 a multiple of 4) from snapshot idx; the same
// rounding as the single-step kernel.
__device__ __forceinline__ float4 born_inject4(const Step2Args &A, int b, int idx, int i, int j0,
                                               float4 d, const float4 &c) {
  const Geo &g = A.g;
  if (idx < 0 || i < 0 || i >= g.nz || j0 < 0 || j0 >= g.SX) return d;
  const long long so = ((long long)b * A.nsnap + idx) * g.pplane + (long long)i * g.SX + j0;
  if (!RTM_IN((long long)b * A.nsnap + idx, A.len.smax, A.err) || !RTM_IN(so + 3, A.len.snap, A.err) ||
      !RTM_IN((long long)i * g.nx + min(j0 + 3, g.nx - 1), A.len.refl, A.err))
    return d;
  float sdq, inv;
  snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + idx], sdq, inv);
  const float4 S = snap_load4(A.snap, so, A.snap_dtype, sdq);
  const float *m = A.refl + (long long)i * g.nx + j0;
  if (j0 < g.nx) d.x = fmaf(c.x * __ldg(m), S.x, d.x);
  if (j0 + 1 < g.nx) d.y = fmaf(c.y * __ldg(m + 1), S.y, d.y);
  if (j0 + 2 < g.nx) d.z = fmaf(c.z * __ldg(m + 2), S.z, d.z);
  if (j0 + 3 < g.nx) d.w = fmaf(c.w * __ldg(m + 3), S.w, d.w);
  return d;
}

}  // namespace s2
}  // namespace rtm
