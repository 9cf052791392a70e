// rtm_prop.cu — wave propagation kernels (sm_103a).
//
// One launch of k_step advances B independent grids (velocity sample x shot)
// by one leapfrog step of the 2D acoustic wave equation (§2.2, Eq. 4),
// 2nd order in time and 8th order in space (§3).  The padded-grid field is
// stepped in the variable v = h u (h = sqrt(g), g the sponge factor), in which
// the symmetric sponge scheme
//     u^{n+1} = h (2 h u^n + c L(h u^n)) - g^2 u^{n-1} + c f^n
// reads v^{n+1} = g (2 v^n + c L v^n) - g^2 v^{n-1} + c f^n.  h == 1 on the
// physical grid, so sources, receivers, snapshots and images see u itself.
// The recurrence is carried in difference form, d^n = v^n - v^{n-1}:
//     d^{n+1} = g^2 d^n + g c L v^n - (1 - g)^2 v^n + c f^n,
//     v^{n+1} = v^n + d^{n+1}
// (d^{n+1} = d^n + c L v^n + c f^n inside the sponge-free region), the same
// scheme in exact arithmetic.  In FP32 it keeps the time difference to full
// relative precision instead of to eps |v|, which removes the rounding error
// that the two-level form feeds into its non-decaying mode at every step.
// L v is summed ring by ring, the centre taken off each ring's neighbour sum
// with one rounding (see the stencil below), which keeps the cancellation of
// the plain 17-term sum out of FP32.
// The same kernel steps the reverse-time (adjoint) field, which obeys the
// same recurrence with the data injected at the receivers (§3).
//
// Fused into the step (all optional, block-uniform branches):
//   - source injection c f^n (forward) / receiver injection c d (backward),
//     through a shared-memory staging pass only in blocks that own such cells;
//   - trace recording (modelling);
//   - storing the CURRENT field u^n as a quantised snapshot S^n whose scale
//     max|S^n| was reduced by the previous launch (no extra read of u^n);
//   - reducing max|u^{n+1}| for the next snapshot's scale;
//   - the imaging condition of Eq. 5: num += S^k w^k, den += (S^k)^2, and the
//     final max(den) used by the normalisation.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "rtm_common.h"
#include "rtm_launch.h"

namespace rtm {

__device__ __forceinline__ float lane4(const float4 &v, int l) {
  return l == 0 ? v.x : (l == 1 ? v.y : (l == 2 ? v.z : v.w));
}

// Quantised store of 4 consecutive physical values (16-byte aligned for f32,
// 8-byte for 16-bit codes).
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

__device__ __forceinline__ float4 snap_load4(const void *base, long long off, int dtype,
                                             float s) {
  if (dtype == 0) return *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(base) + off);
  uint2 u;
  float4 r;
  if (dtype == 2) {
    u = *reinterpret_cast<const uint2 *>(reinterpret_cast<const __half *>(base) + off);
    float2 a = __half22float2(*reinterpret_cast<__half2 *>(&u.x));
    float2 b = __half22float2(*reinterpret_cast<__half2 *>(&u.y));
    r = make_float4(a.x * s, a.y * s, b.x * s, b.y * s);
  } else {
    u = *reinterpret_cast<const uint2 *>(reinterpret_cast<const __nv_bfloat16 *>(base) + off);
    float2 a = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.x));
    float2 b = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&u.y));
    r = make_float4(a.x * s, a.y * s, b.x * s, b.y * s);
  }
  return r;
}

// Scale of a stored snapshot: s with S ~= q s; inv = 1/s used when quantising.
__device__ __forceinline__ void snap_scale(int dtype, unsigned mbits, float &s, float &inv) {
  if (dtype == 0) {
    s = 1.f;
    inv = 1.f;
    return;
  }
  const float m = __uint_as_float(mbits);
  if (!(m > 0.f)) {
    s = 0.f;
    inv = 0.f;
    return;
  }
  if (dtype == 2) {  // FP16: s = max / 2^15
    s = m * (1.f / 32768.f);
    inv = 32768.f / m;
  } else {           // BF16: s = max
    s = m;
    inv = 1.f / m;
  }
}

// Block-wide max of a non-negative value, one atomicMax on its float bits.
// Must be reached by every thread of the block.
__device__ __forceinline__ void block_max_atomic(float v, unsigned *dst, float *red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (threadIdx.x == 0) red[threadIdx.y] = v;
  __syncthreads();
  if (threadIdx.y == 0) {
    v = threadIdx.x < (STEP_THREADS / 32) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 4; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0 && v > 0.f) atomicMax(dst, __float_as_uint(v));
  }
}

template <int MODE>
__global__ void __launch_bounds__(STEP_THREADS, 2) k_step(const StepArgs A, const StepRT rt) {
  __shared__ __align__(16) float s[SH][SW];
  __shared__ float red[STEP_THREADS / 32];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const Geo &g = A.g;
  const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ;
#ifdef RTM_DEBUG
  // an item or sample outside its table is recorded; the block then works on
  // item 0 / sample 0 instead of reading past the buffers
  const int b = RTM_IN(blockIdx.z, A.len.items, A.err) ? (int)blockIdx.z : 0;
  const int smp0 = A.item_sample[b];
  const int smp = RTM_IN(smp0, A.len.nsample, A.err) ? smp0 : 0;
#else
  const int b = blockIdx.z;
  const int smp = A.item_sample[b];
#endif
  const float *__restrict__ cur = A.fa + (long long)b * g.plane;
  float *__restrict__ out = A.fb + (long long)b * g.plane;
  float *__restrict__ dd = A.fd + (long long)b * g.plane;
  const float *__restrict__ cc = A.c_all + (long long)smp * g.plane;

  // 1. current field, tile + halo, into shared memory (zero beyond the buffer)
  constexpr int SW4 = SW / 4;
  for (int i = tid; i < SH * SW4; i += STEP_THREADS) {
    const int r = i / SW4, c4 = i - r * SW4;
    const int gr = z0 - HALO + r, gc = x0 - HALO + 4 * c4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gr >= 0 && gr < g.NZ && gc >= 0 && gc < g.P)
      v = __ldg(reinterpret_cast<const float4 *>(cur + (long long)gr * g.P + gc));
    *reinterpret_cast<float4 *>(&s[r][4 * c4]) = v;
  }
  // 2. time difference and c at this thread's 4 x 4 points
  const int col = x0 + 4 * tx, row0 = z0 + 4 * ty;
  const bool colok = col < g.P;
  float4 pv[4], cv[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    if (colok && row0 + r < g.NZ) {
      const long long o = (long long)(row0 + r) * g.P + col;
      pv[r] = *reinterpret_cast<const float4 *>(dd + o);
      cv[r] = __ldg(reinterpret_cast<const float4 *>(cc + o));
    } else {
      pv[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      cv[r] = pv[r];
    }
  }
  __syncthreads();

  // 3. stencil
  const int sc = HALO + 4 * tx;
  float4 zc[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) zc[q] = *reinterpret_cast<const float4 *>(&s[4 * ty + q][sc]);
  const bool interior = (z0 >= g.nb) && (z0 + TZ <= g.NZ - g.nb) && (x0 >= g.X0 + g.nb) &&
                        (x0 + TX <= g.X0 + g.NX - g.nb);
  float res[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const float4 xl = *reinterpret_cast<const float4 *>(&s[4 * ty + 4 + r][sc - 4]);
    const float4 xr = *reinterpret_cast<const float4 *>(&s[4 * ty + 4 + r][sc + 4]);
    const float4 xc = zc[r + 4];
    const float v[12] = {xl.x, xl.y, xl.z, xl.w, xc.x, xc.y, xc.z, xc.w, xr.x, xr.y, xr.z, xr.w};
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const float ce = v[4 + l];
      // L v ring by ring (the centre weight is -2 sum a_m exactly): the
      // ring's neighbours are summed, then the centre is taken off with one
      // rounding, so each ring's term is a small second difference and FP32
      // cancellation stays small.  dx == dz: one ring of 4 neighbours per m,
      // fma(v0, -4, (x_-m + x_+m) + (z_-m + z_+m)); otherwise each direction
      // with its own weight, fma(v0, -2, x_-m + x_+m).
      float lap = 0.f;
      if (A.k.iso) {
#pragma unroll
        for (int m = 4; m >= 1; --m) {
          const float s = (v[4 + l - m] + v[4 + l + m]) +
                          (lane4(zc[r + 4 - m], l) + lane4(zc[r + 4 + m], l));
          lap = fmaf(A.k.ax[m - 1], fmaf(ce, -4.f, s), lap);
        }
      } else {
#pragma unroll
        for (int m = 4; m >= 1; --m) {
          lap = fmaf(A.k.ax[m - 1], fmaf(ce, -2.f, v[4 + l - m] + v[4 + l + m]), lap);
          lap = fmaf(A.k.az[m - 1],
                     fmaf(ce, -2.f, lane4(zc[r + 4 - m], l) + lane4(zc[r + 4 + m], l)), lap);
        }
      }
      const float c = lane4(cv[r], l), p = lane4(pv[r], l);
      float nd;  // d^{n+1} before injection
      if (interior) {
        nd = fmaf(c, lap, p);
      } else {
        const float gg = A.gz[min(row0 + r, g.NZ - 1)] * A.gx[min(col + l, g.P - 1)];
        const float om = 1.f - gg;
        // points with g == 1 take the interior formula whatever their tile
        nd = gg == 1.f ? fmaf(c, lap, p) : fmaf(gg * gg, p, fmaf(gg * c, lap, -(om * om) * ce));
      }
      res[r][l] = nd;
    }
  }

  // 3b. Born modelling: the secondary source c m S^{n+1} of the perturbation
  //     field at every physical pixel, on imaging steps
  const int j0 = col - g.CP;  // physical column of lane 0 (multiple of 4)
  const bool jok = j0 >= 0 && j0 < g.SX;
  if (MODE == MODE_BORN && rt.img_idx >= 0 && jok &&
      RTM_IN((long long)b * A.nsnap + rt.img_idx, A.len.smax, A.err)) {
    float sdq, inv;
    snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + rt.img_idx], sdq, inv);
    const long long sbase = ((long long)b * A.nsnap + rt.img_idx) * g.pplane + j0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = row0 + r - g.nb;
      if (i >= 0 && i < g.nz && RTM_IN(sbase + (long long)i * g.SX + 3, A.len.snap, A.err) &&
          RTM_IN((long long)i * g.nx + min(j0 + 3, g.nx - 1), A.len.refl, A.err)) {
        const float4 S = snap_load4(A.snap, sbase + (long long)i * g.SX, A.snap_dtype, sdq);
        const float Sv[4] = {S.x, S.y, S.z, S.w};
#pragma unroll
        for (int l = 0; l < 4; ++l)
          if (j0 + l < g.nx)
            res[r][l] = fmaf(lane4(cv[r], l) * __ldg(A.refl + (long long)i * g.nx + j0 + l), Sv[l],
                             res[r][l]);
      }
    }
  }

  // 4. injection / recording through shared memory (only blocks that own
  //    a source or receiver cell; the condition is block-uniform)
#ifdef RTM_DEBUG
  const int shot0 = A.item_shot[b];
  const bool shot_ok = RTM_IN(shot0, A.len.nshot, A.err) &&
                       RTM_IN(blockIdx.y * g.ntx + blockIdx.x + 1, g.ntx * g.ntz + 1, A.err);
  const int shot = shot_ok ? shot0 : 0;
#else
  const int shot = A.item_shot[b];
  constexpr bool shot_ok = true;
#endif
  bool stage = false;
  int sr = -1, scl = -1, rp0 = 0, rp1 = 0;
  if (MODE == MODE_FWD || MODE == MODE_MODEL) {
    sr = A.src_row[shot] - z0;
    scl = A.src_col[shot] - x0;
    if (sr >= 0 && sr < TZ && scl >= 0 && scl < TX)
      stage = true;
    else
      sr = -1;
  }
  if (MODE != MODE_FWD && shot_ok) {
    const int tile = blockIdx.y * g.ntx + blockIdx.x;
    rp0 = A.rtile_ptr[tile];
    rp1 = A.rtile_ptr[tile + 1];
    if (rp1 > rp0) stage = true;
  }
  if (stage) {
    __syncthreads();  // every read of the input tile is done
#pragma unroll
    for (int r = 0; r < 4; ++r)
      *reinterpret_cast<float4 *>(&s[HALO + 4 * ty + r][sc]) =
          make_float4(res[r][0], res[r][1], res[r][2], res[r][3]);
    __syncthreads();
    if (MODE == MODE_FWD || MODE == MODE_MODEL) {
      if (sr >= 0 && tid == 0 && RTM_IN(rt.n, A.nt, A.err)) {
        const long long o = (long long)(z0 + sr) * g.P + (x0 + scl);
        s[HALO + sr][HALO + scl] += cc[o] * (A.wav[rt.n] * A.src_scale);
      }
    } else if (MODE == MODE_BWD) {
      const long long d0 = ((long long)shot * A.nt + (rt.n - 1)) * A.nrec;
      const float *d = A.seis + d0;
      for (int e = rp0 + tid; e < rp1; e += STEP_THREADS) {
        if (!RTM_IN(e, A.len.rent, A.err)) continue;
        const int2 en = A.rtile_ent[e];
        const int lr = en.x / TX, lc = en.x - lr * TX;
        const long long o = (long long)(z0 + lr) * g.P + (x0 + lc);
        if (RTM_IN(en.x, TX * TZ, A.err) && RTM_IN(o, g.plane, A.err) &&
            RTM_IN(en.y, A.nrec, A.err) && RTM_IN(d0 + en.y, A.len.nshot * A.nt * A.nrec, A.err))
          atomicAdd(&s[HALO + lr][HALO + lc], cc[o] * d[en.y]);
      }
    }
    __syncthreads();
    if (MODE == MODE_MODEL || MODE == MODE_BORN) {
      const long long r0 = ((long long)b * A.nt + rt.n) * A.nrec;
      float *ro = A.rec_out + r0;
      for (int e = rp0 + tid; e < rp1; e += STEP_THREADS) {
        if (!RTM_IN(e, A.len.rent, A.err)) continue;
        const int2 en = A.rtile_ent[e];
        const int lr = en.x / TX, lc = en.x - lr * TX;
        const long long o = (long long)(z0 + lr) * g.P + (x0 + lc);
        if (RTM_IN(en.x, TX * TZ, A.err) && RTM_IN(o, g.plane, A.err) &&
            RTM_IN(r0 + en.y, A.len.rec_out, A.err))
          ro[en.y] = cur[o] + s[HALO + lr][HALO + lc];  // v^{n+1} = v^n + d^{n+1}
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float4 t = *reinterpret_cast<const float4 *>(&s[HALO + 4 * ty + r][sc]);
      res[r][0] = t.x;
      res[r][1] = t.y;
      res[r][2] = t.z;
      res[r][3] = t.w;
    }
  }

  // 5. new difference and new field v^{n+1} = v^n + d^{n+1}
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    if (colok && row0 + r < g.NZ) {
      const long long o = (long long)(row0 + r) * g.P + col;
      *reinterpret_cast<float4 *>(dd + o) = make_float4(res[r][0], res[r][1], res[r][2], res[r][3]);
      const float4 ce = zc[r + 4];
      res[r][0] += ce.x;
      res[r][1] += ce.y;
      res[r][2] += ce.z;
      res[r][3] += ce.w;
      *reinterpret_cast<float4 *>(out + o) = make_float4(res[r][0], res[r][1], res[r][2], res[r][3]);
    }
  }

  // 6. forward: store the current field as a snapshot, reduce the new max
  if (MODE == MODE_FWD) {
    if (rt.snap_idx >= 0 && jok && RTM_IN((long long)b * A.nsnap + rt.snap_idx, A.len.smax, A.err)) {
      float sdq, inv;
      snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + rt.snap_idx], sdq, inv);
      const long long base = ((long long)b * A.nsnap + rt.snap_idx) * g.pplane + j0;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = row0 + r - g.nb;
        if (i >= 0 && i < g.nz) {
          float4 v = zc[r + 4];
          if (j0 + 1 >= g.nx) v.y = 0.f;
          if (j0 + 2 >= g.nx) v.z = 0.f;
          if (j0 + 3 >= g.nx) v.w = 0.f;
          if (RTM_IN(base + (long long)i * g.SX + 3, A.len.snap, A.err))
            snap_store4(A.snap, base + (long long)i * g.SX, A.snap_dtype, v, inv);
        }
      }
    }
    if (rt.max_idx >= 0) {
      float m = 0.f;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = row0 + r - g.nb;
#pragma unroll
        for (int l = 0; l < 4; ++l)
          if (i >= 0 && i < g.nz && j0 + l >= 0 && j0 + l < g.nx) m = fmaxf(m, fabsf(res[r][l]));
      }
      const long long k = (long long)b * A.nsnap + rt.max_idx;
      block_max_atomic(m, &A.smax[RTM_IN(k, A.len.smax, A.err) ? k : 0], red);
    }
  }

  // 7. backward: imaging condition of Eq. 5 (numerator and illumination)
  if (MODE == MODE_BWD && rt.img_idx >= 0) {
    float dm = 0.f;
    if (jok && RTM_IN((long long)b * A.nsnap + rt.img_idx, A.len.smax, A.err)) {
      float sdq, inv;
      snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + rt.img_idx], sdq, inv);
      const long long sbase = ((long long)b * A.nsnap + rt.img_idx) * g.pplane + j0;
      const long long pbase = (long long)b * g.pplane + j0;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int i = row0 + r - g.nb;
        if (i >= 0 && i < g.nz && RTM_IN(sbase + (long long)i * g.SX + 3, A.len.snap, A.err) &&
            RTM_IN(pbase + (long long)i * g.SX + 3, A.len.items * g.pplane, A.err)) {
          const float4 S = snap_load4(A.snap, sbase + (long long)i * g.SX, A.snap_dtype, sdq);
          float4 *pn = reinterpret_cast<float4 *>(A.num + pbase + (long long)i * g.SX);
          float4 *pd = reinterpret_cast<float4 *>(A.den + pbase + (long long)i * g.SX);
          float4 nu = *pn, de = *pd;
          nu.x = fmaf(S.x, res[r][0], nu.x);
          nu.y = fmaf(S.y, res[r][1], nu.y);
          nu.z = fmaf(S.z, res[r][2], nu.z);
          nu.w = fmaf(S.w, res[r][3], nu.w);
          de.x = fmaf(S.x, S.x, de.x);
          de.y = fmaf(S.y, S.y, de.y);
          de.z = fmaf(S.z, S.z, de.z);
          de.w = fmaf(S.w, S.w, de.w);
          *pn = nu;
          *pd = de;
          dm = fmaxf(dm, fmaxf(fmaxf(de.x, de.y), fmaxf(de.z, de.w)));
        }
      }
    }
    if (rt.dmax_flag) block_max_atomic(dm, &A.dmax[b], red);
  }
}

// Quantised store of the field of every item as snapshot idx (used for the
// last forward field u^{nt}, which no later step reads).
__global__ void k_snap_store(const StepArgs A, const float *field, int idx) {
  const Geo &g = A.g;
  const int b = blockIdx.z, i = blockIdx.y;
  const int j0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (j0 >= g.SX) return;
  float4 v = *reinterpret_cast<const float4 *>(field + (long long)b * g.plane +
                                               (long long)(i + g.nb) * g.P + (j0 + g.CP));
  if (j0 + 1 >= g.nx) v.y = 0.f;
  if (j0 + 2 >= g.nx) v.z = 0.f;
  if (j0 + 3 >= g.nx) v.w = 0.f;
  float sdq, inv;
  snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + idx], sdq, inv);
  snap_store4(A.snap, ((long long)b * A.nsnap + idx) * g.pplane + (long long)i * g.SX + j0,
              A.snap_dtype, v, inv);
}

// c = (v dt)^2 on the padded grid of every sample, velocity copied from the
// nearest physical cell into the sponge, zero outside the padded domain.
__global__ void k_prep_c(const float *vel, float *c_all, Geo g, double dt) {
  const int smp = blockIdx.z, I = blockIdx.y;
  const float *v = vel + (long long)smp * g.nz * g.nx;
  float *c = c_all + (long long)smp * g.plane + (long long)I * g.P;
  const int i = min(max(I - g.nb, 0), g.nz - 1);
  for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < g.P; col += gridDim.x * blockDim.x) {
    float val = 0.f;
    if (col >= g.X0 && col < g.X0 + g.NX) {
      const int j = min(max(col - g.CP, 0), g.nx - 1);
      const double vd = (double)v[(long long)i * g.nx + j] * dt;
      val = (float)(vd * vd);
    }
    c[col] = val;
  }
}

// Range of a velocity array: out[0] = max (float bits), out[1] = min (float
// bits of the smallest positive value), out[2] = count of non-finite or
// non-positive values.
__global__ void k_vrange(const float *v, long long n, unsigned *out) {
  float mx = 0.f, mn = 3.0e38f;
  unsigned bad = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float x = v[e];
    if (!(x > 0.f) || !isfinite(x)) {
      ++bad;
    } else {
      mx = fmaxf(mx, x);
      mn = fminf(mn, x);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], __float_as_uint(mx));
    atomicMin(&out[1], __float_as_uint(mn));
    if (bad) atomicAdd(&out[2], bad);
  }
}

// ------------------------------------------------------------ launchers --

cudaError_t launch_step(int mode, const StepArgs &A, const StepRT &rt, int B, cudaStream_t st) {
  dim3 grid(A.g.ntx, A.g.ntz, B), block(32, STEP_THREADS / 32);
  if (mode == MODE_FWD)
    k_step<MODE_FWD><<<grid, block, 0, st>>>(A, rt);
  else if (mode == MODE_MODEL)
    k_step<MODE_MODEL><<<grid, block, 0, st>>>(A, rt);
  else if (mode == MODE_BORN)
    k_step<MODE_BORN><<<grid, block, 0, st>>>(A, rt);
  else
    k_step<MODE_BWD><<<grid, block, 0, st>>>(A, rt);
  return cudaGetLastError();
}

cudaError_t launch_snap_store(const StepArgs &A, const float *field, int idx, int B,
                              cudaStream_t st) {
  const int n4 = A.g.SX / 4;
  dim3 grid((n4 + 127) / 128, A.g.nz, B);
  k_snap_store<<<grid, 128, 0, st>>>(A, field, idx);
  return cudaGetLastError();
}

cudaError_t launch_prep_c(const float *vel, float *c_all, const Geo &g, double dt, int nsample,
                          cudaStream_t st) {
  dim3 grid((g.P + 255) / 256, g.NZ, nsample);
  k_prep_c<<<grid, 256, 0, st>>>(vel, c_all, g, dt);
  return cudaGetLastError();
}

cudaError_t launch_vrange(const float *v, long long n, unsigned *out, cudaStream_t st) {
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_vrange<<<(unsigned)blocks, 256, 0, st>>>(v, n, out);
  return cudaGetLastError();
}

}  // namespace rtm
