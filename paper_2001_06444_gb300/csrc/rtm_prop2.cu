// rtm_prop2.cu — two-time-step propagation kernel with TMA-staged tiles.
//
// One launch of k_step2 advances B grids (velocity sample x shot) by TWO
// leapfrog steps of the scheme of §2.2 Eq. 4 / §3 (see rtm_prop.cu for the
// scheme and its difference form).  A block owns a centre tile of
// C2Z x C2X points.  Three TMA bulk-tensor loads bring in
//   v^n with a halo of 8 (two stencil radii),
//   d^n and c with a halo of 4,
// out-of-range boxes filled with zeros by the copy engine, which realises the
// zero field beyond the padded grid.  Substep 1 computes (v^{n+1}, d^{n+1}) on
// the tile plus a 4-point ring ("extended" region) in shared memory, substep
// 2 computes (v^{n+2}, d^{n+2}) on the centre from it, and only the centre is
// written back: per two updates each point's v, d and c are read once and v
// and d written once (about 10 B per update instead of 20).
//
// The intermediate field v^{n+1} never leaves the chip, so everything the
// method does at step n+1 happens here too: source / receiver injection
// (every block whose extended region holds the cell injects into its own
// copy), trace recording, FP32 snapshot stores, and the imaging condition of
// Eq. 5.  Half-precision snapshots need the global max of the field first, so
// they are only taken from the launch OUTPUT (reduced here, stored by the next
// launch from its input tile); the host pairs steps so snapshot steps land on
// outputs.
//
// Most blocks lie clear of the absorbing band and run a body compiled with
// the interior update alone.  Blocks that reach the band stage the row and
// column sponge factors of their region in shared memory while the tiles
// load, and evaluate the sponge form at every point (it reproduces the
// interior update's bits where g = 1).
//
// Every wait is bounded: if the TMA transaction does not complete, the block
// raises an error flag (reported as RTM_ERR_TIMEOUT) and returns.
#include <cuda.h>

#include <atomic>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "rtm_common.h"
#include "rtm_launch.h"

namespace rtm {

namespace {

constexpr int C2X = 120, C2Z = 24;           // centre tile
constexpr int EX = C2X + 8, EZ = C2Z + 8;     // extended region (halo 4)
constexpr int VX = C2X + 16, VZ = C2Z + 16;   // v^n tile (halo 8)
constexpr int NTH = 256;                      // 32 x 8 threads
constexpr unsigned kTxBytes = (VX * VZ + 2 * EX * EZ) * 4;
constexpr unsigned long long kWaitNs = 1000000000ull;  // bound of a device-side wait: 1 s

struct Smem {
  float v0[VZ][VX];   // v^n            (TMA destination)
  float d[EZ][EX];    // d^n -> d^{n+1} -> d^{n+2} (TMA destination, updated in place)
  float c[EZ][EX];    // (v dt)^2       (TMA destination)
  float v1[EZ][EX];   // v^{n+1}
  unsigned long long bar;
  float red[NTH / 32];
  float gxs[EX];  // sponge factors of the extended region's columns ...
  float gzs[EZ];  // ... and rows (filled by blocks that reach the sponge)
};
static_assert(sizeof(float) * VX * VZ % 128 == 0, "tile offsets must stay 128-byte aligned");
static_assert(sizeof(float) * EX * EZ % 128 == 0, "tile offsets must stay 128-byte aligned");

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

// Paired FP32 arithmetic (two lanes per instruction).  Each lane rounds
// exactly like the scalar operation, so results equal the scalar kernel's;
// a - b is formed as fma(b, -1, a), which rounds once like a subtraction.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

// One leapfrog update of 4 consecutive points in difference form.
//   zc[0..8]: the 9 rows (centre row zc[4]) of the 4-column strip,
//   xl, xr:   the 4 columns left and right of the strip in the centre row,
//   dv, cv:   d^n and c at the strip,
//   SPONGE:   the block's region reaches the sponge: every point takes the
//             sponge form (which gives the interior formula's bits where
//             g = 1), with gzr the row's factor and gxs the strip's four (in
//             shared memory).  Blocks clear of the sponge compile in the
//             interior formula alone.  (Choosing between the two forms per
//             row measured slower.)
// Returns d^{n+1} (before injection); v^{n+1} = v^n + d^{n+1}.  Lanes are
// processed in pairs (0,1) and (2,3).
template <bool SPONGE>
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
      const float2 tx = __fadd2_rn(sub2(xm, ce), sub2(xp, ce));
      lap = __ffma2_rn(make_float2(k.ax[m - 1], k.ax[m - 1]), tx, lap);
      const float2 zm = l == 0 ? make_float2(zc[4 - m].x, zc[4 - m].y)
                               : make_float2(zc[4 - m].z, zc[4 - m].w);
      const float2 zp = l == 0 ? make_float2(zc[4 + m].x, zc[4 + m].y)
                               : make_float2(zc[4 + m].z, zc[4 + m].w);
      const float2 tz = __fadd2_rn(sub2(zm, ce), sub2(zp, ce));
      lap = __ffma2_rn(make_float2(k.az[m - 1], k.az[m - 1]), tz, lap);
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
  float sdq, inv;
  snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + idx], sdq, inv);
  const float4 S = snap_load4(A.snap, ((long long)b * A.nsnap + idx) * g.pplane +
                                          (long long)i * g.SX + j0, A.snap_dtype, sdq);
  const float *m = A.refl + (long long)i * g.nx + j0;
  if (j0 < g.nx) d.x = fmaf(c.x * __ldg(m), S.x, d.x);
  if (j0 + 1 < g.nx) d.y = fmaf(c.y * __ldg(m + 1), S.y, d.y);
  if (j0 + 2 < g.nx) d.z = fmaf(c.z * __ldg(m + 2), S.z, d.z);
  if (j0 + 3 < g.nx) d.w = fmaf(c.w * __ldg(m + 3), S.w, d.w);
  return d;
}

// Substep 1: (v^{n+1}, d^{n+1}) on the extended region, rows 4ty..4ty+3 and
// columns 4tx..4tx+3 of it, into S.d and S.v1.
template <int MODE, bool SPONGE>
__device__ __forceinline__ void substep1(Smem &S, const Step2Args &A, const Step2RT &rt, int b,
                                         int x0, int z0) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const Geo &g = A.g;
  float4 zc[12];
#pragma unroll
  for (int q = 0; q < 12; ++q)
    zc[q] = *reinterpret_cast<const float4 *>(&S.v0[4 * ty + q][4 + 4 * tx]);
  const int gcol = x0 - 4 + 4 * tx;
  const float *gxs = &S.gxs[4 * tx];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int er = 4 * ty + r;
    const float4 xl = *reinterpret_cast<const float4 *>(&S.v0[er + 4][4 * tx]);
    const float4 xr = *reinterpret_cast<const float4 *>(&S.v0[er + 4][8 + 4 * tx]);
    const float4 dv = *reinterpret_cast<const float4 *>(&S.d[er][4 * tx]);
    const float4 cv = *reinterpret_cast<const float4 *>(&S.c[er][4 * tx]);
    const float gzr = SPONGE ? S.gzs[er] : 1.f;
    const float4 nd = update4<SPONGE>(&zc[r], xl, xr, dv, cv, A.k, gzr, gxs);
    *reinterpret_cast<float4 *>(&S.d[er][4 * tx]) = nd;
    if (MODE != MODE_BORN) {
      const float4 ce = zc[r + 4];
      *reinterpret_cast<float4 *>(&S.v1[er][4 * tx]) =
          make_float4(ce.x + nd.x, ce.y + nd.y, ce.z + nd.z, ce.w + nd.w);
    }
  }
  // Born modelling: the source term joins each row's new difference, in a
  // second pass over this thread's own rows (fewer registers live in the
  // stencil loop), then v^{n+1} = v^n + d^{n+1}
  if (MODE == MODE_BORN) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int er = 4 * ty + r;
      const float4 cv = *reinterpret_cast<const float4 *>(&S.c[er][4 * tx]);
      const float4 nd = born_inject4(A, b, rt.img_mid_idx, z0 - 4 + er - g.nb, gcol - g.CP,
                                     *reinterpret_cast<const float4 *>(&S.d[er][4 * tx]), cv);
      const float4 ce = zc[r + 4];
      *reinterpret_cast<float4 *>(&S.d[er][4 * tx]) = nd;
      *reinterpret_cast<float4 *>(&S.v1[er][4 * tx]) =
          make_float4(ce.x + nd.x, ce.y + nd.y, ce.z + nd.z, ce.w + nd.w);
    }
  }
}

// Substep 2: d^{n+2} (res, before injection) and v^{n+1} (cen) on the
// centre, rows 3ty..3ty+2 and columns 4tx..4tx+3 of it.
template <int MODE, bool SPONGE>
__device__ __forceinline__ void substep2(const Smem &S, const Step2Args &A, const Step2RT &rt,
                                         int b, int x0, int z0, float4 (&res)[3],
                                         float4 (&cen)[3]) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const Geo &g = A.g;
  float4 zc[11];
#pragma unroll
  for (int q = 0; q < 11; ++q)
    zc[q] = *reinterpret_cast<const float4 *>(&S.v1[3 * ty + q][4 + 4 * tx]);
  const int gcol = x0 + 4 * tx;
  const float *gxs = &S.gxs[4 + 4 * tx];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int er = 4 + 3 * ty + r;
    const float4 xl = *reinterpret_cast<const float4 *>(&S.v1[er][4 * tx]);
    const float4 xr = *reinterpret_cast<const float4 *>(&S.v1[er][8 + 4 * tx]);
    const float4 dv = *reinterpret_cast<const float4 *>(&S.d[er][4 + 4 * tx]);
    const float4 cv = *reinterpret_cast<const float4 *>(&S.c[er][4 + 4 * tx]);
    const float gzr = SPONGE ? S.gzs[er] : 1.f;
    res[r] = update4<SPONGE>(&zc[r], xl, xr, dv, cv, A.k, gzr, gxs);
    cen[r] = zc[r + 4];
  }
  if (MODE == MODE_BORN) {  // as in substep 1
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float4 cv = *reinterpret_cast<const float4 *>(&S.c[4 + 3 * ty + r][4 + 4 * tx]);
      res[r] = born_inject4(A, b, rt.img_out_idx, z0 + 3 * ty + r - g.nb, gcol - g.CP, res[r], cv);
    }
  }
}

}  // namespace

template <int MODE>
__global__ void __launch_bounds__(NTH, 3)
    k_step2(const __grid_constant__ CUtensorMap map_v, const __grid_constant__ CUtensorMap map_d,
            const __grid_constant__ CUtensorMap map_c, const Step2Args A, const Step2RT rt) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA destinations must be 128-byte aligned: align the base explicitly
  Smem &S = *reinterpret_cast<Smem *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int b = blockIdx.z;
  const Geo &g = A.g;
  const int x0 = blockIdx.x * C2X, z0 = blockIdx.y * C2Z;
  const int smp = A.one_sample ? 0 : A.item_sample[b];  // c tile's sample, before the copies
  const int shot = A.item_shot[b];

  // blocks whose extended region stays clear of the sponge (g = 1 there)
  const bool interior = (z0 - 4 >= g.nb) && (z0 + C2Z + 4 <= g.NZ - g.nb) &&
                        (x0 - 4 >= g.X0 + g.nb) && (x0 + C2X + 4 <= g.X0 + g.NX - g.nb);

  // ---- 1. TMA: v^n (halo 8), d^n and c (halo 4) ----------------------------
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.bar)), "r"(1)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&S.bar)),
                 "r"(kTxBytes)
                 : "memory");
    tma_load_3d(&S.v0[0][0], &map_v, x0 - 8, z0 - 8, b, &S.bar);
    tma_load_3d(&S.d[0][0], &map_d, x0 - 4, z0 - 4, b, &S.bar);
    tma_load_3d(&S.c[0][0], &map_c, x0 - 4, z0 - 4, smp, &S.bar);
  }
  if (!interior) {  // the extended region's sponge factors, edge-clamped
    if (tid < EX) S.gxs[tid] = A.gx[min(max(x0 - 4 + tid, 0), g.P - 1)];
    if (tid < EZ) S.gzs[tid] = A.gz[min(max(z0 - 4 + tid, 0), g.NZ - 1)];
  }
  // backward imaging launches: start pulling this thread's num, den and
  // snapshot rows into L2 while the tile loads and the stencil run
  if (MODE == MODE_BWD && (rt.img_mid_idx >= 0 || rt.img_out_idx >= 0) && tx < C2X / 4) {
    const int j0 = x0 + 4 * tx - g.CP;
    if (j0 >= 0 && j0 < g.SX) {
      const int esz = A.snap_dtype == 0 ? 4 : 2;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int i = z0 + 3 * ty + r - g.nb;
        if (i >= 0 && i < g.nz) {
          const long long po = (long long)b * g.pplane + (long long)i * g.SX + j0;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(A.num + po));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(A.den + po));
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int idx = u == 0 ? rt.img_mid_idx : rt.img_out_idx;
            if (idx >= 0) {
              const long long so = ((long long)b * A.nsnap + idx) * g.pplane + (long long)i * g.SX + j0;
              asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(A.snap) +
                                                             so * esz));
            }
          }
        }
      }
    }
  }
  if (!mbar_wait_bounded(&S.bar, 0, kWaitNs)) {
    if (tid == 0) atomicExch(A.err, 1);
    // let the copies in flight land (bounded) before the block exits
    mbar_wait_bounded(&S.bar, 0, kWaitNs);
    return;
  }
  if (!interior) __syncthreads();  // (block-uniform) the sponge factors are in place

  const bool wide = tx < C2X / 4;  // threads that own centre columns

  // deferred half-precision snapshot of the INPUT field v^n (its max was
  // reduced by the launch that produced it)
  if (MODE == MODE_FWD && rt.snap_in_idx >= 0 && wide) {
    float sdq, inv;
    snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + rt.snap_in_idx], sdq, inv);
    const int j0 = x0 + 4 * tx - g.CP;
    if (j0 >= 0 && j0 < g.SX) {
      const long long base = ((long long)b * A.nsnap + rt.snap_in_idx) * g.pplane + j0;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int i = z0 + 3 * ty + r - g.nb;
        if (i >= 0 && i < g.nz) {
          float4 v = *reinterpret_cast<const float4 *>(&S.v0[8 + 3 * ty + r][8 + 4 * tx]);
          if (j0 + 1 >= g.nx) v.y = 0.f;
          if (j0 + 2 >= g.nx) v.z = 0.f;
          if (j0 + 3 >= g.nx) v.w = 0.f;
          snap_store4(A.snap, base + (long long)i * g.SX, A.snap_dtype, v, inv);
        }
      }
    }
  }

  // ---- 2. substep 1 on the extended region (rows 4ty..4ty+3, cols 4tx..) --
  // (blocks clear of the sponge run a body without the sponge formula; a
  // warp whose rows lie 4 or more past the grid skips: substep 2 reads rows
  // up to 4 past its own, and computes none below the grid's last row + 1)
  if (interior)
    substep1<MODE, false>(S, A, rt, b, x0, z0);
  else if (z0 - 4 + 4 * ty < g.NZ + 4)
    substep1<MODE, true>(S, A, rt, b, x0, z0);
  __syncthreads();

  // injection at step t1 into every cell of the extended region: add to
  // d^{n+1}, then re-form v^{n+1} = v^n + d^{n+1} at those cells (the same
  // rounding order as the single-step kernel)
  {
    const int tile = blockIdx.y * g.ntx2 + blockIdx.x;
    if (MODE == MODE_FWD || MODE == MODE_MODEL) {
      const int sr = A.src_row[shot] - (z0 - 4), sc = A.src_col[shot] - (x0 - 4);
      if (sr >= 0 && sr < EZ && sc >= 0 && sc < EX) {  // block-uniform
        if (tid == 0) {
          S.d[sr][sc] += S.c[sr][sc] * (A.wav[rt.t1] * A.src_scale);
          S.v1[sr][sc] = S.v0[sr + 4][sc + 4] + S.d[sr][sc];
        }
        __syncthreads();
      }
    } else if (MODE == MODE_BWD) {
      const int p0 = A.rext_ptr[tile], p1 = A.rext_ptr[tile + 1];
      if (p1 > p0) {  // block-uniform
        const float *dsamp = A.seis + ((long long)shot * A.nt + rt.t1) * A.nrec;
        for (int e = p0 + tid; e < p1; e += NTH) {
          const int2 en = A.rext_ent[e];
          const int er = en.x / EX, ec = en.x - er * EX;
          atomicAdd(&S.d[er][ec], S.c[er][ec] * dsamp[en.y]);
        }
        __syncthreads();
        for (int e = p0 + tid; e < p1; e += NTH) {
          const int2 en = A.rext_ent[e];
          const int er = en.x / EX, ec = en.x - er * EX;
          S.v1[er][ec] = S.v0[er + 4][ec + 4] + S.d[er][ec];  // duplicates write equal values
        }
        __syncthreads();
      }
    }
  }

  // step-(n+1) work on the centre: recording, FP32 snapshot, imaging
  if (MODE == MODE_MODEL || MODE == MODE_BORN) {
    const int tile = blockIdx.y * g.ntx2 + blockIdx.x;
    const int p0 = A.rcen_ptr[tile], p1 = A.rcen_ptr[tile + 1];
    float *ro = A.rec_out + ((long long)b * A.nt + rt.t1) * A.nrec;
    for (int e = p0 + tid; e < p1; e += NTH) {
      const int2 en = A.rcen_ent[e];
      ro[en.y] = (&S.v1[0][0])[en.x];
    }
  }
  const int j0 = x0 + 4 * tx - g.CP;  // physical column of this thread's strip
  const bool jok = wide && j0 >= 0 && j0 < g.SX;
  float dm = 0.f;  // running max of den for the max-den reduction
  if (MODE == MODE_FWD && rt.snap_mid_idx >= 0 && jok) {
    const long long base = ((long long)b * A.nsnap + rt.snap_mid_idx) * g.pplane + j0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int i = z0 + 3 * ty + r - g.nb;
      if (i >= 0 && i < g.nz) {
        float4 v = *reinterpret_cast<const float4 *>(&S.v1[4 + 3 * ty + r][4 + 4 * tx]);
        if (j0 + 1 >= g.nx) v.y = 0.f;
        if (j0 + 2 >= g.nx) v.z = 0.f;
        if (j0 + 3 >= g.nx) v.w = 0.f;
        snap_store4(A.snap, base + (long long)i * g.SX, 0, v, 1.f);
      }
    }
  }
  if (MODE == MODE_BWD && rt.img_mid_idx >= 0 && jok) {
    float sdq, inv;
    snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + rt.img_mid_idx], sdq, inv);
    const long long sbase = ((long long)b * A.nsnap + rt.img_mid_idx) * g.pplane + j0;
    const long long pbase = (long long)b * g.pplane + j0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int i = z0 + 3 * ty + r - g.nb;
      if (i >= 0 && i < g.nz) {
        const float4 w = *reinterpret_cast<const float4 *>(&S.v1[4 + 3 * ty + r][4 + 4 * tx]);
        const float4 Sv = snap_load4(A.snap, sbase + (long long)i * g.SX, A.snap_dtype, sdq);
        float4 *pn = reinterpret_cast<float4 *>(A.num + pbase + (long long)i * g.SX);
        float4 *pd = reinterpret_cast<float4 *>(A.den + pbase + (long long)i * g.SX);
        float4 nu = *pn, de = *pd;
        nu.x = fmaf(Sv.x, w.x, nu.x);
        nu.y = fmaf(Sv.y, w.y, nu.y);
        nu.z = fmaf(Sv.z, w.z, nu.z);
        nu.w = fmaf(Sv.w, w.w, nu.w);
        de.x = fmaf(Sv.x, Sv.x, de.x);
        de.y = fmaf(Sv.y, Sv.y, de.y);
        de.z = fmaf(Sv.z, Sv.z, de.z);
        de.w = fmaf(Sv.w, Sv.w, de.w);
        *pn = nu;
        *pd = de;
        dm = fmaxf(dm, fmaxf(fmaxf(de.x, de.y), fmaxf(de.z, de.w)));
      }
    }
  }
  if (MODE == MODE_BWD && rt.dmax_flag == 1) block_max_atomic(dm, &A.dmax[b], S.red);

  // ---- 3. substep 2 on the centre (rows 3ty..3ty+2, cols 4tx..4tx+3) -------
  float4 res[3];
  float4 cen[3];
  if (wide) {
    if (interior) {
      substep2<MODE, false>(S, A, rt, b, x0, z0, res, cen);
    } else if (z0 + 3 * ty < g.NZ) {
      substep2<MODE, true>(S, A, rt, b, x0, z0, res, cen);
    } else {  // rows past the grid: nothing of them is stored
#pragma unroll
      for (int r = 0; r < 3; ++r) res[r] = cen[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }

  // injection at step t2 on the centre (staged through the d tile)
  {
    const int tile = blockIdx.y * g.ntx2 + blockIdx.x;
    bool stage = false;
    int sr = -1, sc = -1, p0 = 0, p1 = 0;
    if (MODE == MODE_FWD || MODE == MODE_MODEL) {
      sr = A.src_row[shot] - z0;
      sc = A.src_col[shot] - x0;
      if (sr >= 0 && sr < C2Z && sc >= 0 && sc < C2X)
        stage = true;
      else
        sr = -1;
    }
    if (MODE != MODE_FWD) {
      p0 = A.rcen_ptr[tile];
      p1 = A.rcen_ptr[tile + 1];
      if (p1 > p0) stage = true;
    }
    if (stage) {
      __syncthreads();  // all reads of S.d for substep 2 are done
      if (wide) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
          *reinterpret_cast<float4 *>(&S.d[4 + 3 * ty + r][4 + 4 * tx]) = res[r];
      }
      __syncthreads();
      if (MODE == MODE_FWD || MODE == MODE_MODEL) {
        if (sr >= 0 && tid == 0)
          S.d[4 + sr][4 + sc] += S.c[4 + sr][4 + sc] * (A.wav[rt.t2] * A.src_scale);
      } else if (MODE == MODE_BWD) {
        const float *dsamp = A.seis + ((long long)shot * A.nt + rt.t2) * A.nrec;
        for (int e = p0 + tid; e < p1; e += NTH) {
          const int2 en = A.rcen_ent[e];
          atomicAdd(&(&S.d[0][0])[en.x], (&S.c[0][0])[en.x] * dsamp[en.y]);
        }
      }
      __syncthreads();
      if (MODE == MODE_MODEL || MODE == MODE_BORN) {
        float *ro = A.rec_out + ((long long)b * A.nt + rt.t2) * A.nrec;
        for (int e = p0 + tid; e < p1; e += NTH) {
          const int2 en = A.rcen_ent[e];
          ro[en.y] = (&S.v1[0][0])[en.x] + (&S.d[0][0])[en.x];  // v^{n+2} = v^{n+1} + d^{n+2}
        }
      }
      if (wide) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
          res[r] = *reinterpret_cast<const float4 *>(&S.d[4 + 3 * ty + r][4 + 4 * tx]);
      }
    }
  }

  // ---- 4. write d^{n+2}, v^{n+2}; step-(n+2) work ----------------------------
  float mx = 0.f;
  if (wide) {
    const int col = x0 + 4 * tx;
    float *vo = A.v_out + (long long)b * g.plane;
    float *dq = A.d_out + (long long)b * g.plane;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int row = z0 + 3 * ty + r;
      const float4 nv = make_float4(cen[r].x + res[r].x, cen[r].y + res[r].y, cen[r].z + res[r].z,
                                    cen[r].w + res[r].w);
      if (row < g.NZ && col < g.P) {
        const long long o = (long long)row * g.P + col;
        *reinterpret_cast<float4 *>(dq + o) = res[r];
        *reinterpret_cast<float4 *>(vo + o) = nv;
      }
      res[r] = nv;  // from here on res holds v^{n+2}
      const int i = row - g.nb;
      if (i >= 0 && i < g.nz) {
        if (MODE == MODE_FWD && rt.max_out_idx >= 0) {
#pragma unroll
          for (int l = 0; l < 4; ++l)
            if (j0 + l >= 0 && j0 + l < g.nx) mx = fmaxf(mx, fabsf(lane4(nv, l)));
        }
        if (MODE == MODE_FWD && rt.snap_out_idx >= 0 && jok) {
          float4 v = nv;
          if (j0 + 1 >= g.nx) v.y = 0.f;
          if (j0 + 2 >= g.nx) v.z = 0.f;
          if (j0 + 3 >= g.nx) v.w = 0.f;
          snap_store4(A.snap, ((long long)b * A.nsnap + rt.snap_out_idx) * g.pplane +
                                  (long long)i * g.SX + j0,
                      0, v, 1.f);
        }
        if (MODE == MODE_BWD && rt.img_out_idx >= 0 && jok) {
          float sdq, inv;
          snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + rt.img_out_idx], sdq, inv);
          const float4 Sv =
              snap_load4(A.snap, ((long long)b * A.nsnap + rt.img_out_idx) * g.pplane +
                                     (long long)i * g.SX + j0,
                         A.snap_dtype, sdq);
          const long long po = (long long)b * g.pplane + (long long)i * g.SX + j0;
          float4 *pn = reinterpret_cast<float4 *>(A.num + po);
          float4 *pd = reinterpret_cast<float4 *>(A.den + po);
          float4 nu = *pn, de = *pd;
          nu.x = fmaf(Sv.x, nv.x, nu.x);
          nu.y = fmaf(Sv.y, nv.y, nu.y);
          nu.z = fmaf(Sv.z, nv.z, nu.z);
          nu.w = fmaf(Sv.w, nv.w, nu.w);
          de.x = fmaf(Sv.x, Sv.x, de.x);
          de.y = fmaf(Sv.y, Sv.y, de.y);
          de.z = fmaf(Sv.z, Sv.z, de.z);
          de.w = fmaf(Sv.w, Sv.w, de.w);
          *pn = nu;
          *pd = de;
          dm = fmaxf(dm, fmaxf(fmaxf(de.x, de.y), fmaxf(de.z, de.w)));
        }
      }
    }
  }
  if (MODE == MODE_FWD && rt.max_out_idx >= 0)
    block_max_atomic(mx, &A.smax[(long long)b * A.nsnap + rt.max_out_idx], S.red);
  if (MODE == MODE_BWD && rt.dmax_flag == 2) block_max_atomic(dm, &A.dmax[b], S.red);
}

// Self-test of the bounded wait: one block arms an mbarrier for bytes that no
// copy will deliver (nothing is issued), so its wait runs out after the bound
// and it raises the flag, exactly as k_step2 does when a TMA transaction never
// completes.  Touches nothing but its own shared memory and the flag.
__global__ void k_wait_probe(int *flag, unsigned long long ns) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar)),
                 "r"(16u)
                 : "memory");
  if (!mbar_wait_bounded(&bar, 0, ns) && threadIdx.x == 0) atomicExch(flag, 1);
}

cudaError_t launch_wait_probe(int *flag, unsigned long long ns, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(flag, ns);
  return cudaGetLastError();
}

size_t step2_smem_bytes() { return sizeof(Smem) + 128; }
int step2_tile_x() { return C2X; }
int step2_tile_z() { return C2Z; }
int step2_ext() { return 4; }

cudaError_t launch_step2(int mode, const CUtensorMap &mv, const CUtensorMap &md,
                         const CUtensorMap &mc, const Step2Args &A, const Step2RT &rt, int B,
                         cudaStream_t st) {
  // the shared-memory opt-in, once per mode (launches come from several
  // request threads; setting it twice is harmless, the flags are atomic)
  static std::atomic<bool> attr_set[4];
  const size_t smem = step2_smem_bytes();
  dim3 grid(A.g.ntx2, A.g.ntz2, B), block(32, NTH / 32);
  auto launch = [&](auto kernel, int slot) -> cudaError_t {
    if (!attr_set[slot].load(std::memory_order_acquire)) {
      const cudaError_t e =
          cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_set[slot].store(true, std::memory_order_release);
    }
    kernel<<<grid, block, smem, st>>>(mv, md, mc, A, rt);
    return cudaGetLastError();
  };
  switch (mode) {
    case MODE_FWD: return launch(k_step2<MODE_FWD>, 0);
    case MODE_MODEL: return launch(k_step2<MODE_MODEL>, 1);
    case MODE_BWD: return launch(k_step2<MODE_BWD>, 2);
    case MODE_BORN: return launch(k_step2<MODE_BORN>, 3);
  }
  return cudaErrorInvalidValue;
}

}  // namespace rtm
