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
#include "rtm_step2_dev.cuh"

namespace rtm {

namespace {

using namespace s2;

constexpr int C2Z = 24;                       // centre tile height
constexpr int EZ = C2Z + 8;                   // extended region height (halo 4)
constexpr int VZ = C2Z + 16;                  // v^n tile height (halo 8)
constexpr unsigned kTxBytes = (VX * VZ + 2 * EX * EZ) * 4;

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

// Substep 1: (v^{n+1}, d^{n+1}) on the extended region, rows 4ty..4ty+3 and
// columns 4tx..4tx+3 of it, into S.d and S.v1.
template <int MODE, bool SPONGE, bool ISO>
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
    const float4 nd = update4<SPONGE, ISO>(&zc[r], xl, xr, dv, cv, A.k, gzr, gxs);
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
template <int MODE, bool SPONGE, bool ISO>
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
    res[r] = update4<SPONGE, ISO>(&zc[r], xl, xr, dv, cv, A.k, gzr, gxs);
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
  const Geo &g = A.g;
  // snake order: with `reverse` the launch walks the tiles from the end
  const bool rev = rt.reverse != 0;
  const int bx = rev ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
  const int by = rev ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y;
  const int b = rev ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z;
  const int x0 = bx * C2X, z0 = by * C2Z;
  const int smp = A.one_sample ? 0 : A.item_sample[b];  // c tile's sample, before the copies
  const int shot = A.item_shot[b];
#ifdef RTM_DEBUG
  // block-level indices of the debug checks (the copy engine zero-fills a
  // plane outside the c map, so a bad sample is recorded, not read)
  const bool shot_ok = RTM_IN(b, A.len.items, A.err) && RTM_IN(smp, A.len.nsample, A.err) &&
                       RTM_IN(shot, A.len.nshot, A.err) &&
                       RTM_IN(by * g.ntx2 + bx + 1, g.ntx2 * g.ntz2 + 1, A.err);
#else
  constexpr bool shot_ok = true;
#endif

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
  // L2 prefetch of the v and d rows of the tile that the block `ahead`
  // launches later will load (it takes this block's place on the SM when a
  // resident block retires), one bulk prefetch per row, clipped to the plane
  if (rt.ahead > 0 && tid < VZ + EZ) {
    const long long nblk = (long long)gridDim.x * gridDim.y * gridDim.z;
    const long long lin =
        blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z) +
        rt.ahead;
    if (lin < nblk) {
      int px = (int)(lin % gridDim.x);
      const long long q = lin / gridDim.x;
      int py = (int)(q % gridDim.y), pz = (int)(q / gridDim.y);
      if (rev) {
        px = gridDim.x - 1 - px;
        py = gridDim.y - 1 - py;
        pz = gridDim.z - 1 - pz;
      }
      const bool vrow = tid < VZ;
      const int row = vrow ? py * C2Z - 8 + tid : py * C2Z - 4 + (tid - VZ);
      const int c0 = max(px * C2X - (vrow ? 8 : 4), 0);
      const int c1 = min(px * C2X - (vrow ? 8 : 4) + (vrow ? VX : EX), g.P);
      if (row >= 0 && row < g.NZ && c1 > c0) {
        const float *src = (vrow ? A.v_in : A.d_in) + (long long)pz * g.plane +
                           (long long)row * g.P + c0;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src),
                     "r"((unsigned)(c1 - c0) * 4u)
                     : "memory");
      }
    }
  }
  if (!interior) {  // the extended region's sponge factors, edge-clamped
    if (tid < EX) S.gxs[tid] = A.gx[min(max(x0 - 4 + tid, 0), g.P - 1)];
    if (tid < EZ) S.gzs[tid] = A.gz[min(max(z0 - 4 + tid, 0), g.NZ - 1)];
  }
  // backward imaging launches: start pulling this thread's num, den and
  // snapshot rows into L2 while the tile loads and the stencil run
  if (MODE == MODE_BWD && (rt.img_mid_idx >= 0 || rt.img_out_idx >= 0 || rt.img_in_idx >= 0) &&
      tx < C2X / 4) {
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
          for (int u = 0; u < 3; ++u) {
            const int idx = u == 0 ? rt.img_mid_idx : (u == 1 ? rt.img_out_idx : rt.img_in_idx);
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
  float dm = 0.f;                  // running max of den for the max-den reduction

  // imaging with the INPUT field v^n (the centre of the v^n tile)
  if (MODE == MODE_BWD && rt.img_in_idx >= 0 && wide &&
      RTM_IN((long long)b * A.nsnap + rt.img_in_idx, A.len.smax, A.err)) {
    const int j0 = x0 + 4 * tx - g.CP;
    if (j0 >= 0 && j0 < g.SX) {
      float sdq, inv;
      snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + rt.img_in_idx], sdq, inv);
      const long long sbase = ((long long)b * A.nsnap + rt.img_in_idx) * g.pplane + j0;
      const long long pbase = (long long)b * g.pplane + j0;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int i = z0 + 3 * ty + r - g.nb;
        if (i >= 0 && i < g.nz && RTM_IN(sbase + (long long)i * g.SX + 3, A.len.snap, A.err) &&
            RTM_IN(pbase + (long long)i * g.SX + 3, A.len.items * g.pplane, A.err)) {
          const float4 w = *reinterpret_cast<const float4 *>(&S.v0[8 + 3 * ty + r][8 + 4 * tx]);
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
  }
  if (MODE == MODE_BWD && rt.dmax_flag == 3)
    block_max_atomic(dm, &A.dmax[RTM_IN(b, A.len.items, A.err) ? b : 0], S.red);

  // deferred half-precision snapshot of the INPUT field v^n (its max was
  // reduced by the launch that produced it)
  if (MODE == MODE_FWD && rt.snap_in_idx >= 0 && wide) {
    float sdq, inv;
    snap_scale(A.snap_dtype,
               A.smax[RTM_IN((long long)b * A.nsnap + rt.snap_in_idx, A.len.smax, A.err)
                          ? (long long)b * A.nsnap + rt.snap_in_idx : 0],
               sdq, inv);
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
          if (RTM_IN(base + (long long)i * g.SX + 3, A.len.snap, A.err))
            snap_store4(A.snap, base + (long long)i * g.SX, A.snap_dtype, v, inv);
        }
      }
    }
  }

  // ---- 2. substep 1 on the extended region (rows 4ty..4ty+3, cols 4tx..) --
  // (blocks clear of the sponge run a body without the sponge formula; a
  // warp whose rows lie 4 or more past the grid skips: substep 2 reads rows
  // up to 4 past its own, and computes none below the grid's last row + 1)
  if (A.k.iso) {
    if (interior)
      substep1<MODE, false, true>(S, A, rt, b, x0, z0);
    else if (z0 - 4 + 4 * ty < g.NZ + 4)
      substep1<MODE, true, true>(S, A, rt, b, x0, z0);
  } else {
    if (interior)
      substep1<MODE, false, false>(S, A, rt, b, x0, z0);
    else if (z0 - 4 + 4 * ty < g.NZ + 4)
      substep1<MODE, true, false>(S, A, rt, b, x0, z0);
  }
  __syncthreads();

  // injection at step t1 into every cell of the extended region: add to
  // d^{n+1}, then re-form v^{n+1} = v^n + d^{n+1} at those cells (the same
  // rounding order as the single-step kernel)
  {
    const int tile = by * g.ntx2 + bx;
    if (MODE == MODE_FWD || MODE == MODE_MODEL) {
      const int sr = A.src_row[shot] - (z0 - 4), sc = A.src_col[shot] - (x0 - 4);
      if (sr >= 0 && sr < EZ && sc >= 0 && sc < EX) {  // block-uniform
        if (tid == 0 && RTM_IN(rt.t1, A.nt, A.err)) {
          S.d[sr][sc] += S.c[sr][sc] * (A.wav[rt.t1] * A.src_scale);
          S.v1[sr][sc] = S.v0[sr + 4][sc + 4] + S.d[sr][sc];
        }
        __syncthreads();
      }
    } else if (MODE == MODE_BWD) {
      const int p0 = shot_ok ? A.rext_ptr[tile] : 0, p1 = shot_ok ? A.rext_ptr[tile + 1] : 0;
      if (p1 > p0) {  // block-uniform
        const long long d0 = ((long long)shot * A.nt + rt.t1) * A.nrec;
        const float *dsamp = A.seis + d0;
        for (int e = p0 + tid; e < p1; e += NTH) {
          if (!RTM_IN(e, A.len.rent, A.err)) continue;
          const int2 en = A.rext_ent[e];
          const int er = en.x / EX, ec = en.x - er * EX;
          if (RTM_IN(en.x, EX * EZ, A.err) && RTM_IN(en.y, A.nrec, A.err) &&
              RTM_IN(d0 + en.y, A.len.nshot * A.nt * A.nrec, A.err))
            atomicAdd(&S.d[er][ec], S.c[er][ec] * dsamp[en.y]);
        }
        __syncthreads();
        for (int e = p0 + tid; e < p1; e += NTH) {
          if (!RTM_IN(e, A.len.rent, A.err) || !RTM_IN(A.rext_ent[e].x, EX * EZ, A.err)) continue;
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
    const int tile = by * g.ntx2 + bx;
    const int p0 = shot_ok ? A.rcen_ptr[tile] : 0, p1 = shot_ok ? A.rcen_ptr[tile + 1] : 0;
    const long long r0 = ((long long)b * A.nt + rt.t1) * A.nrec;
    float *ro = A.rec_out + r0;
    for (int e = p0 + tid; e < p1; e += NTH) {
      if (!RTM_IN(e, A.len.rcen, A.err)) continue;
      const int2 en = A.rcen_ent[e];
      if (RTM_IN(en.x, EX * EZ, A.err) && RTM_IN(r0 + en.y, A.len.rec_out, A.err))
        ro[en.y] = (&S.v1[0][0])[en.x];
    }
  }
  const int j0 = x0 + 4 * tx - g.CP;  // physical column of this thread's strip
  const bool jok = wide && j0 >= 0 && j0 < g.SX;
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
        if (RTM_IN(base + (long long)i * g.SX + 3, A.len.snap, A.err))
          snap_store4(A.snap, base + (long long)i * g.SX, 0, v, 1.f);
      }
    }
  }
  if (MODE == MODE_BWD && rt.img_mid_idx >= 0 && jok &&
      RTM_IN((long long)b * A.nsnap + rt.img_mid_idx, A.len.smax, A.err)) {
    float sdq, inv;
    snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + rt.img_mid_idx], sdq, inv);
    const long long sbase = ((long long)b * A.nsnap + rt.img_mid_idx) * g.pplane + j0;
    const long long pbase = (long long)b * g.pplane + j0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int i = z0 + 3 * ty + r - g.nb;
      if (i >= 0 && i < g.nz && RTM_IN(sbase + (long long)i * g.SX + 3, A.len.snap, A.err) &&
          RTM_IN(pbase + (long long)i * g.SX + 3, A.len.items * g.pplane, A.err)) {
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
  if (MODE == MODE_BWD && rt.dmax_flag == 1)
    block_max_atomic(dm, &A.dmax[RTM_IN(b, A.len.items, A.err) ? b : 0], S.red);

  // ---- 3. substep 2 on the centre (rows 3ty..3ty+2, cols 4tx..4tx+3) -------
  float4 res[3];
  float4 cen[3];
  if (wide) {
    if (interior) {
      if (A.k.iso)
        substep2<MODE, false, true>(S, A, rt, b, x0, z0, res, cen);
      else
        substep2<MODE, false, false>(S, A, rt, b, x0, z0, res, cen);
    } else if (z0 + 3 * ty < g.NZ) {
      if (A.k.iso)
        substep2<MODE, true, true>(S, A, rt, b, x0, z0, res, cen);
      else
        substep2<MODE, true, false>(S, A, rt, b, x0, z0, res, cen);
    } else {  // rows past the grid: nothing of them is stored
#pragma unroll
      for (int r = 0; r < 3; ++r) res[r] = cen[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }

  // injection at step t2 on the centre (staged through the d tile)
  {
    const int tile = by * g.ntx2 + bx;
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
    if (MODE != MODE_FWD && shot_ok) {
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
        if (sr >= 0 && tid == 0 && RTM_IN(rt.t2, A.nt, A.err))
          S.d[4 + sr][4 + sc] += S.c[4 + sr][4 + sc] * (A.wav[rt.t2] * A.src_scale);
      } else if (MODE == MODE_BWD) {
        const long long d0 = ((long long)shot * A.nt + rt.t2) * A.nrec;
        const float *dsamp = A.seis + d0;
        for (int e = p0 + tid; e < p1; e += NTH) {
          if (!RTM_IN(e, A.len.rcen, A.err)) continue;
          const int2 en = A.rcen_ent[e];
          if (RTM_IN(en.x, EX * EZ, A.err) && RTM_IN(en.y, A.nrec, A.err) &&
              RTM_IN(d0 + en.y, A.len.nshot * A.nt * A.nrec, A.err))
            atomicAdd(&(&S.d[0][0])[en.x], (&S.c[0][0])[en.x] * dsamp[en.y]);
        }
      }
      __syncthreads();
      if (MODE == MODE_MODEL || MODE == MODE_BORN) {
        const long long r0 = ((long long)b * A.nt + rt.t2) * A.nrec;
        float *ro = A.rec_out + r0;
        for (int e = p0 + tid; e < p1; e += NTH) {
          if (!RTM_IN(e, A.len.rcen, A.err)) continue;
          const int2 en = A.rcen_ent[e];
          if (RTM_IN(en.x, EX * EZ, A.err) && RTM_IN(r0 + en.y, A.len.rec_out, A.err))
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
      if (row < g.NZ && col < g.P &&
          RTM_IN((long long)b * g.plane + (long long)row * g.P + col + 3, A.len.items * g.plane,
                 A.err)) {
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
        if (MODE == MODE_FWD && rt.snap_out_idx >= 0 && jok &&
            RTM_IN(((long long)b * A.nsnap + rt.snap_out_idx) * g.pplane + (long long)i * g.SX + j0 + 3,
                   A.len.snap, A.err)) {
          float4 v = nv;
          if (j0 + 1 >= g.nx) v.y = 0.f;
          if (j0 + 2 >= g.nx) v.z = 0.f;
          if (j0 + 3 >= g.nx) v.w = 0.f;
          snap_store4(A.snap, ((long long)b * A.nsnap + rt.snap_out_idx) * g.pplane +
                                  (long long)i * g.SX + j0,
                      0, v, 1.f);
        }
        if (MODE == MODE_BWD && rt.img_out_idx >= 0 && jok &&
            RTM_IN((long long)b * A.nsnap + rt.img_out_idx, A.len.smax, A.err) &&
            RTM_IN(((long long)b * A.nsnap + rt.img_out_idx) * g.pplane + (long long)i * g.SX + j0 + 3,
                   A.len.snap, A.err) &&
            RTM_IN((long long)b * g.pplane + (long long)i * g.SX + j0 + 3, A.len.items * g.pplane,
                   A.err)) {
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
  if (MODE == MODE_FWD && rt.max_out_idx >= 0) {
    const long long k = (long long)b * A.nsnap + rt.max_out_idx;
    block_max_atomic(mx, &A.smax[RTM_IN(k, A.len.smax, A.err) ? k : 0], S.red);
  }
  if (MODE == MODE_BWD && rt.dmax_flag == 2)
    block_max_atomic(dm, &A.dmax[RTM_IN(b, A.len.items, A.err) ? b : 0], S.red);
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
  // per (mode, device): the shared-memory opt-in and the number of blocks
  // resident at once (launches come from several request threads; computing
  // either twice is harmless)
  static std::atomic<int> resident[4][64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  const size_t smem = step2_smem_bytes();
  dim3 grid(A.g.ntx2, A.g.ntz2, B), block(32, NTH / 32);
  auto launch = [&](auto kernel, int slot) -> cudaError_t {
    int nres = resident[slot][dev].load(std::memory_order_acquire);
    if (nres == 0) {
      cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (r != cudaSuccess) return r;
      int per_sm = 0, nsm = 0;
      r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NTH, smem);
      if (r != cudaSuccess) return r;
      r = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (r != cudaSuccess) return r;
      nres = per_sm > 0 ? per_sm * nsm : 1;
      resident[slot][dev].store(nres, std::memory_order_release);
    }
    Step2RT r2 = rt;
    r2.ahead = rt.ahead ? nres : 0;  // the block that takes this block's place
    kernel<<<grid, block, smem, st>>>(mv, md, mc, A, r2);
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
