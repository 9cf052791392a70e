// rtm_prop2p.cu — persistent two-time-step propagation kernel with a
// two-stage copy ring.
//
// k_step2p advances B grids by TWO leapfrog steps of the scheme of §2.2 Eq. 4
// / §3 (difference form, see rtm_prop.cu) with exactly the per-point
// arithmetic of k_step2 (rtm_prop2.cu), so the three propagation kernels give
// the same bits.  What differs is how the work reaches the SM:
//
//   * Persistent blocks.  The grid holds as many blocks as fit on the GPU at
//     once (two per SM); block i walks tiles i, i + G, i + 2G, ... of the
//     launch's tile list (item-major, then tile row, then tile column).
//   * Two-stage copy ring.  Each block owns two shared-memory stages of
//     {v^n (halo 8), d^n (halo 4), c (halo 4)}, each with its own mbarrier.
//     The TMA bulk-tensor loads of tile k+1 are issued before tile k is
//     computed, so the copy of the next tile overlaps the stencil of the
//     current one (the one-tile-per-block kernel only overlaps copies of
//     different blocks).
//   * v^{n+1} over v^n.  After substep 1 has read its whole stencil window,
//     v^{n+1} is written into the v^n tile at its (+4, +4) offset instead of a
//     separate array, which keeps a stage at 54 KB and two blocks per SM.
//     Blocks that inject at the intermediate step add the injection to d^{n+1}
//     in shared memory first and then form v^{n+1} = v^n + d^{n+1} from it,
//     which is the rounding order of the other kernels.
//   * Snake order.  With `reverse` set the tile list is walked from its end,
//     and the host alternates it between consecutive launches, so a launch
//     starts on the grids the previous launch wrote last, still in L2.
//   * Tile height.  R1 rows per thread at substep 1 give an extended region of
//     8 R1 rows and a centre of 8 (R1 - 1) rows: 120 x 24 (R1 = 4) or 120 x 16
//     (R1 = 3).  The launch configuration picks one.
//
// Every wait is bounded: if a TMA transaction does not complete within the
// bound, the block raises the error flag (reported as RTM_ERR_TIMEOUT), lets
// the copies it issued land (bounded again) and returns; the decision is
// taken block-wide so no thread is left at a barrier.
#include <cuda.h>

#include <atomic>
#include <cuda_runtime.h>

#include "rtm_common.h"
#include "rtm_launch.h"
#include "rtm_step2_dev.cuh"

namespace rtm {

namespace {

using namespace s2;

template <int R1>
struct Shape {
  static constexpr int EZ = 8 * R1;     // extended region rows (4 per side around the centre)
  static constexpr int C2Z = EZ - 8;    // centre rows
  static constexpr int R2 = R1 - 1;     // centre rows per thread at substep 2
  static constexpr int VZ = C2Z + 16;   // v^n tile rows (halo 8)
  static constexpr unsigned kTx = (VX * VZ + 2 * EX * EZ) * 4;  // bytes per stage
};

template <int R1>
struct Stage {
  float v0[Shape<R1>::VZ][VX];  // v^n; after substep 1, v^{n+1} at offset (+4, +4)
  float d[Shape<R1>::EZ][EX];   // d^n -> d^{n+1} -> d^{n+2}, updated in place
  float c[Shape<R1>::EZ][EX];   // (v dt)^2
  float gxs[EX];                // sponge factors of the extended region's columns ...
  float gzs[(Shape<R1>::EZ + 31) / 32 * 32];  // ... and rows (tiles that reach the sponge)
};

template <int R1>
struct SmemP {
  Stage<R1> st[2];
  unsigned long long bar[2];
  float red[NTH / 32];
};
static_assert(sizeof(Stage<4>) % 128 == 0 && sizeof(Stage<3>) % 128 == 0 &&
                  sizeof(Stage<5>) % 128 == 0,
              "stages must keep the TMA destinations 128-byte aligned");
static_assert(sizeof(float) * VX * Shape<4>::VZ % 128 == 0 &&
                  sizeof(float) * VX * Shape<3>::VZ % 128 == 0 &&
                  sizeof(float) * EX * Shape<4>::EZ % 128 == 0 &&
                  sizeof(float) * EX * Shape<3>::EZ % 128 == 0,
              "tile offsets must stay 128-byte aligned");

struct TileRef {
  int b, x0, z0, tile;  // item slot, first memory column and row of the centre, tile in grid
};

template <int R1>
__device__ __forceinline__ TileRef tile_at(const Geo &g, int t) {
  const int tpi = g.ntx2 * g.ntz2;
  const int b = t / tpi, r = t - b * tpi;
  const int tz = r / g.ntx2, tx = r - tz * g.ntx2;
  return TileRef{b, tx * C2X, tz * Shape<R1>::C2Z, r};
}

template <int R1>
__device__ __forceinline__ bool tile_interior(const Geo &g, int x0, int z0) {
  return (z0 - 4 >= g.nb) && (z0 + Shape<R1>::C2Z + 4 <= g.NZ - g.nb) && (x0 - 4 >= g.X0 + g.nb) &&
         (x0 + C2X + 4 <= g.X0 + g.NX - g.nb);
}

// v^{n+1} at extended-region offset `off` = r * EX + c (receiver tables).
template <int R1>
__device__ __forceinline__ float &v1_at(Stage<R1> &S, int off) {
  return S.v0[(off >> 7) + 4][(off & (EX - 1)) + 4];
}
static_assert(EX == 128, "v1_at decodes offsets with EX = 128");

// Issue tile t into stage S (all threads call; thread 0 issues the copies).
template <int R1>
__device__ __forceinline__ void issue_tile(Stage<R1> &S, unsigned long long *bar,
                                           const CUtensorMap *mv, const CUtensorMap *md,
                                           const CUtensorMap *mc, const Step2Args &A, int t) {
  const Geo &g = A.g;
  const TileRef T = tile_at<R1>(g, t);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid == 0) {
    const int smp = A.one_sample ? 0 : A.item_sample[T.b];
    (void)RTM_IN(smp, A.len.nsample, A.err);  // (the copy engine clips the box; a bad plane is
                                              // recorded, not read)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(Shape<R1>::kTx)
                 : "memory");
    tma_load_3d(&S.v0[0][0], mv, T.x0 - 8, T.z0 - 8, T.b, bar);
    tma_load_3d(&S.d[0][0], md, T.x0 - 4, T.z0 - 4, T.b, bar);
    tma_load_3d(&S.c[0][0], mc, T.x0 - 4, T.z0 - 4, smp, bar);
  }
  if (!tile_interior<R1>(g, T.x0, T.z0)) {  // edge-clamped sponge factors
    if (tid < EX) S.gxs[tid] = A.gx[min(max(T.x0 - 4 + tid, 0), g.P - 1)];
    if (tid < Shape<R1>::EZ) S.gzs[tid] = A.gz[min(max(T.z0 - 4 + tid, 0), g.NZ - 1)];
  }
}

// Backward imaging launches: pull tile t's num, den and snapshot rows into L2
// while the current tile computes.
template <int R1>
__device__ __forceinline__ void prefetch_imaging(const Step2Args &A, const Step2RT &rt, int t) {
  const Geo &g = A.g;
  const TileRef T = tile_at<R1>(g, t);
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (tx >= C2X / 4) return;
  const int j0 = T.x0 + 4 * tx - g.CP;
  if (j0 < 0 || j0 >= g.SX) return;
  const int esz = A.snap_dtype == 0 ? 4 : 2;
#pragma unroll
  for (int r = 0; r < Shape<R1>::R2; ++r) {
    const int i = T.z0 + Shape<R1>::R2 * ty + r - g.nb;
    if (i >= 0 && i < g.nz) {
      const long long po = (long long)T.b * g.pplane + (long long)i * g.SX + j0;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(A.num + po));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(A.den + po));
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        const int idx = u == 0 ? rt.img_mid_idx : (u == 1 ? rt.img_out_idx : rt.img_in_idx);
        if (idx >= 0) {
          const long long so =
              ((long long)T.b * A.nsnap + idx) * g.pplane + (long long)i * g.SX + j0;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char *>(A.snap) +
                                                         so * esz));
        }
      }
    }
  }
}

// Substep 1 on rows R1 ty .. R1 ty + R1 - 1, columns 4tx..4tx+3 of the
// extended region: d^{n+1} into nd (Born source included) and S.d; v^n of the
// same cells into ce.
template <int MODE, bool SPONGE, bool ISO, int R1>
__device__ __forceinline__ void substep1p(Stage<R1> &S, const Step2Args &A, const Step2RT &rt,
                                          int b, int x0, int z0, float4 (&ce)[R1],
                                          float4 (&nd)[R1]) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const Geo &g = A.g;
  float4 zc[R1 + 8];
#pragma unroll
  for (int q = 0; q < R1 + 8; ++q)
    zc[q] = *reinterpret_cast<const float4 *>(&S.v0[R1 * ty + q][4 + 4 * tx]);
  const float *gxs = &S.gxs[4 * tx];
#pragma unroll
  for (int r = 0; r < R1; ++r) {
    const int er = R1 * ty + r;
    const float4 xl = *reinterpret_cast<const float4 *>(&S.v0[er + 4][4 * tx]);
    const float4 xr = *reinterpret_cast<const float4 *>(&S.v0[er + 4][8 + 4 * tx]);
    const float4 dv = *reinterpret_cast<const float4 *>(&S.d[er][4 * tx]);
    const float4 cv = *reinterpret_cast<const float4 *>(&S.c[er][4 * tx]);
    const float gzr = SPONGE ? S.gzs[er] : 1.f;
    nd[r] = update4<SPONGE, ISO>(&zc[r], xl, xr, dv, cv, A.k, gzr, gxs);
    ce[r] = zc[r + 4];
  }
  if (MODE == MODE_BORN) {  // the Born source joins each row's new difference
    const int gcol = x0 - 4 + 4 * tx;
#pragma unroll
    for (int r = 0; r < R1; ++r) {
      const int er = R1 * ty + r;
      const float4 cv = *reinterpret_cast<const float4 *>(&S.c[er][4 * tx]);
      nd[r] = born_inject4(A, b, rt.img_mid_idx, z0 - 4 + er - g.nb, gcol - g.CP, nd[r], cv);
    }
  }
#pragma unroll
  for (int r = 0; r < R1; ++r) *reinterpret_cast<float4 *>(&S.d[R1 * ty + r][4 * tx]) = nd[r];
}

// Substep 2 on centre rows R2 ty .. R2 ty + R2 - 1: d^{n+2} (res, before
// injection) and v^{n+1} (cen), reading v^{n+1} from the v^n tile's offset.
template <int MODE, bool SPONGE, bool ISO, int R1>
__device__ __forceinline__ void substep2p(const Stage<R1> &S, const Step2Args &A,
                                          const Step2RT &rt, int b, int x0, int z0,
                                          float4 (&res)[R1 - 1], float4 (&cen)[R1 - 1]) {
  constexpr int R2 = R1 - 1;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const Geo &g = A.g;
  float4 zc[R2 + 8];
#pragma unroll
  for (int q = 0; q < R2 + 8; ++q)
    zc[q] = *reinterpret_cast<const float4 *>(&S.v0[R2 * ty + q + 4][8 + 4 * tx]);
  const float *gxs = &S.gxs[4 + 4 * tx];
#pragma unroll
  for (int r = 0; r < R2; ++r) {
    const int er = 4 + R2 * ty + r;
    const float4 xl = *reinterpret_cast<const float4 *>(&S.v0[er + 4][4 + 4 * tx]);
    const float4 xr = *reinterpret_cast<const float4 *>(&S.v0[er + 4][12 + 4 * tx]);
    const float4 dv = *reinterpret_cast<const float4 *>(&S.d[er][4 + 4 * tx]);
    const float4 cv = *reinterpret_cast<const float4 *>(&S.c[er][4 + 4 * tx]);
    const float gzr = SPONGE ? S.gzs[er] : 1.f;
    res[r] = update4<SPONGE, ISO>(&zc[r], xl, xr, dv, cv, A.k, gzr, gxs);
    cen[r] = zc[r + 4];
  }
  if (MODE == MODE_BORN) {
    const int gcol = x0 + 4 * tx;
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const float4 cv = *reinterpret_cast<const float4 *>(&S.c[4 + R2 * ty + r][4 + 4 * tx]);
      res[r] = born_inject4(A, b, rt.img_out_idx, z0 + R2 * ty + r - g.nb, gcol - g.CP, res[r], cv);
    }
  }
}

// num += S w, den += S^2 over 4 physical columns of row i; returns max(den).
__device__ __forceinline__ float image4(const Step2Args &A, int b, int idx, int i, int j0,
                                        const float4 &w) {
  const Geo &g = A.g;
  const long long so = ((long long)b * A.nsnap + idx) * g.pplane + (long long)i * g.SX + j0;
  const long long po = (long long)b * g.pplane + (long long)i * g.SX + j0;
  if (!RTM_IN((long long)b * A.nsnap + idx, A.len.smax, A.err) || !RTM_IN(so + 3, A.len.snap, A.err) ||
      !RTM_IN(po + 3, A.len.items * g.pplane, A.err))
    return 0.f;
  float sdq, inv;
  snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + idx], sdq, inv);
  const float4 Sv = snap_load4(A.snap, so, A.snap_dtype, sdq);
  float4 *pn = reinterpret_cast<float4 *>(A.num + po);
  float4 *pd = reinterpret_cast<float4 *>(A.den + po);
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
  return fmaxf(fmaxf(de.x, de.y), fmaxf(de.z, de.w));
}

// Imaging with the input field: the snapshot (dequantised), num and den of
// this thread's centre rows, loaded before the block waits for its tile
// copies, so their latency overlaps the copies.  ok[r] marks loaded rows.
template <int R1>
struct InImg {
  float4 S[R1 - 1], N[R1 - 1], D[R1 - 1];
  bool ok[R1 - 1];
};

template <int R1>
__device__ __forceinline__ void load_in_imaging(const Step2Args &A, const Step2RT &rt, int t,
                                                InImg<R1> &p) {
  constexpr int R2 = R1 - 1;
  const Geo &g = A.g;
  const TileRef T = tile_at<R1>(g, t);
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int j0 = T.x0 + 4 * tx - g.CP;
  const bool jok = tx < C2X / 4 && j0 >= 0 && j0 < g.SX;
  const long long ks = (long long)T.b * A.nsnap + rt.img_in_idx;
  float sdq = 0.f, inv;
  const bool sok = jok && RTM_IN(ks, A.len.smax, A.err);
  if (sok) snap_scale(A.snap_dtype, A.smax[ks], sdq, inv);
#pragma unroll
  for (int r = 0; r < R2; ++r) {
    const int i = T.z0 + R2 * ty + r - g.nb;
    const long long so = ks * g.pplane + (long long)i * g.SX + j0;
    const long long po = (long long)T.b * g.pplane + (long long)i * g.SX + j0;
    p.ok[r] = sok && i >= 0 && i < g.nz && RTM_IN(so + 3, A.len.snap, A.err) &&
              RTM_IN(po + 3, A.len.items * g.pplane, A.err);
    if (p.ok[r]) {
      p.S[r] = snap_load4(A.snap, so, A.snap_dtype, sdq);
      p.N[r] = *reinterpret_cast<const float4 *>(A.num + po);
      p.D[r] = *reinterpret_cast<const float4 *>(A.den + po);
    }
  }
}

// num += S w, den += S^2 with preloaded operands (the rounding of image4);
// returns max(den).
__device__ __forceinline__ float image4_pre(const Step2Args &A, int b, int i, int j0,
                                            const float4 &w, const float4 &Sv, float4 nu,
                                            float4 de) {
  const long long po = (long long)b * A.g.pplane + (long long)i * A.g.SX + j0;
  nu.x = fmaf(Sv.x, w.x, nu.x);
  nu.y = fmaf(Sv.y, w.y, nu.y);
  nu.z = fmaf(Sv.z, w.z, nu.z);
  nu.w = fmaf(Sv.w, w.w, nu.w);
  de.x = fmaf(Sv.x, Sv.x, de.x);
  de.y = fmaf(Sv.y, Sv.y, de.y);
  de.z = fmaf(Sv.z, Sv.z, de.z);
  de.w = fmaf(Sv.w, Sv.w, de.w);
  *reinterpret_cast<float4 *>(A.num + po) = nu;
  *reinterpret_cast<float4 *>(A.den + po) = de;
  return fmaxf(fmaxf(de.x, de.y), fmaxf(de.z, de.w));
}

// FP32 snapshot of 4 physical columns (columns past nx stored as zero).
__device__ __forceinline__ void snap_f32(const Step2Args &A, int b, int idx, int i, int j0,
                                         float4 v) {
  const Geo &g = A.g;
  if (j0 + 1 >= g.nx) v.y = 0.f;
  if (j0 + 2 >= g.nx) v.z = 0.f;
  if (j0 + 3 >= g.nx) v.w = 0.f;
  const long long so = ((long long)b * A.nsnap + idx) * g.pplane + (long long)i * g.SX + j0;
  if (RTM_IN(so + 3, A.len.snap, A.err)) snap_store4(A.snap, so, 0, v, 1.f);
}

// One tile: both substeps, the fused work of steps n+1 and n+2, the stores.
// IN_IMG compiles in the imaging with the input field (rt.img_in_idx, dmax
// flag 3); instances without it must not be launched with either set.
template <int MODE, int R1, bool IN_IMG>
__device__ __forceinline__ void tile_body(Stage<R1> &S, float *red, const Step2Args &A,
                                          const Step2RT &rt, int t, const InImg<R1> *pre) {
  constexpr int EZ = Shape<R1>::EZ, C2Z = Shape<R1>::C2Z, R2 = Shape<R1>::R2;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const Geo &g = A.g;
  const TileRef T = tile_at<R1>(g, t);
  const int b = T.b, x0 = T.x0, z0 = T.z0, tile = T.tile;
  const int shot = RTM_IN(b, A.len.items, A.err) ? A.item_shot[b] : 0;
  const bool interior = tile_interior<R1>(g, x0, z0);
#ifdef RTM_DEBUG
  const bool shot_ok = RTM_IN(shot, A.len.nshot, A.err) && RTM_IN(tile + 1, g.ntx2 * g.ntz2 + 1, A.err);
#else
  constexpr bool shot_ok = true;
#endif
  const bool wide = tx < C2X / 4;  // threads that own centre columns
  const int j0 = x0 + 4 * tx - g.CP;  // physical column of this thread's centre strip
  const bool jok = wide && j0 >= 0 && j0 < g.SX;

  // deferred half-precision snapshot of the INPUT field v^n (its max was
  // reduced by the launch that produced it)
  if (MODE == MODE_FWD && rt.snap_in_idx >= 0 && jok &&
      RTM_IN((long long)b * A.nsnap + rt.snap_in_idx, A.len.smax, A.err)) {
    float sdq, inv;
    snap_scale(A.snap_dtype, A.smax[(long long)b * A.nsnap + rt.snap_in_idx], sdq, inv);
    const long long base = ((long long)b * A.nsnap + rt.snap_in_idx) * g.pplane + j0;
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const int i = z0 + R2 * ty + r - g.nb;
      if (i >= 0 && i < g.nz && RTM_IN(base + (long long)i * g.SX + 3, A.len.snap, A.err)) {
        float4 v = *reinterpret_cast<const float4 *>(&S.v0[8 + R2 * ty + r][8 + 4 * tx]);
        if (j0 + 1 >= g.nx) v.y = 0.f;
        if (j0 + 2 >= g.nx) v.z = 0.f;
        if (j0 + 3 >= g.nx) v.w = 0.f;
        snap_store4(A.snap, base + (long long)i * g.SX, A.snap_dtype, v, inv);
      }
    }
  }

  // imaging with the INPUT field v^n (the centre of the v^n tile), before
  // substep 1 overwrites it; operands preloaded by the caller when it can
  float dm = 0.f;  // running max of den for the max-den reduction
  if (IN_IMG && MODE == MODE_BWD && rt.img_in_idx >= 0 && jok) {
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const int i = z0 + R2 * ty + r - g.nb;
      const float4 w = *reinterpret_cast<const float4 *>(&S.v0[8 + R2 * ty + r][8 + 4 * tx]);
      if (pre) {
        if (pre->ok[r]) dm = fmaxf(dm, image4_pre(A, b, i, j0, w, pre->S[r], pre->N[r], pre->D[r]));
      } else if (i >= 0 && i < g.nz) {
        dm = fmaxf(dm, image4(A, b, rt.img_in_idx, i, j0, w));
      }
    }
  }
  if (IN_IMG && MODE == MODE_BWD && rt.dmax_flag == 3)
    block_max_atomic(dm, &A.dmax[RTM_IN(b, A.len.items, A.err) ? b : 0], red);

  // ---- substep 1 (a warp whose rows lie 4 or more past the grid skips:
  // substep 2 reads rows up to 4 past its own, and computes none below the
  // grid's last row + 1) ------------------------------------------------------
  float4 ce[R1], nd[R1];
  const bool run1 = interior || (z0 - 4 + R1 * ty < g.NZ + 4);  // warp-uniform
  if (run1) {
    if (A.k.iso) {
      if (interior)
        substep1p<MODE, false, true, R1>(S, A, rt, b, x0, z0, ce, nd);
      else
        substep1p<MODE, true, true, R1>(S, A, rt, b, x0, z0, ce, nd);
    } else {
      if (interior)
        substep1p<MODE, false, false, R1>(S, A, rt, b, x0, z0, ce, nd);
      else
        substep1p<MODE, true, false, R1>(S, A, rt, b, x0, z0, ce, nd);
    }
  }
  __syncthreads();  // every read of v^n is done: the tile may take v^{n+1}

  // injection at step t1 into every cell of the extended region, added to
  // d^{n+1}; the owning threads then form v^{n+1} from the updated d
  bool inj1 = false;
  if (MODE == MODE_FWD || MODE == MODE_MODEL) {
    const int sr = A.src_row[shot] - (z0 - 4), sc = A.src_col[shot] - (x0 - 4);
    inj1 = sr >= 0 && sr < EZ && sc >= 0 && sc < EX;  // block-uniform
    if (inj1 && tid == 0 && RTM_IN(rt.t1, A.nt, A.err))
      S.d[sr][sc] += S.c[sr][sc] * (A.wav[rt.t1] * A.src_scale);
  } else if (MODE == MODE_BWD) {
    const int p0 = shot_ok ? A.rext_ptr[tile] : 0, p1 = shot_ok ? A.rext_ptr[tile + 1] : 0;
    inj1 = p1 > p0;  // block-uniform
    if (inj1) {
      const long long d0 = ((long long)shot * A.nt + rt.t1) * A.nrec;
      const float *dsamp = A.seis + d0;
      for (int e = p0 + tid; e < p1; e += NTH) {
        if (!RTM_IN(e, A.len.rent, A.err)) continue;
        const int2 en = A.rext_ent[e];
        const int er = en.x >> 7, ec = en.x & (EX - 1);
        if (RTM_IN(en.x, EX * EZ, A.err) && RTM_IN(en.y, A.nrec, A.err) &&
            RTM_IN(d0 + en.y, A.len.nshot * A.nt * A.nrec, A.err))
          atomicAdd(&S.d[er][ec], S.c[er][ec] * dsamp[en.y]);
      }
    }
  }
  if (inj1) {
    __syncthreads();
    if (run1) {
#pragma unroll
      for (int r = 0; r < R1; ++r)
        nd[r] = *reinterpret_cast<const float4 *>(&S.d[R1 * ty + r][4 * tx]);
    }
  }
  if (run1) {
#pragma unroll
    for (int r = 0; r < R1; ++r)
      *reinterpret_cast<float4 *>(&S.v0[R1 * ty + r + 4][4 * tx + 4]) =
          make_float4(ce[r].x + nd[r].x, ce[r].y + nd[r].y, ce[r].z + nd[r].z, ce[r].w + nd[r].w);
  }
  __syncthreads();

  // step-(n+1) work on the centre: recording, FP32 snapshot, imaging
  if (MODE == MODE_MODEL || MODE == MODE_BORN) {
    const int p0 = shot_ok ? A.rcen_ptr[tile] : 0, p1 = shot_ok ? A.rcen_ptr[tile + 1] : 0;
    const long long r0 = ((long long)b * A.nt + rt.t1) * A.nrec;
    float *ro = A.rec_out + r0;
    for (int e = p0 + tid; e < p1; e += NTH) {
      if (!RTM_IN(e, A.len.rcen, A.err)) continue;
      const int2 en = A.rcen_ent[e];
      if (RTM_IN(en.x, EX * EZ, A.err) && RTM_IN(r0 + en.y, A.len.rec_out, A.err))
        ro[en.y] = v1_at<R1>(S, en.x);
    }
  }
  if (MODE == MODE_FWD && rt.snap_mid_idx >= 0 && jok) {
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const int i = z0 + R2 * ty + r - g.nb;
      if (i >= 0 && i < g.nz)
        snap_f32(A, b, rt.snap_mid_idx, i, j0,
                 *reinterpret_cast<const float4 *>(&S.v0[8 + R2 * ty + r][8 + 4 * tx]));
    }
  }
  if (MODE == MODE_BWD && rt.img_mid_idx >= 0 && jok) {
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const int i = z0 + R2 * ty + r - g.nb;
      if (i >= 0 && i < g.nz)
        dm = fmaxf(dm, image4(A, b, rt.img_mid_idx, i, j0,
                              *reinterpret_cast<const float4 *>(&S.v0[8 + R2 * ty + r][8 + 4 * tx])));
    }
  }
  if (MODE == MODE_BWD && rt.dmax_flag == 1)
    block_max_atomic(dm, &A.dmax[RTM_IN(b, A.len.items, A.err) ? b : 0], red);

  // ---- substep 2 on the centre ---------------------------------------------
  float4 res[R2];
  float4 cen[R2];
  if (wide) {
    if (interior) {
      if (A.k.iso)
        substep2p<MODE, false, true, R1>(S, A, rt, b, x0, z0, res, cen);
      else
        substep2p<MODE, false, false, R1>(S, A, rt, b, x0, z0, res, cen);
    } else if (z0 + R2 * ty < g.NZ) {
      if (A.k.iso)
        substep2p<MODE, true, true, R1>(S, A, rt, b, x0, z0, res, cen);
      else
        substep2p<MODE, true, false, R1>(S, A, rt, b, x0, z0, res, cen);
    } else {  // rows past the grid: nothing of them is stored
#pragma unroll
      for (int r = 0; r < R2; ++r) res[r] = cen[r] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }

  // injection at step t2 on the centre (staged through the d tile)
  {
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
        for (int r = 0; r < R2; ++r)
          *reinterpret_cast<float4 *>(&S.d[4 + R2 * ty + r][4 + 4 * tx]) = res[r];
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
            ro[en.y] = v1_at<R1>(S, en.x) + (&S.d[0][0])[en.x];  // v^{n+2} = v^{n+1} + d^{n+2}
        }
      }
      if (wide) {
#pragma unroll
        for (int r = 0; r < R2; ++r)
          res[r] = *reinterpret_cast<const float4 *>(&S.d[4 + R2 * ty + r][4 + 4 * tx]);
      }
    }
  }

  // ---- write d^{n+2}, v^{n+2}; step-(n+2) work -------------------------------
  float mx = 0.f;
  if (wide) {
    const int col = x0 + 4 * tx;
    float *vo = A.v_out + (long long)b * g.plane;
    float *dq = A.d_out + (long long)b * g.plane;
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const int row = z0 + R2 * ty + r;
      const float4 nv = make_float4(cen[r].x + res[r].x, cen[r].y + res[r].y, cen[r].z + res[r].z,
                                    cen[r].w + res[r].w);
      if (row < g.NZ && col < g.P &&
          RTM_IN((long long)b * g.plane + (long long)row * g.P + col + 3, A.len.items * g.plane,
                 A.err)) {
        const long long o = (long long)row * g.P + col;
        *reinterpret_cast<float4 *>(dq + o) = res[r];
        *reinterpret_cast<float4 *>(vo + o) = nv;
      }
      const int i = row - g.nb;
      if (i >= 0 && i < g.nz) {
        if (MODE == MODE_FWD && rt.max_out_idx >= 0) {
#pragma unroll
          for (int l = 0; l < 4; ++l)
            if (j0 + l >= 0 && j0 + l < g.nx) mx = fmaxf(mx, fabsf(lane4(nv, l)));
        }
        if (MODE == MODE_FWD && rt.snap_out_idx >= 0 && jok) snap_f32(A, b, rt.snap_out_idx, i, j0, nv);
        if (MODE == MODE_BWD && rt.img_out_idx >= 0 && jok)
          dm = fmaxf(dm, image4(A, b, rt.img_out_idx, i, j0, nv));
      }
    }
  }
  if (MODE == MODE_FWD && rt.max_out_idx >= 0) {
    const long long k = (long long)b * A.nsnap + rt.max_out_idx;
    block_max_atomic(mx, &A.smax[RTM_IN(k, A.len.smax, A.err) ? k : 0], red);
  }
  if (MODE == MODE_BWD && rt.dmax_flag == 2)
    block_max_atomic(dm, &A.dmax[RTM_IN(b, A.len.items, A.err) ? b : 0], red);
}

}  // namespace

template <int MODE, int R1>
__global__ void __launch_bounds__(NTH, 2)
    k_step2p(const __grid_constant__ CUtensorMap map_v, const __grid_constant__ CUtensorMap map_d,
             const __grid_constant__ CUtensorMap map_c, const Step2Args A, const Step2RT rt,
             int ntiles) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // TMA destinations must be 128-byte aligned: align the base explicitly
  SmemP<R1> &S =
      *reinterpret_cast<SmemP<R1> *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int G = gridDim.x;
  if ((int)blockIdx.x >= ntiles) return;  // (the grid is sized to the tiles)
  auto tile_index = [&](int k) {
    const int t = (int)blockIdx.x + k * G;
    return rt.reverse ? ntiles - 1 - t : t;
  };
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.bar[0])), "r"(1)
                 : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.bar[1])), "r"(1)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  issue_tile<R1>(S.st[0], &S.bar[0], &map_v, &map_d, &map_c, A, tile_index(0));
  const bool imaging =
      MODE == MODE_BWD && (rt.img_mid_idx >= 0 || rt.img_out_idx >= 0 || rt.img_in_idx >= 0);
  if (imaging) prefetch_imaging<R1>(A, rt, tile_index(0));
  for (int k = 0; (int)blockIdx.x + k * G < ntiles; ++k) {
    const int s = k & 1;
    const bool has_next = (int)blockIdx.x + (k + 1) * G < ntiles;
    // stage s^1 was released by the barrier that ended tile k-1
    if (has_next) {
      issue_tile<R1>(S.st[s ^ 1], &S.bar[s ^ 1], &map_v, &map_d, &map_c, A, tile_index(k + 1));
      if (imaging) prefetch_imaging<R1>(A, rt, tile_index(k + 1));
    }
    const unsigned phase = (unsigned)(k >> 1) & 1u;
    const bool ok = mbar_wait_bounded(&S.bar[s], phase, kWaitNs);
    // (block-wide decision; also orders the sponge factors staged for tile k)
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(A.err, 1);
      // let the copies in flight land (bounded) before the block exits
      mbar_wait_bounded(&S.bar[s], phase, kWaitNs);
      if (has_next) mbar_wait_bounded(&S.bar[s ^ 1], (unsigned)((k + 1) >> 1) & 1u, kWaitNs);
      return;
    }
    tile_body<MODE, R1, true>(S.st[s], S.red, A, rt, tile_index(k), nullptr);
    // generic-proxy writes of this stage (d in place, v^{n+1}) are ordered
    // before the copy engine's next writes into it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
}

// One tile per block with the same tile body and a single stage: 3 blocks per
// SM overlap one another's copies.  Writing v^{n+1} over v^n frees the
// separate v^{n+1} array of k_step2, which makes room for 120 x 32 tiles
// (R1 = 5, 67 KB) at 3 blocks per SM.  Snake order as in k_step2p.
template <int R1>
struct Smem1 {
  Stage<R1> st;
  unsigned long long bar;
  float red[NTH / 32];
};

// VAR bit 0: imaging with the input field, its operands loaded before the
// tile wait (backward); bit 1: launched as a programmatic dependent.  The
// default launch (VAR 0) carries neither path's code.
template <int MODE, int R1, int VAR>
__global__ void __launch_bounds__(NTH, 3)
    k_step2a(const __grid_constant__ CUtensorMap map_v, const __grid_constant__ CUtensorMap map_d,
             const __grid_constant__ CUtensorMap map_c, const Step2Args A, const Step2RT rt,
             int ntiles) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem1<R1> &S =
      *reinterpret_cast<Smem1<R1> *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if ((int)blockIdx.x >= ntiles) return;  // (the grid is sized to the tiles)
  const int t = rt.reverse ? ntiles - 1 - (int)blockIdx.x : (int)blockIdx.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.bar)), "r"(1)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  constexpr bool IN_IMG = (VAR & 1) != 0, PDL = (VAR & 2) != 0;
  __syncthreads();
  if constexpr (PDL) {
    // launched as a programmatic dependent: copy what the previous launch does
    // not write (c, the sponge factors) while it finishes, then wait for it
    // before the copies of its output fields v^n, d^n
    const TileRef T = tile_at<R1>(A.g, t);
    if (tid == 0) {
      const int smp = A.one_sample ? 0 : A.item_sample[T.b];
      (void)RTM_IN(smp, A.len.nsample, A.err);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&S.bar)),
                   "r"(Shape<R1>::kTx)
                   : "memory");
      tma_load_3d(&S.st.c[0][0], &map_c, T.x0 - 4, T.z0 - 4, smp, &S.bar);
    }
    if (!tile_interior<R1>(A.g, T.x0, T.z0)) {
      if (tid < EX) S.st.gxs[tid] = A.gx[min(max(T.x0 - 4 + tid, 0), A.g.P - 1)];
      if (tid < Shape<R1>::EZ) S.st.gzs[tid] = A.gz[min(max(T.z0 - 4 + tid, 0), A.g.NZ - 1)];
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // every block of this launch has started: the next launch may begin its own
    // preamble on the SMs this launch frees
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (tid == 0) {
      tma_load_3d(&S.st.v0[0][0], &map_v, T.x0 - 8, T.z0 - 8, T.b, &S.bar);
      tma_load_3d(&S.st.d[0][0], &map_d, T.x0 - 4, T.z0 - 4, T.b, &S.bar);
    }
  } else {
    issue_tile<R1>(S.st, &S.bar, &map_v, &map_d, &map_c, A, t);
  }
  if (MODE == MODE_BWD && (rt.img_mid_idx >= 0 || rt.img_out_idx >= 0))
    prefetch_imaging<R1>(A, rt, t);
  // imaging with the input field: its operands load while the tile copies land
  InImg<R1> pre;
  if (IN_IMG && MODE == MODE_BWD && rt.img_in_idx >= 0) load_in_imaging<R1>(A, rt, t, pre);
  const bool ok = mbar_wait_bounded(&S.bar, 0, kWaitNs);
  if (__syncthreads_or(!ok)) {  // (block-wide; also orders the staged sponge factors)
    if (tid == 0) atomicExch(A.err, 1);
    mbar_wait_bounded(&S.bar, 0, kWaitNs);  // let the copies in flight land (bounded)
    return;
  }
  tile_body<MODE, R1, IN_IMG>(S.st, S.red, A, rt, t,
                              IN_IMG && MODE == MODE_BWD && rt.img_in_idx >= 0 ? &pre : nullptr);
}

size_t step2p_smem_bytes(int tile_z) {
  return (tile_z == 16 ? sizeof(SmemP<3>) : sizeof(SmemP<4>)) + 128;
}

size_t step2a_smem_bytes(int tile_z) {
  return (tile_z == 32 ? sizeof(Smem1<5>) : sizeof(Smem1<4>)) + 128;
}

cudaError_t launch_step2a(int mode, int tile_z, const CUtensorMap &mv, const CUtensorMap &md,
                          const CUtensorMap &mc, const Step2Args &A, const Step2RT &rt, int B,
                          cudaStream_t st) {
  if (tile_z != 24 && tile_z != 32) return cudaErrorInvalidValue;
  const long long ntl = (long long)B * A.g.ntx2 * A.g.ntz2;
  if (ntl < 1 || ntl > 0x7fffffffLL) return cudaErrorInvalidValue;
  // the input-field imaging and programmatic-dependent instances exist for the
  // backward and forward migration phases only
  const bool in_img = rt.img_in_idx >= 0 || rt.dmax_flag == 3;
  if (in_img && mode != MODE_BWD) return cudaErrorInvalidValue;
  if (rt.pdl && mode != MODE_BWD && mode != MODE_FWD) return cudaErrorInvalidValue;
  static std::atomic<bool> attr_set[32];
  const size_t smem = step2a_smem_bytes(tile_z);
  dim3 block(32, NTH / 32);
  auto launch = [&](auto kernel, int slot) -> cudaError_t {
    if (!attr_set[slot].load(std::memory_order_acquire)) {
      const cudaError_t e =
          cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_set[slot].store(true, std::memory_order_release);
    }
    if (!rt.pdl) {
      kernel<<<(unsigned)ntl, block, smem, st>>>(mv, md, mc, A, rt, (int)ntl);
      return cudaGetLastError();
    }
    // programmatic dependent launch: blocks may start while the previous
    // kernel on the stream finishes (the kernel waits before reading its outputs)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ntl);
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, mv, md, mc, A, rt, (int)ntl);
  };
  // slot = 16 * (tile_z == 32) + 4 * mode + VAR
  const int var = (in_img ? 1 : 0) | (rt.pdl ? 2 : 0);
  const int slot = (tile_z == 32 ? 16 : 0) + 4 * mode + var;
#define RTM_S2A(M, R, V) launch(k_step2a<M, R, V>, (R == 5 ? 16 : 0) + 4 * M + V)
  switch (slot) {
    case 0: return RTM_S2A(MODE_FWD, 4, 0);
    case 2: return RTM_S2A(MODE_FWD, 4, 2);
    case 4: return RTM_S2A(MODE_MODEL, 4, 0);
    case 8: return RTM_S2A(MODE_BWD, 4, 0);
    case 9: return RTM_S2A(MODE_BWD, 4, 1);
    case 10: return RTM_S2A(MODE_BWD, 4, 2);
    case 11: return RTM_S2A(MODE_BWD, 4, 3);
    case 12: return RTM_S2A(MODE_BORN, 4, 0);
    case 16: return RTM_S2A(MODE_FWD, 5, 0);
    case 18: return RTM_S2A(MODE_FWD, 5, 2);
    case 20: return RTM_S2A(MODE_MODEL, 5, 0);
    case 24: return RTM_S2A(MODE_BWD, 5, 0);
    case 25: return RTM_S2A(MODE_BWD, 5, 1);
    case 26: return RTM_S2A(MODE_BWD, 5, 2);
    case 27: return RTM_S2A(MODE_BWD, 5, 3);
    case 28: return RTM_S2A(MODE_BORN, 5, 0);
  }
#undef RTM_S2A
  return cudaErrorInvalidValue;
}

cudaError_t launch_step2p(int mode, int tile_z, const CUtensorMap &mv, const CUtensorMap &md,
                          const CUtensorMap &mc, const Step2Args &A, const Step2RT &rt, int B,
                          cudaStream_t st) {
  if (tile_z != 24 && tile_z != 16) return cudaErrorInvalidValue;
  const long long ntl = (long long)B * A.g.ntx2 * A.g.ntz2;
  if (ntl < 1 || ntl > (1LL << 30)) return cudaErrorInvalidValue;
  const int ntiles = (int)ntl;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  // per (kernel instance, device): the shared-memory opt-in and the number of
  // blocks resident at once (launches come from several request threads;
  // computing either twice is harmless)
  static std::atomic<int> resident[8][64];
  const size_t smem = step2p_smem_bytes(tile_z);
  dim3 block(32, NTH / 32);
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
      if (per_sm < 1) return cudaErrorInvalidConfiguration;
      nres = per_sm * nsm;
      resident[slot][dev].store(nres, std::memory_order_release);
    }
    const int grid = ntiles < nres ? ntiles : nres;
    kernel<<<grid, block, smem, st>>>(mv, md, mc, A, rt, ntiles);
    return cudaGetLastError();
  };
  const int h = tile_z == 16 ? 4 : 0;
  switch (mode) {
    case MODE_FWD: return h ? launch(k_step2p<MODE_FWD, 3>, 4) : launch(k_step2p<MODE_FWD, 4>, 0);
    case MODE_MODEL: return h ? launch(k_step2p<MODE_MODEL, 3>, 5) : launch(k_step2p<MODE_MODEL, 4>, 1);
    case MODE_BWD: return h ? launch(k_step2p<MODE_BWD, 3>, 6) : launch(k_step2p<MODE_BWD, 4>, 2);
    case MODE_BORN: return h ? launch(k_step2p<MODE_BORN, 3>, 7) : launch(k_step2p<MODE_BORN, 4>, 3);
  }
  return cudaErrorInvalidValue;
}

}  // namespace rtm
