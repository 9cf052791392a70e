// rtm_common.h — structures shared by the host runtime and the kernels.
//
// Memory layout of one propagation grid (one velocity sample x one shot):
//   rows    I in [0, NZ), NZ = nz + 2 nb (padded, sponge on both sides);
//   columns stored at memory column X0 + J for padded column J in [0, NX),
//   NX = nx + 2 nb, with X0 = (4 - nb % 4) % 4 so that the first physical
//   column (memory column CP = X0 + nb) is 16-byte aligned;
//   row pitch P floats (multiple of 32, i.e. 128-byte rows);
//   every column outside [X0, X0 + NX) holds zero forever, which realises the
//   zero field beyond the padded domain.
// Physical-grid arrays (snapshots, imaging accumulators, stacks) are
// [nz][SX] with SX = nx rounded up to 4, column j at offset j.
#pragma once
#include <cstdint>

namespace rtm {

// Debug builds (-DRTM_DEBUG) check the index of every global access whose
// offset the kernels compute from tables or launch scalars.  An index outside
// its array skips the access, records the source line of the first failed
// check in err[1] and raises err[0] = 2; nothing traps, so the context stays
// usable and the call reports the failure.  Release builds compile the checks
// away.
#ifdef RTM_DEBUG
__device__ __forceinline__ bool dbg_in(long long i, long long n, int *err, int line) {
  if (i >= 0 && i < n) return true;
  if (err) {
    atomicCAS(err + 1, 0, line);
    atomicExch(err, 2);
  }
  return false;
}
#define RTM_IN(i, n, err) ::rtm::dbg_in((long long)(i), (long long)(n), (err), __LINE__)
#else
#define RTM_IN(i, n, err) true
#endif

// Array lengths in elements, for the index checks of debug builds only.
struct DbgLen {
  long long items;    // item slots B: item tables, field planes, num / den planes, dmax
  long long nshot;    // shots: source tables, seismogram shots
  long long nsample;  // planes of c_all
  long long snap;     // elements of snap
  long long smax;     // entries of smax
  long long rent;     // entries of rtile_ent / rext_ent
  long long rcen;     // entries of rcen_ent
  long long refl;     // elements of refl
  long long rec_out;  // elements of rec_out
};

constexpr int TX = 128;   // tile width  (memory columns) of the step kernel
constexpr int TZ = 32;    // tile height (rows)
constexpr int HALO = 4;   // stencil radius (8th order)
constexpr int SW = TX + 2 * HALO;
constexpr int SH = TZ + 2 * HALO;
constexpr int STEP_THREADS = 256;  // 32 x 8: 4 columns x 4 rows per thread

struct Geo {
  int NZ, P, X0, NX, nb;  // padded grid
  int nz, nx, SX, CP;     // physical grid and its memory column origin
  int ntx, ntz;           // tiles per grid (single-step kernel)
  int ntx2, ntz2;         // tiles per grid (two-step kernels)
  int tz2;                // centre rows of a two-step tile (24, or 16 for the persistent kernel)
  long long plane;        // NZ * P   (floats)
  long long pplane;       // nz * SX  (elements)
};

struct Coef {
  float c0;     // a0 (1/dx^2 + 1/dz^2) (the kernels subtract the centre per ring instead)
  float ax[4];  // a_m / dx^2
  float az[4];  // a_m / dz^2
  int iso;      // dx == dz: both directions' neighbours are summed before the centre is
                // subtracted (one ring of 4 neighbours per m), else each direction alone
};

// Arguments of one batched launch over B items (blockIdx.z = item slot).
struct StepArgs {
  Geo g;
  Coef k;
  const float *gx, *gz;      // sponge factors per memory column / row
  const float *c_all;        // [nsample][plane]  (v dt)^2, zero outside
  const int *item_sample;    // [B]
  const int *item_shot;      // [B]
  float *fa;                 // [B][plane] current field v^n (read)
  float *fb;                 // [B][plane] receives the new field v^{n+1}
  float *fd;                 // [B][plane] time difference d^n = v^n - v^{n-1}, updated in place
  const int *src_row, *src_col;  // [nshot] memory coordinates of each source
  const float *wav;          // [nt] wavelet
  float src_scale;           // 1 / (dx dz)
  const int *rtile_ptr;      // [ntx*ntz + 1] receivers per tile (CSR)
  const int2 *rtile_ent;     // {local offset (row*TX + col), receiver index}
  int nrec, nt;
  const float *seis;         // [nshot][nt][nrec] data injected backward
  float *rec_out;            // [B][nt][nrec] recorded traces (modelling)
  void *snap;                // [B][nsnap][nz][SX] stored source snapshots
  int snap_dtype;            // 0 f32, 1 bf16, 2 f16
  int nsnap;
  unsigned *smax;            // [B][nsnap] max |S^k| as float bits
  float *num, *den;          // [B][pplane] imaging accumulators
  unsigned *dmax;            // [B] max of den as float bits
  const float *refl;         // [nz][nx] reflectivity m of the Born operator
  int *err;                  // debug builds: index-check flag (may be null)
  DbgLen len;                // debug builds: array lengths
};

// Per-launch scalars.
struct StepRT {
  int n;          // forward: time index of the update (u^{n+1} produced)
                  // backward: k of the produced field w^k
  int snap_idx;   // forward: store the CURRENT field u^n as snapshot snap_idx (-1 none)
  int max_idx;    // forward: reduce max |u^{n+1}| into slot max_idx (-1 none)
  int img_idx;    // backward: image with snapshot img_idx (-1 none); Born:
                  // inject c m S from snapshot img_idx into the new field
  int dmax_flag;  // backward: after imaging, reduce max(den) into dmax
};

// Arguments of one launch of the two-step kernel (blockIdx.z = item slot).
// Receiver lists are per two-step tile, with offsets r * EX + c in the
// tile's extended region (the tile plus a 4-point ring).
struct Step2Args {
  Geo g;
  Coef k;
  const float *gx, *gz;
  const float *c_all;
  const int *item_sample, *item_shot;
  int one_sample;                // every item uses sample 0 (no lookup before the copies)
  float *v_out;                  // [B][plane] receives v^{n+2}
  float *d_out;                  // [B][plane] receives d^{n+2}
  const float *v_in, *d_in;      // [B][plane] v^n, d^n (read through the tensor maps; the
                                 // one-tile-per-block kernel prefetches from them into L2)
  const int *src_row, *src_col;
  const float *wav;
  float src_scale;
  const int *rext_ptr;           // receivers in each tile's extended region
  const int2 *rext_ent;
  const int *rcen_ptr;           // receivers in each tile's centre
  const int2 *rcen_ent;
  int nrec, nt;
  const float *seis;
  float *rec_out;
  void *snap;
  int snap_dtype;
  int nsnap;
  unsigned *smax;
  float *num, *den;
  unsigned *dmax;
  int *err;                      // set to 1 if a bounded wait gave up (2: debug index check)
  const float *refl;             // [nz][nx] reflectivity of the Born operator
  DbgLen len;                    // debug builds: array lengths
};

struct Step2RT {
  int t1, t2;          // sample index injected / recorded at substeps 1 and 2
  int snap_in_idx;     // store the input field (deferred; any dtype) as this snapshot
  int snap_mid_idx;    // store the intermediate field (FP32 only)
  int snap_out_idx;    // store the output field (FP32 only)
  int max_out_idx;     // reduce max |output| into this scale slot (half precision)
  int img_mid_idx;     // image with the intermediate field (backward); Born:
                       // inject c m S from this snapshot at substep 1
  int img_out_idx;     // image with the output field (backward); Born: at substep 2
  int img_in_idx;      // image with the INPUT field v^n (backward; its operands' loads can
                       // start before the tile copies land)
  int dmax_flag;       // reduce max(den) after the imaging with 1: the intermediate,
                       // 2: the output, 3: the input field
  int reverse;         // walk the tile list from its end (snake order over launches)
  int pdl;             // launched as a programmatic dependent of the previous launch: read
                       // its outputs only after griddepcontrol.wait
  int ahead;           // one-tile-per-block kernel: blocks resident at once (each block
                       // prefetches into L2 the tile of the block `ahead` launches later);
                       // 0 = no prefetch
};

enum { MODE_FWD = 0, MODE_MODEL = 1, MODE_BWD = 2, MODE_BORN = 3 };

}  // namespace rtm
