/*
 * rtm.h — C ABI of the GB300 reverse-time-migration (RTM) library.
 *
 * The library computes the data-parallel stage of the uncertainty-quantified
 * seismic imaging workflow of "A workflow for seismic imaging with quantified
 * uncertainty" (arXiv 2001.06444): for every velocity sample of an ensemble and
 * every shot, 2D constant-density acoustic modelling (§2.2, Eq. 4, discretised
 * 2nd order in time and 8th order in space as stated in §3), reverse-time
 * propagation of the recorded data (§3, the adjoint problem), the
 * source-normalised zero-lag cross-correlation imaging condition (§2.2, Eq. 5),
 * shot stacking and the Laplacian filter on the brute stack (§3), and per-pixel
 * ensemble statistics of the images (§2.3).
 *
 * Discrete definition (the paper leaves these unstated; one reading is fixed):
 *   padded grid NZ x NX = (nz + 2 nb) x (nx + 2 nb), sponge of nb cells on all
 *   four sides outside the physical grid, velocity edge-replicated into it;
 *   c = (v dt)^2;  L = 8th-order central Laplacian with coefficients
 *   {-205/72, 8/5, -1/5, 8/315, -1/560} / h^2 per axis, zero beyond the padded
 *   grid;  sponge g = g_x g_z, g_1(k) = exp(-(0.015 (nb - k))^2) at distance k
 *   from the outer edge (k < nb), 1 inside;  h = sqrt(g);
 *   u^{n+1} = h (2 h u^n + c L(h u^n)) - g^2 u^{n-1} + c f^n,
 *   f^n = wavelet[n] / (dx dz) at the source cell, u^0 = u^{-1} = 0,
 *   trace sample d[n][r] = u^{n+1}(receiver r), n = 0 .. nt-1.
 *   Backward (exact discrete adjoint, the same recurrence):
 *   w^k = h (2 h w^{k+1} + c L(h w^{k+1})) - g^2 w^{k+2} + c R^T d[k-1],
 *   k = nt .. 1, w^{nt+1} = w^{nt+2} = 0.
 *   Imaging set K = { k : 1 <= k <= nt, k mod isnap == 0 }:
 *   num = sum_K S^k w^k, den = sum_K (S^k)^2 with S^k = u^k (optionally
 *   quantised), I_shot = num / (den + eps max(den)), stack = sum over shots,
 *   optional filter I_f = -(D_zz + D_xx) I_stack (3-point, replicated edges).
 *
 * Conventions for every call:
 *   - Arrays are row-major, x fastest: velocity / image [nz][nx],
 *     seismograms [shot][nt][nrec].
 *   - Large arrays (velocity, seismograms, images, statistics) may be device
 *     memory or host memory; host buffers are staged through device memory on
 *     the given stream and the call then synchronises that stream.  Device
 *     buffers are used in place, the call is asynchronous on `stream` (a
 *     cudaStream_t, NULL = the legacy default stream) unless stated otherwise.
 *     A migration or Born modelling given the legacy default stream, whose
 *     launch configuration captures phases into CUDA graphs, runs on a stream
 *     the context owns, after the work already on the legacy stream and before
 *     later work there (events join the two): the legacy stream cannot be
 *     captured.
 *   - Acquisition arrays (source and receiver indices, the wavelet) are small
 *     and are always HOST memory; they are copied during the call.
 *   - The caller owns every pointer it passes.  The library owns its work
 *     buffers (wavefields, snapshot store, partial images), which live in a
 *     stream-ordered pool of the context and are reused across calls.
 *   - Every call returns an rtm_status; no call aborts the process.  After an
 *     error, rtm_last_error(ctx) describes it.
 *   - One context serves one device and may be used from one host thread at a
 *     time (the request loop has its own worker thread inside).
 */
#ifndef RTM_H
#define RTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RTM_OK = 0,
  RTM_ERR_ARG = 1,     /* bad shape, null pointer, index outside the physical grid */
  RTM_ERR_CFL = 2,     /* the velocity violates the leapfrog stability bound       */
  RTM_ERR_NOMEM = 3,   /* the work can never fit the context's memory budget       */
  RTM_ERR_BUSY = 4,    /* request queue full; context still running requests        */
  RTM_ERR_TIMEOUT = 5, /* a bounded wait expired                                    */
  RTM_ERR_CUDA = 6,    /* a CUDA runtime call failed                                */
  RTM_ERR_STATE = 7    /* unknown ticket or context state                           */
} rtm_status;

enum { RTM_SNAP_F32 = 0, RTM_SNAP_BF16 = 1, RTM_SNAP_F16 = 2 };

enum { RTM_REQ_QUEUED = 0, RTM_REQ_RUNNING = 1, RTM_REQ_DONE = 2, RTM_REQ_FAILED = 3 };

typedef struct rtm_ctx rtm_ctx;

/* Grid of one migration (§4.1 describes the experiments by extent and
 * velocities; spacing and step count are the caller's).  nx, nz: physical
 * cells; nb: sponge width added on every side; dx, dz in m; dt in s;
 * nt: number of time updates. */
typedef struct {
  int nx, nz, nb;
  double dx, dz, dt;
  int nt;
} rtm_grid;

/* Acquisition (Listing 1 of §4.3 loops over shot locations; §4.1/§4.2 record
 * with near-surface hydrophones).  Indices are PHYSICAL grid cells:
 * 0 <= ix < nx, 0 <= iz < nz.  All pointers are host memory.  One receiver
 * spread and one wavelet (nt samples, wavelet[n] = w(n dt)) serve all shots. */
typedef struct {
  int nshot;
  const int *src_ix, *src_iz;   /* [nshot] */
  int nrec;
  const int *rec_ix, *rec_iz;   /* [nrec] */
  const float *wavelet;         /* [nt] */
} rtm_acq;

/* Migration options.  isnap: imaging interval (>= 1); snap_dtype: RTM_SNAP_*,
 * storage of the forward snapshots S^k (F16: q = RN(S/s), s = max|S^k| / 2^15;
 * BF16: s = max|S^k|; F32: exact); eps: stabiliser of the source
 * normalisation of Eq. 5 (typical 1e-6); laplacian: 1 applies the §3 filter.
 * checkpoint: 0 keeps every snapshot of a shot on the device; C > 0 keeps
 * only the wavefield state every C steps (C rounded up to even) and, in the
 * backward pass, recomputes each C-step segment's snapshots from its state
 * before imaging it, trading one extra forward pass for memory (the image is
 * bit-identical); -1 picks the C that needs the least memory. */
typedef struct {
  int isnap;
  int snap_dtype;
  double eps;
  int laplacian;
  int checkpoint;
} rtm_opts;

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * device memory the context may hold for work buffers (0 = 85% of the free
 * memory at creation).  Admission trusts the budget: a caller that allocates
 * device memory of its own after creating the context should pass a budget
 * that leaves room for it, else work admitted near the budget can fail with
 * RTM_ERR_CUDA (out of memory).  Returns RTM_ERR_ARG for a null ctx pointer
 * or a bad device, RTM_ERR_CUDA if the device cannot be initialised. */
int rtm_ctx_create(rtm_ctx **ctx, int device, size_t hbm_budget_bytes);

/* Destroy a context: cancels queued requests, waits (bounded, 600 s) for
 * running ones, frees every buffer it owns.  If requests are still running
 * after the bound, returns RTM_ERR_BUSY and leaves the context alive (the
 * call may be repeated).  NULL is accepted. */
int rtm_ctx_destroy(rtm_ctx *ctx);

/* Cap the number of (sample, shot) migrations the context keeps in flight at
 * once (0 = as many as the memory budget holds).  More items per launch hide
 * latency; fewer keep the working set in L2.  Returns RTM_ERR_ARG if
 * max_items < 0. */
int rtm_ctx_set_batch(rtm_ctx *ctx, int max_items);

/* Counters of the propagation kernels, accumulated while profiling is on.
 * step_ms is device time measured with CUDA events around each run of
 * back-to-back step launches (forward or backward phase of a batch);
 * step_bytes counts the algorithmic bytes of those launches: 16 B per padded
 * point update (read u^n, u^{n-1}, c; write u^{n+1}), plus b per physical
 * pixel for each snapshot stored or read (b = 4 or 2) and 16 B per physical
 * pixel per imaging step (num and den read and written).  launches counts
 * every kernel the library launched.  codec_ms and codec_bytes are the same
 * for the codec kernels of rtm_compress / rtm_decompress: device time of
 * each kernel, and its algorithmic bytes (the floats read or written plus
 * the stream bytes written or read).  eik_ms and eik_updates are the device
 * time of the traveltime solver launches of rtm_eikonal and the node updates
 * they made (4 sweeps x nodes per iteration, the last one included). */
typedef struct {
  long long step_launches;
  double step_ms;
  double step_bytes;
  double point_updates;
  long long launches;
  long long migrations;
  long long codec_launches;
  double codec_ms;
  double codec_bytes;
  long long eik_launches;
  double eik_ms;
  double eik_updates;
  long long graph_launches;  /* phases replayed as one captured CUDA graph (counted always) */
  long long requests_peak_running;  /* most request-loop requests running at once */
  long long requests_backfilled;    /* requests started past an older one waiting for memory */
} rtm_stats;

/* Turn profiling on (1) or off (0).  With profiling on, every migration
 * call synchronises its stream at the end to read its events. */
int rtm_ctx_set_profiling(rtm_ctx *ctx, int on);

/* Copy the counters into *out; reset them if reset != 0. */
int rtm_ctx_stats(rtm_ctx *ctx, rtm_stats *out, int reset);

/* Choose how migrations shaped like (grid, acq, opts) are launched on this
 * context, by timing short trial migrations (trial_steps time steps, 64 if
 * <= 0) of every candidate on synthetic inputs:
 *   - the propagation kernel and its tile: the two-step kernel with one
 *     120 x 24 tile per block (kernel 2), with or without each block
 *     prefetching into L2 the tile that a later block will load; the
 *     persistent two-step kernel (kernel 3: two blocks per SM walk the tile
 *     list, the copies of the next tile overlapping the current one) with
 *     120 x 24 or 120 x 16 centre tiles; the two-step kernel with one tile
 *     per block that writes v^{n+1} over v^n in shared memory (kernel 4),
 *     which fits 120 x 24 or 120 x 32 tiles at 3 blocks per SM; or the
 *     single-step kernel (kernel 1);
 *   - the number of migrations in flight;
 *   - whether each phase of a batch is captured and replayed as a CUDA graph.
 * The fastest is used by later rtm_migrate, rtm_migrate_ensemble and
 * request-loop calls with the same grid, nt, isnap and snapshot format.  All
 * candidates give bit-identical results.
 * choice (nullable, 5 ints): {kernel 1 to 4, items cap (0 = memory), graph 0
 * or 1, tile height 16, 24 or 32, L2 prefetch 0 or 1}.  Synchronises the
 * stream. */
int rtm_autotune(rtm_ctx *ctx, const rtm_grid *grid, const rtm_acq *acq,
                 const rtm_opts *opts, int trial_steps, int *choice, void *stream);

/* Forward modelling (§2.2, Eq. 4 with the wavelet as source term; Listing 1,
 * `isotropicAcousticModeling`).  vel: [nz][nx] m/s; shot: index into acq, or
 * -1 for every shot of acq (advanced side by side); seis: output
 * [nt][nrec] for one shot, [nshot][nt][nrec] for all, with
 * d[n][r] = u^{n+1}(receiver r).  Checks the CFL bound of §3 (RTM_ERR_CFL)
 * before any launch. */
int rtm_model(rtm_ctx *ctx, const rtm_grid *grid, const float *vel,
              const rtm_acq *acq, int shot, float *seis, void *stream);

/* Device memory a migration needs: *call_bytes once per call (model tables,
 * stacks) and *item_bytes per (sample, shot) migration in flight (fields,
 * snapshot store, imaging accumulators).  A call runs with at least one item
 * in flight, so it needs call_bytes + item_bytes of the context budget; more
 * items in flight raise throughput.  No device work; RTM_ERR_ARG on bad
 * arguments. */
int rtm_plan_bytes(const rtm_grid *grid, const rtm_acq *acq, const rtm_opts *opts,
                   int nsample, size_t *call_bytes, size_t *item_bytes);

/* Reverse time migration of all shots of acq over one velocity model
 * (§2.2 Eq. 5 imaging, §3 Laplacian on the brute stack; Listing 1 loop).
 * seis: [nshot][nt][nrec] observed data; image: [nz][nx] output (the filtered
 * stack if opts->laplacian, else the plain stack).  Shots are processed in
 * batches sized to the memory budget; the stack is Kahan-compensated FP32 in
 * shot order, so the result does not depend on the batch size. */
int rtm_migrate(rtm_ctx *ctx, const rtm_grid *grid, const float *vel,
                const rtm_acq *acq, const float *seis, const rtm_opts *opts,
                float *image, void *stream);

/* Migration of the same shots over an ensemble of nsample velocity models
 * (the Monte Carlo loop of §2 / §3 stage 2).  vels: [nsample][nz][nx];
 * images: [nsample][nz][nx].  All (sample, shot) migrations are scheduled as
 * independent work items; images[s] equals rtm_migrate of vels[s]. */
int rtm_migrate_ensemble(rtm_ctx *ctx, const rtm_grid *grid, int nsample,
                         const float *vels, const rtm_acq *acq,
                         const float *seis, const rtm_opts *opts,
                         float *images, void *stream);

/* Born (linearised) modelling, the adjoint of the imaging numerator of Eq. 5
 * and the forward operator of least-squares migration: the source
 * wavefield of each shot of acq is propagated in vel and kept at the imaging
 * steps k (k mod isnap == 0) in opts->snap_dtype, and a perturbation field,
 * at rest at first, is driven at those steps by the secondary source
 * c m S^k (c = (v dt)^2, m = refl [nz][nx] at each physical pixel) and
 * recorded like rtm_model: seis [nshot][nt][nrec], d[n][r] = du^{n+1}(r).
 * <born(m), d> equals <m, num(d)> where num is the migration's
 * unnormalised numerator.  opts->eps and opts->laplacian are not used;
 * opts->checkpoint must be 0 (RTM_ERR_ARG).  Arrays host or device; checks
 * the CFL bound like rtm_migrate. */
int rtm_born(rtm_ctx *ctx, const rtm_grid *grid, const float *vel, const rtm_acq *acq,
             const float *refl, const rtm_opts *opts, float *seis, void *stream);

/* The adjoint of rtm_born (the gradient operator of least-squares
 * migration): the imaging numerator of Eq. 5, sum over the shots of sum over
 * the imaging steps of S^k w^k, with no illumination normalisation and no
 * Laplacian filter (opts->eps and opts->laplacian are not used).  Same
 * arguments and checks as rtm_migrate; image [nz][nx].  With the same grid,
 * velocity, acquisition and options, <rtm_born(m), d> = <m,
 * rtm_migrate_adjoint(d)> up to FP32 rounding, in every snapshot format
 * (both read the same stored snapshots). */
int rtm_migrate_adjoint(rtm_ctx *ctx, const rtm_grid *grid, const float *vel,
                        const rtm_acq *acq, const float *seis, const rtm_opts *opts, float *image,
                        void *stream);

/* Least-squares migration: the reflectivity m [nz][nx] that minimises
 * ||B m - d||^2 over niter iterations of conjugate gradients on the normal
 * equations (CGLS), starting from m = 0, with B = rtm_born and B^T =
 * rtm_migrate_adjoint under the same grid, velocity, acquisition and
 * options.  This is the least-squares counterpart of the migration of §2.2
 * (Eq. 5 is one application of B^T followed by a normalisation).  Each
 * iteration costs one Born modelling and one adjoint migration; vector
 * updates and inner products run on the device (FP64 inner products, fixed
 * order).  seis [nshot][nt][nrec] and refl: host or device.  misfit (host,
 * nullable, niter + 1 values) receives ||d - B m_k||^2 after k iterations.
 * opts->checkpoint must be 0.  Stops early (filling misfit) if the
 * gradient vanishes.  Synchronises the stream. */
int rtm_lsrtm(rtm_ctx *ctx, const rtm_grid *grid, const float *vel, const rtm_acq *acq,
              const float *seis, const rtm_opts *opts, int niter, float *refl, double *misfit,
              void *stream);

/* Per-pixel statistics of n images (§2.3; stage 3 of §3): mean and standard
 * deviation (divisor n-1; 0 when n == 1) reduced in FP64, and the 5% and 95%
 * quantiles (linear interpolation between order statistics at h = (n-1) p).
 * images: [n][npix] float; mean, std: [npix] double; q05, q95: [npix] float. */
int rtm_ensemble_stats(rtm_ctx *ctx, const float *images, int n, long npix,
                       double *mean, double *std_, float *q05, float *q95,
                       void *stream);

/* Uncertainty maps of Eqs. 6 and 7 (§2.3) from a standard-deviation map and
 * a mean map: c = (s_max - s) / (s_max - s_min) (1 where s_max == s_min) and
 * r = s / mean (0 where mean == 0).  All arrays [npix] double. */
int rtm_uncertainty_maps(rtm_ctx *ctx, const double *mean, const double *std_,
                         long npix, double *conf, double *ratio, void *stream);

/* A migration request for the request loop (continuous batching).  All
 * pointers must stay valid until rtm_poll reports DONE or FAILED; vel, seis
 * and image are device memory. */
typedef struct {
  rtm_grid grid;
  const float *vel;
  rtm_acq acq;
  const float *seis;
  rtm_opts opts;
  float *image;
} rtm_request;

/* Queue a migration request; its shots join the device work of requests
 * already in flight as soon as memory for their snapshot buffers is free.
 * Requests start in arrival order, except that while the oldest waits for
 * memory a later one that fits in what is free may start first (at most 16
 * times per waiting request).  A request whose device-side wait gave up ends
 * FAILED with RTM_ERR_TIMEOUT; other requests are not affected.
 * Returns RTM_ERR_NOMEM if the request could never fit the budget,
 * RTM_ERR_BUSY if the queue is full, RTM_ERR_CFL / RTM_ERR_ARG as rtm_migrate. */
int rtm_submit(rtm_ctx *ctx, const rtm_request *req, uint64_t *ticket);

/* State of a request (RTM_REQ_*), waiting up to timeout_ms for it to reach
 * DONE or FAILED (0 = do not wait).  Returns RTM_ERR_TIMEOUT if the wait
 * expired first (the state is still written), RTM_ERR_STATE for an unknown
 * ticket.  A DONE or FAILED ticket is forgotten after it is reported. */
int rtm_poll(rtm_ctx *ctx, uint64_t ticket, int *state, int timeout_ms);

/* Forward modelling of one shot without allocating device memory (the
 * paper has no counterpart; this serves callers that cannot allocate while
 * they run, e.g. inside a host framework whose allocator owns all device
 * memory, or in a real-time loop where an allocation could stall the
 * device).  Same arguments and result as rtm_model with one shot, but vel
 * [nz][nx] and seis [nt][nrec] must be device memory and no context is used:
 * the work runs in a 32 MiB scratch array that the library holds on every
 * device that loads it.  The device is the current one.  The first call on a
 * device looks up the scratch address (and may load the library's device
 * code), so make it before any stream capture.  The call synchronises the
 * stream once for the stability check, then returns with the modelling
 * queued.  Every call shares the scratch and overwrites it, so calls whose
 * work overlaps on the GPU race.  Returns RTM_ERR_NOMEM if the padded grid
 * needs more than the scratch (about 2 M padded points), RTM_ERR_ARG for bad
 * arguments or host pointers, RTM_ERR_CFL, RTM_ERR_CUDA. */
int rtm_model_noalloc(const rtm_grid *grid, const float *vel, const rtm_acq *acq,
                      int shot, float *seis, void *stream);

/* Self-test of device-side failure detection (no counterpart in the paper).
 * The propagation kernels wait on an mbarrier for their TMA copies with a
 * bound of about one second; a wait that runs out raises an error flag and
 * the block returns, so the context stays usable.  This call runs the same
 * bounded wait on a barrier that no copy will complete, for wait_ms
 * milliseconds, and stores in *raised 1 if the flag came back to the host.
 * Synchronises the stream. */
int rtm_selftest_wait(rtm_ctx *ctx, int wait_ms, int *raised, void *stream);

/* Test hook for the reporting of device-side failures (no counterpart in the
 * paper).  The next `count` migration or modelling calls on this context
 * (direct calls, request-loop requests or autotuner trials, in the order they
 * start) run normally but begin with their wait-timeout flag already raised,
 * exactly as if one of their bounded device-side waits had given up.  So the
 * path that reports it can be tested without making a GPU wait run out: a
 * call that synchronises returns RTM_ERR_TIMEOUT itself, an asynchronous
 * call's flag is returned by the next call on the context, a request ends
 * FAILED with RTM_ERR_TIMEOUT, and no other call or request is affected.
 * count = 0 cancels what is left; RTM_ERR_ARG for count < 0. */
int rtm_ctx_inject_wait_timeout(rtm_ctx *ctx, int count);

/* ------------------------------------------------------------- codec --
 * Error-bounded compression of velocity models, images and seismograms
 * (§3 and §4.2, Tables 1-2: the workflow stores and moves its arrays
 * through a transform block codec, in a fixed-accuracy mode with an absolute
 * tolerance and in a lossless mode).  Each n0 x n1 float array (row-major)
 * becomes one stream: 4 x 4 blocks, a block exponent and 28-bit fixed point
 * (fixed accuracy) or the float bits as order-preserving integers
 * (lossless), an exactly reversible integer transform, and bit-plane coding
 * of the coefficients down to the lowest plane the tolerance needs.  Fixed
 * accuracy returns every element within max(tol, 2^(e-23)) of its input,
 * where max |x| over its block is f 2^e with f in [0.5, 1); lossless returns
 * the input bits exactly (NaN, infinities and -0 included).  The stream
 * layout (header, chunk index, bit section) is given in the library's codec
 * source.  Both calls synchronise the stream before they return. */

/* Bytes one stream of an n0 x n1 array can take at most (0 if the shape is
 * not supported: n0, n1 >= 1 and fewer than 2^32 / 20 blocks of 4 x 4). */
uint64_t rtm_compress_bound(long long n0, long long n1);

/* Compress count arrays data [count][n0][n1] (host or device).  tol > 0:
 * fixed accuracy with absolute tolerance tol; tol == 0: lossless.  Stream i
 * is written at out + i * out_stride (host or device; out_stride >=
 * rtm_compress_bound(n0, n1), a multiple of 16; out 16-byte aligned) and its
 * byte count to out_bytes[i] (host).  An array holding a NaN or an infinity
 * cannot be coded with tol > 0: its out_bytes is 0 and the call returns
 * RTM_ERR_ARG after coding the others.  Device scratch of about
 * 1.25 x the input is taken from the context's pool for the call. */
int rtm_compress(rtm_ctx *ctx, const float *data, long long count, long long n0, long long n1,
                 double tol, void *out, uint64_t out_stride, uint64_t *out_bytes,
                 void *stream);

/* Decompress count streams in + i * in_stride (host or device; in_stride a
 * multiple of 16 and at least the stream's bytes; in 16-byte aligned) into
 * data [count][n0][n1] (host or device); count <= 65535.  The mode and the
 * tolerance come from each stream's header.  RTM_ERR_ARG names the first
 * stream that is malformed or was not made for n0 x n1 (the elements of its
 * damaged chunks are then unspecified).  Device scratch of 4 bytes per 4 x 4
 * block of up to 2^24 blocks at a time (the decode's block lists), plus 288
 * bytes per stream, is taken from the context's pool for the call. */
int rtm_decompress(rtm_ctx *ctx, const void *in, uint64_t in_stride, long long count,
                   long long n0, long long n1, float *data, void *stream);

/* ----------------------------------------------------------- eikonal --
 * First-arrival traveltimes: the forward operator of the tomography stage
 * (§2.1 Eq. 1: traveltimes of the proposed velocity model from the eikonal
 * equation |grad T| = 1/v; §3: solved for every source at each sampler
 * iteration, which dominates that stage).  The first-order upwind scheme on
 * the nz x nx grid (spacings dz, dx in m): with a, b the smaller vertical and
 * horizontal neighbour times, ((T-a)^+/dz)^2 + ((T-b)^+/dx)^2 = (1/v)^2, and
 * T = 0 at the source node.  Its discrete solution is unique (the one fast
 * marching computes); the device reaches it by parallel fast sweeping, one
 * (sample, source) problem per CTA, in FP32.
 * vel: [nsample][nz][nx] m/s, host or device, positive and finite
 * (RTM_ERR_ARG otherwise).  Sources and receivers: host arrays of node
 * indices.  times: [nsample][nsrc][nrec] s at the receivers, fields:
 * [nsample][nsrc][nz][nx] s, either may be NULL but not both; host or device.
 * flags: where each problem's work field lives.  0 chooses: in shared
 * memory (one problem per SM, the lowest latency per solve) when the
 * problems fit one per SM, else in an L2-resident device buffer (many
 * problems per SM, the highest throughput); RTM_EIK_OFFCHIP or RTM_EIK_SHARED
 * force one (fields larger than shared memory always stay off chip).
 * max_iter (<= 0: 64) caps the iterations of four sweeps; iters (host,
 * nullable, [nsample * nsrc]) receives the iterations each problem took to
 * reach its fixed point (the last one changing nothing), -1 at the cap, in
 * which case the call returns RTM_ERR_STATE after writing every output.
 * Synchronises the stream. */
#define RTM_EIK_OFFCHIP 1
#define RTM_EIK_SHARED 2
int rtm_eikonal(rtm_ctx *ctx, int nz, int nx, double dz, double dx, int nsample,
                const float *vel, int nsrc, const int *src_iz, const int *src_ix, int nrec,
                const int *rec_iz, const int *rec_ix, int max_iter, int flags, float *times,
                float *fields, int *iters, void *stream);

/* Text of the last error on this context (never NULL). */
const char *rtm_last_error(rtm_ctx *ctx);

/* The largest v dt / min(dx, dz) the scheme is stable for: 2 / sqrt(2 * 2048/315)
 * for square cells (§3: every RTM checks its own CFL condition).  For
 * rectangular cells the bound the library applies is
 * v dt sqrt((1/dx^2 + 1/dz^2) 2048/315) <= 2. */
double rtm_cfl_limit(void);

#ifdef __cplusplus
}
#endif

#endif /* RTM_H */
