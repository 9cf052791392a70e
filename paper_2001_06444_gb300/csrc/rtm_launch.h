// rtm_launch.h — host-side launchers of the kernels (internal to the library).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "rtm_common.h"

namespace rtm {

// propagation (rtm_prop.cu)
cudaError_t launch_step(int mode, const StepArgs &A, const StepRT &rt, int B, cudaStream_t st);
cudaError_t launch_snap_store(const StepArgs &A, const float *field, int idx, int B,
                              cudaStream_t st);
cudaError_t launch_prep_c(const float *vel, float *c_all, const Geo &g, double dt, int nsample,
                          cudaStream_t st);
cudaError_t launch_vrange(const float *v, long long n, unsigned *out, cudaStream_t st);

// two-step TMA kernel (rtm_prop2.cu): maps of the current v (box with halo 8)
// and d (halo 4) buffers and of c; tile geometry
cudaError_t launch_step2(int mode, const CUtensorMap &mv, const CUtensorMap &md,
                         const CUtensorMap &mc, const Step2Args &A, const Step2RT &rt, int B,
                         cudaStream_t st);
size_t step2_smem_bytes();
// persistent two-step kernel with a two-stage copy ring (rtm_prop2p.cu):
// tile_z = 24 or 16 centre rows; maps with boxes (C2X + 16, tile_z + 16) for v
// and (C2X + 8, tile_z + 8) for d and c; one block per resident slot
cudaError_t launch_step2p(int mode, int tile_z, const CUtensorMap &mv, const CUtensorMap &md,
                          const CUtensorMap &mc, const Step2Args &A, const Step2RT &rt, int B,
                          cudaStream_t st);
size_t step2p_smem_bytes(int tile_z);
// two-step kernel, one tile per block, v^{n+1} written over v^n (rtm_prop2p.cu):
// tile_z = 24 or 32 centre rows, maps as for launch_step2p
cudaError_t launch_step2a(int mode, int tile_z, const CUtensorMap &mv, const CUtensorMap &md,
                          const CUtensorMap &mc, const Step2Args &A, const Step2RT &rt, int B,
                          cudaStream_t st);
size_t step2a_smem_bytes(int tile_z);
// bounded-wait self-test: raises *flag after waiting `ns` for bytes that never arrive
cudaError_t launch_wait_probe(int *flag, unsigned long long ns, cudaStream_t st);
int step2_tile_x();
int step2_tile_z();
int step2_ext();

// imaging and statistics (rtm_post.cu)
// Normalise each item's image (Eq. 5 with eps max(den)) and add it, in item
// order, to its sample's Kahan-compensated stack; zero num and den.
// (nsample: planes of the stacks; err: index-check flag of debug builds)
cudaError_t launch_norm_stack(float *num, float *den, const unsigned *dmax,
                              const int *item_sample, int B, float eps, long long pplane,
                              float *stack_all, float *comp_all, int nsample, int *err,
                              cudaStream_t st);
// Final image of nsample samples: (optionally) the Laplacian filter of the
// compensated stack, written compactly as [nsample][nz][nx].
cudaError_t launch_filter(const float *stack_all, const float *comp_all, int nsample, int nz,
                          int nx, int SX, float rdz2, float rdx2, int laplacian, float *out,
                          cudaStream_t st);
// Per-pixel ensemble statistics.
cudaError_t launch_ens_stats(const float *images, int n, long long npix, double *mean,
                             double *std_, float *q05, float *q95, cudaStream_t st);
// Eq. 6 / Eq. 7 maps; scratch must hold 2 unsigned long long.
cudaError_t launch_unc_maps(const double *mean, const double *std_, long long npix,
                            double *conf, double *ratio, unsigned long long *scratch,
                            cudaStream_t st);
int ens_stats_max_n();

}  // namespace rtm
