// rtm_noalloc.cu — forward modelling that allocates no device memory.
//
// Some callers cannot allocate device memory while they run: a host framework
// whose caching allocator already holds the whole device, a real-time loop
// where an allocation (which may synchronise the device) would break its
// timing, or a plug-in that must not change its host's memory accounting.
// For them rtm_model_noalloc models one shot in a fixed scratch area that the
// library reserves as a file-scope __device__ array (every GPU that loads the
// library holds it until the process exits).  The caller still passes the
// velocity and the seismogram buffers.  The scratch is shared by every call
// and keeps the last call's contents, so the call clears what must start at
// zero, and calls whose work overlaps on the GPU race with each other.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/rtm.h"
#include "rtm_common.h"
#include "rtm_engine.h"
#include "rtm_launch.h"

namespace {

using namespace rtm;

// Every GPU that loads the library holds this much device memory until exit.
constexpr size_t kScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_base[kMaxDevices];  // device address of g_scratch, per device

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does it; make that call outside any
// stream capture).
unsigned char *scratch_base(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_base[dev] = static_cast<unsigned char *>(p);
  }
  return g_base[dev];
}

}  // namespace

extern "C" int rtm_model_noalloc(const rtm_grid *grid, const float *vel, const rtm_acq *acq,
                                 int shot, float *seis, void *stream) {
  int rc;
  if ((rc = check_grid(nullptr, grid)) || (rc = check_acq(nullptr, grid, acq, true))) return rc;
  if (!vel || !seis || shot < 0 || shot >= acq->nshot) return RTM_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return RTM_ERR_CUDA;
  }
  if (!is_device_ptr(vel) || !is_device_ptr(seis)) return RTM_ERR_ARG;
  const Geo g = make_geo(*grid);
  const int ntiles = g.ntx * g.ntz;
  // layout of the scratch: c, three field planes, then the small tables
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = up256(off + bytes);
    return o;
  };
  const size_t o_c = take((size_t)g.plane * 4);
  const size_t o_fa = take((size_t)g.plane * 4);
  const size_t o_fb = take((size_t)g.plane * 4);
  const size_t o_fd = take((size_t)g.plane * 4);
  const size_t o_gx = take((size_t)g.P * 4);
  const size_t o_gz = take((size_t)g.NZ * 4);
  const size_t o_rp = take((size_t)(ntiles + 1) * 4);
  const size_t o_re = take((size_t)std::max(acq->nrec, 1) * sizeof(int2));
  const size_t o_wv = take((size_t)grid->nt * 4);
  const size_t o_src = take(4 * sizeof(int));   // src row, src col, item sample, item shot
  const size_t o_rng = take(4 * sizeof(unsigned));
  if (off > kScratchBytes) return RTM_ERR_NOMEM;
  unsigned char *base = scratch_base(dev);
  if (!base) return RTM_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;

  // host-side tables, built as for the allocating entry points (pageable
  // copies are staged before cudaMemcpyAsync returns)
  std::vector<float> gx, gz;
  sponge_tables(g, gx, gz);
  std::vector<int> rptr;
  std::vector<int2> rent;
  receiver_tiles(g, *acq, rptr, rent);
  const int src[4] = {acq->src_iz[shot] + g.nb, acq->src_ix[shot] + g.CP, 0, 0};
  const unsigned rng0[4] = {0u, 0x7f7fffffu, 0u, 0u};
  auto E = [](cudaError_t e) { return e == cudaSuccess; };
  if (!E(cudaMemcpyAsync(base + o_gx, gx.data(), gx.size() * 4, cudaMemcpyHostToDevice, st)) ||
      !E(cudaMemcpyAsync(base + o_gz, gz.data(), gz.size() * 4, cudaMemcpyHostToDevice, st)) ||
      !E(cudaMemcpyAsync(base + o_rp, rptr.data(), rptr.size() * 4, cudaMemcpyHostToDevice, st)) ||
      !E(cudaMemcpyAsync(base + o_re, rent.data(), rent.size() * sizeof(int2),
                         cudaMemcpyHostToDevice, st)) ||
      !E(cudaMemcpyAsync(base + o_wv, acq->wavelet, (size_t)grid->nt * 4, cudaMemcpyHostToDevice,
                         st)) ||
      !E(cudaMemcpyAsync(base + o_src, src, sizeof(src), cudaMemcpyHostToDevice, st)) ||
      !E(cudaMemcpyAsync(base + o_rng, rng0, sizeof(rng0), cudaMemcpyHostToDevice, st)))
    return RTM_ERR_CUDA;
  // stability check of §3 on the caller's velocity
  unsigned rng[4];
  if (!E(launch_vrange(vel, (long long)grid->nx * grid->nz,
                       reinterpret_cast<unsigned *>(base + o_rng), st)) ||
      !E(cudaMemcpyAsync(rng, base + o_rng, sizeof(rng), cudaMemcpyDeviceToHost, st)) ||
      !E(cudaStreamSynchronize(st)))
    return RTM_ERR_CUDA;
  if (rng[2]) return RTM_ERR_ARG;
  float vmax;
  std::memcpy(&vmax, &rng[0], 4);
  const double cn = vmax * grid->dt *
                    std::sqrt((1.0 / (grid->dx * grid->dx) + 1.0 / (grid->dz * grid->dz)) *
                              2048.0 / 315.0) / 2.0;
  if (cn > 1.0) return RTM_ERR_CFL;
  // fields start at zero: the scratch keeps whatever the last call left
  for (size_t o : {o_fa, o_fb, o_fd})
    if (!E(cudaMemsetAsync(base + o, 0, (size_t)g.plane * 4, st))) return RTM_ERR_CUDA;
  if (!E(launch_prep_c(vel, reinterpret_cast<float *>(base + o_c), g, grid->dt, 1, st)))
    return RTM_ERR_CUDA;
  StepArgs A;
  std::memset(&A, 0, sizeof(A));
  A.g = g;
  A.k = make_coef(*grid);
  A.gx = reinterpret_cast<const float *>(base + o_gx);
  A.gz = reinterpret_cast<const float *>(base + o_gz);
  A.c_all = reinterpret_cast<const float *>(base + o_c);
  // {source row, source column, item sample 0, item shot 0}: the one item
  // reads its source as entry 0 of one-entry tables
  const int *srcd = reinterpret_cast<const int *>(base + o_src);
  A.src_row = srcd;
  A.src_col = srcd + 1;
  A.item_sample = srcd + 2;
  A.item_shot = srcd + 3;
  A.wav = reinterpret_cast<const float *>(base + o_wv);
  A.src_scale = (float)(1.0 / (grid->dx * grid->dz));
  A.rtile_ptr = reinterpret_cast<const int *>(base + o_rp);
  A.rtile_ent = reinterpret_cast<const int2 *>(base + o_re);
  A.nrec = acq->nrec;
  A.nt = grid->nt;
  A.rec_out = seis;
  // lengths for the index checks of debug builds (which record nothing here:
  // the call has no flag to report; a failed check only skips its access)
  A.len.items = 1;
  A.len.nshot = 1;
  A.len.nsample = 1;
  A.len.rent = (long long)rent.size();
  A.len.rec_out = (long long)grid->nt * acq->nrec;
  float *fa = reinterpret_cast<float *>(base + o_fa), *fb = reinterpret_cast<float *>(base + o_fb);
  A.fd = reinterpret_cast<float *>(base + o_fd);
  StepRT rt{};
  rt.snap_idx = rt.max_idx = rt.img_idx = -1;
  for (int n = 0; n < grid->nt; ++n) {
    rt.n = n;
    A.fa = fa;
    A.fb = fb;
    if (!E(launch_step(MODE_MODEL, A, rt, 1, st))) return RTM_ERR_CUDA;
    std::swap(fa, fb);
  }
  return RTM_OK;
}
