// fh_project_static: the compatibility projection of fh_project without any
// device allocation.
//
// Some callers cannot allocate device memory: a plug-in hosted by another
// application that owns the GPU's memory budget, or a loop that by policy
// must not allocate after start-up (allocation can block, fragment a pool or
// fail late). They cannot create an fh_ctx, whose scratch comes from
// cudaMalloc. This entry point runs the same five projection kernels, but its
// only scratch (the half spectrum, plus the twiddle tables) lives in the
// file-scope arrays below, which every GPU that loads this library holds until
// the process exits.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "fh_kernels.h"

namespace fh {

// largest grid the static scratch can serve: nx * ny * nz <= kStaticMaxVoxels
constexpr long long kStaticMaxVoxels = 32768;
// 9 half spectra of nx * ny * (nz/2 + 1) <= N complex entries each: 4.5 MiB
constexpr long long kStaticSpectrum = 9 * kStaticMaxVoxels;

static __device__ __align__(256) double2 g_static_spectrum[kStaticSpectrum];
static __device__ __align__(256) double2 g_static_twiddles[kTwiddleTables];
static_assert(kTwiddleTables == 1784, "the header states the size of the static twiddle tables");

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;

// Set-up of the calling thread's current device, on every call: resolve the
// device addresses of the static arrays (they change when the device's context
// is destroyed and created again, e.g. after cudaDeviceReset) and check the
// first twiddle entry, the length-1 table, which holds (1, 0) once the tables
// are written and 0 in a fresh module; write the tables if it does not.
int static_setup(int dev, cudaStream_t s, double2** spectrum, double2** twiddles, char* msg, size_t len) {
  if (dev < 0 || dev >= kMaxDevices) {
    snprintf(msg, len, "fh_project_static: device %d outside 0..%d", dev, kMaxDevices - 1);
    return FH_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  cudaError_t e = cudaGetSymbolAddress((void**)spectrum, g_static_spectrum);
  if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)twiddles, g_static_twiddles);
  if (e != cudaSuccess) {
    snprintf(msg, len, "fh_project_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return FH_ERR_CUDA;
  }
  double2 head = make_double2(0.0, 0.0);
  e = cudaMemcpyAsync(&head, *twiddles, sizeof(double2), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && !(head.x == 1.0 && head.y == 0.0)) {
    std::vector<double2> tw(kTwiddleTables);
    fill_twiddle_table(tw.data());
    e = cudaMemcpyAsync(*twiddles, tw.data(), kTwiddleTables * sizeof(double2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) {
    snprintf(msg, len, "fh_project_static: twiddle set-up failed: %s", cudaGetErrorString(e));
    return FH_ERR_CUDA;
  }
  return FH_OK;
}

}  // namespace
}  // namespace fh

extern "C" void fh_internal_set_error(const char* msg);

extern "C" int fh_project_static(const double* A_dev, double* out_dev, int nx, int ny, int nz, double scale,
                                 const double lengths[3], void* cuda_stream) {
  using namespace fh;
  char msg[256];
  auto fail = [&](int code) {
    fh_internal_set_error(msg);
    return code;
  };
  msg[0] = 0;
  fh_internal_set_error("");
  if (!A_dev || !out_dev) {
    snprintf(msg, sizeof msg, "fh_project_static: NULL field pointer");
    return fail(FH_ERR_ARG);
  }
  if (!grid_extents_ok(nx, ny, nz)) {
    snprintf(msg, sizeof msg, "fh_project_static: grid %dx%dx%d: each extent must be 2^a or 3*2^a up to 256, and "
             "nz even with nz/2 of that form", nx, ny, nz);
    return fail(FH_ERR_ARG);
  }
  const long long n = (long long)nx * ny * nz;
  if (n > kStaticMaxVoxels) {
    snprintf(msg, sizeof msg, "fh_project_static: grid %dx%dx%d has %lld voxels, above the static scratch limit of "
             "%lld voxels; use fh_project", nx, ny, nz, n, kStaticMaxVoxels);
    return fail(FH_ERR_ARG);
  }
  if (lengths && !(lengths[0] > 0 && lengths[1] > 0 && lengths[2] > 0 && std::isfinite(lengths[0]) &&
                   std::isfinite(lengths[1]) && std::isfinite(lengths[2]))) {
    snprintf(msg, sizeof msg, "fh_project_static: box lengths must be positive");
    return fail(FH_ERR_ARG);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "fh_project_static: cudaGetDevice: %s", cudaGetErrorString(e));
    return fail(FH_ERR_CUDA);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double2* spectrum = nullptr;
  double2* twiddles = nullptr;
  int rc = static_setup(dev, s, &spectrum, &twiddles, msg, sizeof msg);
  if (rc) return fail(rc);

  Grid g{};
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.nzh = nz / 2 + 1;
  g.n = n;
  g.nspec = (long long)nx * ny * g.nzh;
  g.sx = lengths ? 1.0 / lengths[0] : 1.0;
  g.sy = lengths ? 1.0 / lengths[1] : 1.0;
  g.sz = lengths ? 1.0 / lengths[2] : 1.0;
  const Tiling t = choose_tiling(g);
  const double c = scale / (2.0 * (double)n);
  if ((e = setup_fft_kernels(g, t)) != cudaSuccess ||
      (e = launch_fwd_z(g, t, kZDirect, A_dev, nullptr, nullptr, nullptr, nullptr, spectrum,
                        twiddles, s)) !=
          cudaSuccess ||
      (e = launch_fwd_y(g, t, spectrum, twiddles, nullptr, s)) != cudaSuccess ||
      (e = launch_x_ghat(g, t, spectrum, twiddles, c, nullptr, s)) != cudaSuccess ||
      (e = launch_inv_y(g, t, spectrum, twiddles, nullptr, s)) != cudaSuccess ||
      (e = launch_inv_z(g, t, kIZOut, spectrum, out_dev, nullptr, nullptr, twiddles, nullptr, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    snprintf(msg, sizeof msg, "fh_project_static: %s", cudaGetErrorString(e));
    return fail(FH_ERR_CUDA);
  }
  return FH_OK;
}
