// The five passes of the projection G with the transforms in double-float
// arithmetic (df64.cuh): the kernels of the CG matrix-vector product when a
// solve asks for FH_ARITH_DF64. The pass bodies are those of passes.cuh with
// the element type dfc; this file holds the z passes, the tangent and value
// conversions and the set-up, kernels_df64_yx.cu the y and x passes (plane
// cells: kernels_plane.cu). The CG updates and the p . y dot product stay
// FP64. Every grid: compile-time and run-time plans, plane cells.
#include <algorithm>
#include <cmath>

#include "fft_df64.cuh"
#include "passes.cuh"

namespace fh {

namespace {

template <int M, int MODE>
__global__ void __launch_bounds__(kThreads) k_fwd_z_df(Grid g, int LB, const double* __restrict__ src,
                                                      double* __restrict__ p, double* __restrict__ x,
                                                      const df64* __restrict__ K, const CgScalars* __restrict__ cg,
                                                      dfc* __restrict__ S, const dfc* __restrict__ tw) {
  if (cg_done(cg)) return;
  fwd_z_body<M, MODE>(blockIdx.x, g, LB, src, p, x, K, cg, S, tw);
}
template <int M, int MODE>
__global__ void __launch_bounds__(kThreads) k_inv_z_df(Grid g, int LB, const dfc* __restrict__ S,
                                                      double* __restrict__ out, const double* __restrict__ p,
                                                      double* __restrict__ partials, const dfc* __restrict__ tw,
                                                      const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  inv_z_body<M, MODE>(blockIdx.x, g, LB, S, out, p, partials, tw, cg);
}

__global__ void __launch_bounds__(kThreads) k_df64_roundtrip(const double* __restrict__ in, float* __restrict__ hi,
                                                            float* __restrict__ lo, double* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const df64 v = split_double(in[i]);
    if (hi) hi[i] = v.hi;
    if (lo) lo[i] = v.lo;
    out[i] = join_df64(v);
  }
}

template <class Kern>
cudaError_t allow(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

void twiddles_to_df64(const double2* src, dfc* dst, int n) {
  // FP64 tables hold 53 significant bits, more than the 48 of double-float
  auto split = [](double v) {
    const float hi = (float)v;
    return df64{hi, (float)(v - (double)hi)};
  };
  for (int i = 0; i < n; ++i) dst[i] = dfc{split(src[i].x), split(src[i].y)};
}

cudaError_t setup_df64_kernels(const Grid& g, const Tiling& t) {
  cudaError_t e = cudaSuccess;
  const size_t zs = z_pass_smem(g, df_tiles(t));
  const int M = g.nz / 2;
#define ZCASE(V)                                                       \
  case V:                                                              \
    if ((e = allow(k_fwd_z_df<V, kZDirect>, zs))) return e;            \
    if ((e = allow(k_fwd_z_df<V, kZKApply>, zs))) return e;            \
    if ((e = allow(k_fwd_z_df<V, kZCg>, zs))) return e;                \
    if ((e = allow(k_fwd_z_df<V, kZCgFirst>, zs))) return e;           \
    if ((e = allow(k_inv_z_df<V, kIZOut>, zs))) return e;              \
    if ((e = allow(k_inv_z_df<V, kIZDot>, zs))) return e;              \
    if ((e = allow(k_inv_z_df<V, kIZRhs>, zs))) return e;              \
    break;
  FH_SWITCH_HALF_EVEN(M, ZCASE)
#undef ZCASE
  if ((e = setup_df64_yx_kernels(g, t))) return e;
  return setup_df64_batch_kernels(g, t);
}

// the packed tangent [45][N] in double-float (K_df[i] from K[i])
__global__ void __launch_bounds__(kThreads) k_tangent_to_df64(const double* __restrict__ K, df64* __restrict__ K_df,
                                                             long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    K_df[i] = split_double(K[i]);
}

cudaError_t launch_tangent_to_df64(const Grid& g, const double* K, df64* K_df, cudaStream_t s) {
  const long long count = 45LL * g.n;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (count + kThreads - 1) / kThreads;
  if (blocks > 8LL * sms) blocks = 8LL * sms;
  k_tangent_to_df64<<<(unsigned)blocks, kThreads, 0, s>>>(K, K_df, count);
  return cudaGetLastError();
}

cudaError_t launch_fwd_z_df(const Grid& g, const Tiling& t, int mode, const double* src, double* p, double* x,
                            const df64* K, const CgScalars* cg, dfc* S, const dfc* tw, cudaStream_t s) {
  const size_t smem = z_pass_smem(g, t);
  const unsigned grid = (unsigned)z_pass_ctas(g, t);
  const int M = g.nz / 2;
#define ZL(V)                                                                                                    \
  case V:                                                                                                        \
    switch (mode) {                                                                                              \
      case kZDirect: k_fwd_z_df<V, kZDirect><<<grid, kThreads, smem, s>>>(g, t.lines_z, src, p, x, K, cg, S, tw); break; \
      case kZKApply: k_fwd_z_df<V, kZKApply><<<grid, kThreads, smem, s>>>(g, t.lines_z, src, p, x, K, cg, S, tw); break; \
      case kZCg: k_fwd_z_df<V, kZCg><<<grid, kThreads, smem, s>>>(g, t.lines_z, src, p, x, K, cg, S, tw); break;         \
      case kZCgFirst: k_fwd_z_df<V, kZCgFirst><<<grid, kThreads, smem, s>>>(g, t.lines_z, src, p, x, K, cg, S, tw); break; \
      default: return cudaErrorInvalidValue;                                                                     \
    }                                                                                                            \
    break;
  FH_SWITCH_HALF(M, ZL)
#undef ZL
  return cudaGetLastError();
}

cudaError_t launch_inv_z_df(const Grid& g, const Tiling& t, int mode, const dfc* S, double* out, const double* p,
                            double* partials, const dfc* tw, const CgScalars* cg, cudaStream_t s) {
  const size_t smem = z_pass_smem(g, t);
  const unsigned grid = (unsigned)z_pass_ctas(g, t);
  const int M = g.nz / 2;
#define IZL(V)                                                                                                     \
  case V:                                                                                                          \
    switch (mode) {                                                                                                \
      case kIZOut: k_inv_z_df<V, kIZOut><<<grid, kThreads, smem, s>>>(g, t.lines_z, S, out, p, partials, tw, cg); break; \
      case kIZDot: k_inv_z_df<V, kIZDot><<<grid, kThreads, smem, s>>>(g, t.lines_z, S, out, p, partials, tw, cg); break; \
      case kIZRhs: k_inv_z_df<V, kIZRhs><<<grid, kThreads, smem, s>>>(g, t.lines_z, S, out, p, partials, tw, cg); break; \
      default: return cudaErrorInvalidValue;                                                                       \
    }                                                                                                              \
    break;
  FH_SWITCH_HALF(M, IZL)
#undef IZL
  return cudaGetLastError();
}

}  // namespace fh

extern "C" void fh_internal_set_error(const char* msg);

extern "C" int fh_df64_roundtrip(const double* in_dev, float* hi_dev, float* lo_dev, double* out_dev, long long n,
                                 void* cuda_stream) {
  fh_internal_set_error("");
  if (n < 0 || (n > 0 && (!in_dev || !out_dev))) {
    fh_internal_set_error("fh_df64_roundtrip: n < 0 or NULL in/out");
    return FH_ERR_ARG;
  }
  if (n == 0) return FH_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const long long blocks = std::min<long long>((n + fh::kThreads - 1) / fh::kThreads, 4096);
  fh::k_df64_roundtrip<<<(unsigned)blocks, fh::kThreads, 0, s>>>(in_dev, hi_dev, lo_dev, out_dev, n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    fh_internal_set_error(cudaGetErrorString(e));
    return FH_ERR_CUDA;
  }
  return FH_OK;
}
