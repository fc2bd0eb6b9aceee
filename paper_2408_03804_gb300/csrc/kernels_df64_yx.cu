// The y and x passes of the projection G with double-float transforms (the
// FH_ARITH_DF64 kernels of kernels_df64.cu): pass bodies of passes.cuh with
// the element type dfc, compile-time and run-time plans; plane cells go to
// kernels_plane.cu.
#include "fft_df64.cuh"
#include "passes.cuh"

namespace fh {

namespace {

// resident CTAs the y and x passes are compiled for: three with compile-time
// plans (80 registers), two with run-time plans, whose double-float odd-radix
// and Rader stages would spill at 80
template <int L>
constexpr int kMinCtasDf = L > 0 ? 3 : 2;

template <int L>
__global__ void __launch_bounds__(kThreads, kMinCtasDf<L>) k_fwd_y_df(Grid g, int BK, dfc* __restrict__ S,
                                                         const dfc* __restrict__ tw, const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  fwd_y_body<L>(blockIdx.x, g, BK, S, tw, cg);
}
template <int L>
__global__ void __launch_bounds__(kThreads, kMinCtasDf<L>) k_x_ghat_df(Grid g, int BK, dfc* __restrict__ S,
                                                          const dfc* __restrict__ tw, double scale,
                                                          const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  x_ghat_body<L>(blockIdx.x, g, BK, S, tw, scale, cg);
}
template <int L>
__global__ void __launch_bounds__(kThreads, kMinCtasDf<L>) k_inv_y_df(Grid g, int BK, dfc* __restrict__ S,
                                                         const dfc* __restrict__ tw, const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  inv_y_body<L>(blockIdx.x, g, BK, S, tw, cg);
}
template <class Kern>
cudaError_t allow(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

cudaError_t setup_df64_yx_kernels(const Grid& g, const Tiling& t) {
  cudaError_t e = cudaSuccess;
#define YCASE(V)                                                          \
  case V:                                                                 \
    if ((e = allow(k_fwd_y_df<V>, y_smem(V, t.bk_y, 3)))) return e;    \
    if ((e = allow(k_inv_y_df<V>, y_smem(V, t.bk_y, 3)))) return e;    \
    break;
  if (g.py.L) {
    if ((e = allow(k_fwd_y_df<0>, y_smem_rt(g.py, t.bk_y, 3)))) return e;
    if ((e = allow(k_inv_y_df<0>, y_smem_rt(g.py, t.bk_y, 3)))) return e;
  } else {
    FH_SWITCH_LEN(g.ny, YCASE)
  }
#undef YCASE
#define XCASE(V)                                                          \
  case V:                                                                 \
    if ((e = allow(k_x_ghat_df<V>, y_smem(V, t.bk_x, 6)))) return e;   \
    break;
  if (g.px.L) {
    if ((e = allow(k_x_ghat_df<0>, y_smem_rt(g.px, t.bk_x, 6)))) return e;
  } else {
    FH_SWITCH_LEN(g.nx, XCASE)
  }
#undef XCASE
  return cudaSuccess;
}

cudaError_t launch_fwd_y_df(const Grid& g, const Tiling& t, dfc* S, const dfc* tw, const CgScalars* cg,
                            cudaStream_t s) {
  if (g.nz == 1) return launch_plane_fwd_y(g, S, tw, cg, s);
  const int NC = (g.nzh + t.bk_y - 1) / t.bk_y;
  const unsigned grid = (unsigned)((long long)g.nx * 3 * NC);
#define YL(V)                                                                                  \
  case V:                                                                                      \
    k_fwd_y_df<V><<<grid, kThreads, y_smem(V, t.bk_y, 3), s>>>(g, t.bk_y, S, tw, cg);       \
    break;
  if (g.py.L) k_fwd_y_df<0><<<grid, kThreads, y_smem_rt(g.py, t.bk_y, 3), s>>>(g, t.bk_y, S, tw, cg);
  else FH_SWITCH_LEN(g.ny, YL)
#undef YL
  return cudaGetLastError();
}

cudaError_t launch_x_ghat_df(const Grid& g, const Tiling& t, dfc* S, const dfc* tw, double scale,
                             const CgScalars* cg, cudaStream_t s) {
  if (g.nz == 1) return launch_plane_x_ghat(g, S, tw, scale, cg, s);
  const int NC = (g.nzh + t.bk_x - 1) / t.bk_x;
  const unsigned grid = (unsigned)((long long)g.ny * NC);
#define XL(V)                                                                                         \
  case V:                                                                                             \
    k_x_ghat_df<V><<<grid, kThreads, y_smem(V, t.bk_x, 6), s>>>(g, t.bk_x, S, tw, scale, cg);      \
    break;
  if (g.px.L) k_x_ghat_df<0><<<grid, kThreads, y_smem_rt(g.px, t.bk_x, 6), s>>>(g, t.bk_x, S, tw, scale, cg);
  else FH_SWITCH_LEN(g.nx, XL)
#undef XL
  return cudaGetLastError();
}

cudaError_t launch_inv_y_df(const Grid& g, const Tiling& t, dfc* S, const dfc* tw, const CgScalars* cg,
                            cudaStream_t s) {
  if (g.nz == 1) return launch_plane_inv_y(g, S, tw, cg, s);
  const int NC = (g.nzh + t.bk_y - 1) / t.bk_y;
  const unsigned grid = (unsigned)((long long)g.nx * 3 * NC);
#define IYL(V)                                                                                 \
  case V:                                                                                      \
    k_inv_y_df<V><<<grid, kThreads, y_smem(V, t.bk_y, 3), s>>>(g, t.bk_y, S, tw, cg);       \
    break;
  if (g.py.L) k_inv_y_df<0><<<grid, kThreads, y_smem_rt(g.py, t.bk_y, 3), s>>>(g, t.bk_y, S, tw, cg);
  else FH_SWITCH_LEN(g.ny, IYL)
#undef IYL
  return cudaGetLastError();
}

}  // namespace fh
