// The five passes of the projection G with the transforms in double-float
// arithmetic (df64.cuh): the kernels of the CG matrix-vector product when a
// solve asks for FH_ARITH_DF64. The pass bodies are those of passes.cuh with
// the element type dfc; K : p, the CG updates and the p . y dot product stay
// FP64. Grids whose x and y extents have compile-time plans and whose nz is
// even only.
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
template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_fwd_y_df(Grid g, int BK, dfc* __restrict__ S,
                                                         const dfc* __restrict__ tw, const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  fwd_y_body<L>(blockIdx.x, g, BK, S, tw, cg);
}
template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_x_ghat_df(Grid g, int BK, dfc* __restrict__ S,
                                                          const dfc* __restrict__ tw, double scale,
                                                          const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  x_ghat_body<L>(blockIdx.x, g, BK, S, tw, scale, cg);
}
template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_inv_y_df(Grid g, int BK, dfc* __restrict__ S,
                                                         const dfc* __restrict__ tw, const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  inv_y_body<L>(blockIdx.x, g, BK, S, tw, cg);
}
template <int M, int MODE>
__global__ void __launch_bounds__(kThreads) k_inv_z_df(Grid g, int LB, const dfc* __restrict__ S,
                                                      double* __restrict__ out, const double* __restrict__ p,
                                                      double* __restrict__ partials, const dfc* __restrict__ tw,
                                                      const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  inv_z_body<M, MODE>(blockIdx.x, g, LB, S, out, p, partials, tw, cg);
}

// ... and a group of cells of one grid shape (blockIdx.y = cell; the cell's
// spectrum and tangent buffers hold double-float data in this form)
template <int M, int MODE>
__global__ void __launch_bounds__(kThreads) k_fwd_z_b_df(Grid g, int LB, const CellView* __restrict__ cells,
                                                        const dfc* __restrict__ tw) {
  const CellView& c = cells[blockIdx.y];
  if (*c.stop) return;
  fwd_z_body<M, MODE>(blockIdx.x, g, LB, c.src, c.p, c.x, reinterpret_cast<const df64*>(c.K), c.cg,
                      reinterpret_cast<dfc*>(c.S), tw);
}
template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_fwd_y_b_df(Grid g, int BK, const CellView* __restrict__ cells,
                                                           const dfc* __restrict__ tw) {
  const CellView& c = cells[blockIdx.y];
  if (*c.stop) return;
  fwd_y_body<L>(blockIdx.x, g, BK, reinterpret_cast<dfc*>(c.S), tw, c.cg);
}
template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_x_ghat_b_df(Grid g, int BK, const CellView* __restrict__ cells,
                                                            const dfc* __restrict__ tw, double scale) {
  const CellView& c = cells[blockIdx.y];
  if (*c.stop) return;
  x_ghat_body<L>(blockIdx.x, g, BK, reinterpret_cast<dfc*>(c.S), tw, scale, c.cg);
}
template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_inv_y_b_df(Grid g, int BK, const CellView* __restrict__ cells,
                                                           const dfc* __restrict__ tw) {
  const CellView& c = cells[blockIdx.y];
  if (*c.stop) return;
  inv_y_body<L>(blockIdx.x, g, BK, reinterpret_cast<dfc*>(c.S), tw, c.cg);
}
template <int M, int MODE>
__global__ void __launch_bounds__(kThreads) k_inv_z_b_df(Grid g, int LB, const CellView* __restrict__ cells,
                                                        const dfc* __restrict__ tw) {
  const CellView& c = cells[blockIdx.y];
  if (*c.stop) return;
  inv_z_body<M, MODE>(blockIdx.x, g, LB, reinterpret_cast<const dfc*>(c.S), c.out, c.p, c.partials, tw, c.cg);
}

// each cell's packed tangent converted to double-float in place (same 8
// bytes per entry), for the cells whose tangent was just evaluated
__global__ void __launch_bounds__(kThreads) k_tangent_to_df64_b(const CellState* __restrict__ cells,
                                                               long long count) {
  const CellState& c = cells[blockIdx.y];
  if (*c.newton_done) return;
  df64* out = reinterpret_cast<df64*>(c.K);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = c.K[i];
    out[i] = split_double(v);
  }
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

size_t y_smem_df(int L, int bk, int fields) { return ((size_t)2 * fields * bk * (L + 1) + L) * sizeof(dfc); }

template <class Kern>
cudaError_t allow(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

bool df64_grid_ok(const Grid& g) { return g.px.L == 0 && g.py.L == 0 && g.nz >= 2; }

void fill_twiddle_table_df(dfc* t) {
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int i = 0; i < kTwiddleTotal; ++i) t[i] = dfc{df64{0.f, 0.f}, df64{0.f, 0.f}};
  auto split = [](long double v) {
    const float hi = (float)v;
    return df64{hi, (float)(v - (long double)hi)};
  };
  for (int L = 1; L <= kMaxN; ++L) {
    if (!fft_length_ok(L)) continue;
    for (int m = 0; m < L; ++m) {
      const long double a = two_pi * (long double)m / (long double)L;
      t[twiddle_offset(L) + m] = dfc{split(cosl(a)), split(-sinl(a))};
    }
  }
}

cudaError_t setup_df64_kernels(const Grid& g, const Tiling& t) {
  if (!df64_grid_ok(g)) return cudaSuccess;
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
    if ((e = allow(k_fwd_z_b_df<V, kZCg>, zs))) return e;              \
    if ((e = allow(k_fwd_z_b_df<V, kZCgFirst>, zs))) return e;         \
    if ((e = allow(k_inv_z_b_df<V, kIZDot>, zs))) return e;            \
    break;
  FH_SWITCH_HALF_EVEN(M, ZCASE)
#undef ZCASE
#define YCASE(V)                                                          \
  case V:                                                                 \
    if ((e = allow(k_fwd_y_df<V>, y_smem_df(V, t.bk_y, 3)))) return e;    \
    if ((e = allow(k_inv_y_df<V>, y_smem_df(V, t.bk_y, 3)))) return e;    \
    if ((e = allow(k_fwd_y_b_df<V>, y_smem_df(V, t.bk_y, 3)))) return e;  \
    if ((e = allow(k_inv_y_b_df<V>, y_smem_df(V, t.bk_y, 3)))) return e;  \
    break;
  FH_SWITCH_LEN(g.ny, YCASE)
#undef YCASE
#define XCASE(V)                                                          \
  case V:                                                                 \
    if ((e = allow(k_x_ghat_df<V>, y_smem_df(V, t.bk_x, 6)))) return e;   \
    if ((e = allow(k_x_ghat_b_df<V>, y_smem_df(V, t.bk_x, 6)))) return e; \
    break;
  FH_SWITCH_LEN(g.nx, XCASE)
#undef XCASE
  return cudaSuccess;
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
  FH_SWITCH_HALF_EVEN(M, ZL)
#undef ZL
  return cudaGetLastError();
}

cudaError_t launch_fwd_y_df(const Grid& g, const Tiling& t, dfc* S, const dfc* tw, const CgScalars* cg,
                            cudaStream_t s) {
  const int NC = (g.nzh + t.bk_y - 1) / t.bk_y;
  const unsigned grid = (unsigned)((long long)g.nx * 3 * NC);
#define YL(V)                                                                                  \
  case V:                                                                                      \
    k_fwd_y_df<V><<<grid, kThreads, y_smem_df(V, t.bk_y, 3), s>>>(g, t.bk_y, S, tw, cg);       \
    break;
  FH_SWITCH_LEN(g.ny, YL)
#undef YL
  return cudaGetLastError();
}

cudaError_t launch_x_ghat_df(const Grid& g, const Tiling& t, dfc* S, const dfc* tw, double scale,
                             const CgScalars* cg, cudaStream_t s) {
  const int NC = (g.nzh + t.bk_x - 1) / t.bk_x;
  const unsigned grid = (unsigned)((long long)g.ny * NC);
#define XL(V)                                                                                         \
  case V:                                                                                             \
    k_x_ghat_df<V><<<grid, kThreads, y_smem_df(V, t.bk_x, 6), s>>>(g, t.bk_x, S, tw, scale, cg);      \
    break;
  FH_SWITCH_LEN(g.nx, XL)
#undef XL
  return cudaGetLastError();
}

cudaError_t launch_inv_y_df(const Grid& g, const Tiling& t, dfc* S, const dfc* tw, const CgScalars* cg,
                            cudaStream_t s) {
  const int NC = (g.nzh + t.bk_y - 1) / t.bk_y;
  const unsigned grid = (unsigned)((long long)g.nx * 3 * NC);
#define IYL(V)                                                                                 \
  case V:                                                                                      \
    k_inv_y_df<V><<<grid, kThreads, y_smem_df(V, t.bk_y, 3), s>>>(g, t.bk_y, S, tw, cg);       \
    break;
  FH_SWITCH_LEN(g.ny, IYL)
#undef IYL
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
  FH_SWITCH_HALF_EVEN(M, IZL)
#undef IZL
  return cudaGetLastError();
}

// ---- batched cells --------------------------------------------------------
cudaError_t launch_tangent_to_df64_batch(const Grid& g, const CellState* cells, int n_cells, cudaStream_t s) {
  const long long count = 45LL * g.n;
  long long blocks = (count + kThreads - 1) / kThreads;
  if (blocks > 1024) blocks = 1024;
  k_tangent_to_df64_b<<<dim3((unsigned)blocks, (unsigned)n_cells), kThreads, 0, s>>>(cells, count);
  return cudaGetLastError();
}

cudaError_t launch_fwd_z_batch_df(const Grid& g, const Tiling& t, int mode, const CellView* cells, int n_cells,
                                  const dfc* tw, cudaStream_t s) {
  const size_t smem = z_pass_smem(g, t);
  const dim3 grid((unsigned)z_pass_ctas(g, t), (unsigned)n_cells);
  const int M = g.nz / 2;
#define ZB(V)                                                                                             \
  case V:                                                                                                 \
    switch (mode) {                                                                                       \
      case kZCg: k_fwd_z_b_df<V, kZCg><<<grid, kThreads, smem, s>>>(g, t.lines_z, cells, tw); break;         \
      case kZCgFirst: k_fwd_z_b_df<V, kZCgFirst><<<grid, kThreads, smem, s>>>(g, t.lines_z, cells, tw); break; \
      default: return cudaErrorInvalidValue;                                                              \
    }                                                                                                     \
    break;
  FH_SWITCH_HALF_EVEN(M, ZB)
#undef ZB
  return cudaGetLastError();
}

cudaError_t launch_fwd_y_batch_df(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                                  const dfc* tw, cudaStream_t s) {
  const int NC = (g.nzh + t.bk_y - 1) / t.bk_y;
  const dim3 grid((unsigned)((long long)g.nx * 3 * NC), (unsigned)n_cells);
#define YB(V)                                                                              \
  case V:                                                                                  \
    k_fwd_y_b_df<V><<<grid, kThreads, y_smem_df(V, t.bk_y, 3), s>>>(g, t.bk_y, cells, tw); \
    break;
  FH_SWITCH_LEN(g.ny, YB)
#undef YB
  return cudaGetLastError();
}

cudaError_t launch_x_ghat_batch_df(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                                   const dfc* tw, double scale, cudaStream_t s) {
  const int NC = (g.nzh + t.bk_x - 1) / t.bk_x;
  const dim3 grid((unsigned)((long long)g.ny * NC), (unsigned)n_cells);
#define XB(V)                                                                                       \
  case V:                                                                                           \
    k_x_ghat_b_df<V><<<grid, kThreads, y_smem_df(V, t.bk_x, 6), s>>>(g, t.bk_x, cells, tw, scale);  \
    break;
  FH_SWITCH_LEN(g.nx, XB)
#undef XB
  return cudaGetLastError();
}

cudaError_t launch_inv_y_batch_df(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                                  const dfc* tw, cudaStream_t s) {
  const int NC = (g.nzh + t.bk_y - 1) / t.bk_y;
  const dim3 grid((unsigned)((long long)g.nx * 3 * NC), (unsigned)n_cells);
#define IYB(V)                                                                             \
  case V:                                                                                  \
    k_inv_y_b_df<V><<<grid, kThreads, y_smem_df(V, t.bk_y, 3), s>>>(g, t.bk_y, cells, tw); \
    break;
  FH_SWITCH_LEN(g.ny, IYB)
#undef IYB
  return cudaGetLastError();
}

cudaError_t launch_inv_z_batch_df(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                                  const dfc* tw, cudaStream_t s) {
  const size_t smem = z_pass_smem(g, t);
  const dim3 grid((unsigned)z_pass_ctas(g, t), (unsigned)n_cells);
  const int M = g.nz / 2;
#define IZB(V)                                                                               \
  case V:                                                                                    \
    k_inv_z_b_df<V, kIZDot><<<grid, kThreads, smem, s>>>(g, t.lines_z, cells, tw);           \
    break;
  FH_SWITCH_HALF_EVEN(M, IZB)
#undef IZB
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
