// The double-float CG passes of batched solves (FH_ARITH_DF64 in
// fft_homog_solve_batched): the pass bodies of passes.cuh with the element
// type dfc over a group of cells of one grid shape (blockIdx.y = cell), each
// cell's spectrum and tangent buffers holding double-float data during CG.
// Batched grids have compile-time plans and an even nz.
#include "fft_df64.cuh"
#include "passes.cuh"

namespace fh {

namespace {

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

template <class Kern>
cudaError_t allow(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

cudaError_t setup_df64_batch_kernels(const Grid& g, const Tiling& t) {
  if (g.nz < 2 || g.px.L || g.py.L) return cudaSuccess;  // grids a batch cannot hold
  cudaError_t e = cudaSuccess;
  const Tiling td = df_tiles(t);
  const size_t zs = z_pass_smem(g, td);
  const int M = g.nz / 2;
#define ZCASE(V)                                                       \
  case V:                                                              \
    if ((e = allow(k_fwd_z_b_df<V, kZCg>, zs))) return e;              \
    if ((e = allow(k_fwd_z_b_df<V, kZCgFirst>, zs))) return e;         \
    if ((e = allow(k_inv_z_b_df<V, kIZDot>, zs))) return e;            \
    break;
  FH_SWITCH_HALF_EVEN(M, ZCASE)
#undef ZCASE
#define YCASE(V)                                                          \
  case V:                                                                 \
    if ((e = allow(k_fwd_y_b_df<V>, y_smem(V, t.bk_y, 3)))) return e;     \
    if ((e = allow(k_inv_y_b_df<V>, y_smem(V, t.bk_y, 3)))) return e;     \
    break;
  FH_SWITCH_LEN(g.ny, YCASE)
#undef YCASE
#define XCASE(V)                                                          \
  case V:                                                                 \
    if ((e = allow(k_x_ghat_b_df<V>, y_smem(V, t.bk_x, 6)))) return e;    \
    break;
  FH_SWITCH_LEN(g.nx, XCASE)
#undef XCASE
  return cudaSuccess;
}

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
    k_fwd_y_b_df<V><<<grid, kThreads, y_smem(V, t.bk_y, 3), s>>>(g, t.bk_y, cells, tw); \
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
    k_x_ghat_b_df<V><<<grid, kThreads, y_smem(V, t.bk_x, 6), s>>>(g, t.bk_x, cells, tw, scale);  \
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
    k_inv_y_b_df<V><<<grid, kThreads, y_smem(V, t.bk_y, 3), s>>>(g, t.bk_y, cells, tw); \
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
