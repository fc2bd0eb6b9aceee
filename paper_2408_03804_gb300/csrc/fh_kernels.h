// Host-side launch interface between the driver (api.cu) and the kernels.
#pragma once

#include "fh_common.cuh"

namespace fh {

// What the forward z pass transforms
enum ZMode : int {
  kZDirect = 0,    // tau = src
  kZKApply = 1,    // tau = K : src            (src read only)
  kZCg = 2,        // x += alpha p ; p = r + beta p ; tau = K : p   (src = r; x, p updated in place)
  kZCgFirst = 3,   // p = r ; tau = K : p
};

// What the inverse z pass does with the real result y
enum IZMode : int {
  kIZOut = 0,      // out = y
  kIZDot = 1,      // out = y ; partial sums of p . y
  kIZRhs = 2,      // out = y ; partial sums of y . y
};

// device-resident CG scalars (one block per context)
struct CgScalars {
  double rr;        // r . r
  double bb;        // b . b
  double alpha;
  double beta;
  double tol;       // relative tolerance on ||r|| / ||b||
  double py;        // last p . y
  int it;           // matrix-vector products done
  int max_it;
  int done;         // 0 running, 1 converged, 2 iteration cap, 3 breakdown (p . y <= 0 or non-finite)
  int products;     // matrix-vector products whose result was used (it, plus one after a breakdown)
};

// launches of a CG loop queued after its convergence return at once
__device__ __forceinline__ bool cg_done(const CgScalars* cg) { return cg != nullptr && cg->done != 0; }

// per-cell pointers of a batched launch (device array, one entry per cell of a
// group of equal grids); `stop` is the cell's skip flag for this launch
struct CellView {
  const int* stop;          // skip the cell when *stop != 0 (its CG done flag, or its Newton flag)
  const double* src;        // forward z pass input: P (right-hand side) or r (CG)
  double* p;
  double* x;
  const double* K;
  const CgScalars* cg;
  double2* S;
  double* out;              // inverse z pass output: r (right-hand side) or y (CG)
  double* partials;         // this cell's partial sums
};

// per-cell state of a batched solve (device array, one entry per cell of a
// group of equal grids)
struct CellState {
  double* F;
  double* x;
  double* r;
  double* p;
  double* y;
  double* P;
  double* K;
  double2* S;
  double* partials;
  double* sums;             // 16 doubles: reductions read by the host
  CgScalars* cg;
  const uint8_t* phase;
  const double* scale;
  const int* newton_done;   // skip mask of the launch: batched kernels leave the cell alone when set
  int* flags;
};

struct Tiling {
  int lines_z;     // z lines per CTA in the z passes
  int bk_y;        // kz columns per CTA in the y passes
  int bk_x;        // kz columns per CTA in the x pass
  int lines_z_df;  // z lines per CTA in the double-float z passes (half the shared memory of lines_z)
};

// the tiles of the double-float passes: lines_z_df z lines per CTA
inline Tiling df_tiles(const Tiling& t) {
  Tiling d = t;
  d.lines_z = t.lines_z_df > 0 ? t.lines_z_df : t.lines_z;
  return d;
}

// the twiddle tables of every supported length into t[kTwiddleTables] (host
// memory): w_L^m = exp(-2 pi i m / L) at twiddle_offset(L) + m, its tangent
// form at kTwiddleTotal + twiddle_offset(L) + m
void fill_twiddle_table(double2* t);
// the tangent form (rho, tau) of w_L^m for m < L into t[L] (host memory)
void fill_tangent_twiddles_of_length(double2* t, int L);

// run-time plan of a length without a compile-time plan (L = 0 when it has
// one); its tables (tw_len entries) go to offset tw_off of the context's table
FftPlan make_fft_plan(int L, int tw_off);
// w_L^m for m < L into t[L] (host memory)
void fill_twiddles_of_length(double2* t, int L);
// the tables of a run-time plan into t[p.tw_len] (host memory)
void fill_plan_tables(double2* t, const FftPlan& p);

// tiles of the five passes; smaller tiles where the default ones would leave
// fewer than min_ctas CTAs in a pass (0: the default tiles)
Tiling choose_tiling(const Grid& g, long long min_ctas = 0);
size_t z_pass_smem(const Grid& g, const Tiling& t);
// shared memory of a y or x pass CTA: `fields` x bk pencils of a compile-time
// length L, or of a run-time plan (whose tables may exceed L entries); the
// same for FP64 and double-float entries (16 bytes each)
size_t y_smem(int L, int bk, int fields);
size_t y_smem_rt(const FftPlan& p, int bk, int fields);
long long z_pass_ctas(const Grid& g, const Tiling& t);

cudaError_t setup_fft_kernels(const Grid& g, const Tiling& t);
cudaError_t launch_fwd_z(const Grid& g, const Tiling& t, int mode, const double* src, double* p, double* x,
                         const double* K, const CgScalars* cg, double2* S, const double2* tw, cudaStream_t s);
cudaError_t launch_fwd_y(const Grid& g, const Tiling& t, double2* S, const double2* tw, const CgScalars* cg,
                         cudaStream_t s);
cudaError_t launch_x_ghat(const Grid& g, const Tiling& t, double2* S, const double2* tw, double scale,
                          const CgScalars* cg, cudaStream_t s);
cudaError_t launch_inv_y(const Grid& g, const Tiling& t, double2* S, const double2* tw, const CgScalars* cg,
                         cudaStream_t s);
cudaError_t launch_inv_z(const Grid& g, const Tiling& t, int mode, const double2* S, double* out, const double* p,
                         double* partials, const double2* tw, const CgScalars* cg, cudaStream_t s);

// the y and x passes of a plane cell (nz = 1; kernels_plane.cu), which the
// launches above dispatch to
cudaError_t setup_plane_kernels(const Grid& g);
cudaError_t launch_plane_fwd_y(const Grid& g, double2* S, const double2* tw, const CgScalars* cg, cudaStream_t s);
cudaError_t launch_plane_x_ghat(const Grid& g, double2* S, const double2* tw, double scale, const CgScalars* cg,
                                cudaStream_t s);
cudaError_t launch_plane_inv_y(const Grid& g, double2* S, const double2* tw, const CgScalars* cg, cudaStream_t s);
struct dfc;
// ... with double-float transforms (setup_plane_kernels prepares both)
cudaError_t launch_plane_fwd_y(const Grid& g, dfc* S, const dfc* tw, const CgScalars* cg, cudaStream_t s);
cudaError_t launch_plane_x_ghat(const Grid& g, dfc* S, const dfc* tw, double scale, const CgScalars* cg,
                                cudaStream_t s);
cudaError_t launch_plane_inv_y(const Grid& g, dfc* S, const dfc* tw, const CgScalars* cg, cudaStream_t s);

// the same five passes with double-float transforms (kernels_df64.cu; plane
// cells dispatch to kernels_plane.cu): the spectrum buffer and a double-float
// copy of the twiddle table (same offsets, run-time plan tables included) as dfc
struct df64;
// K_df = the packed tangent [45][N] in double-float
cudaError_t launch_tangent_to_df64(const Grid& g, const double* K, df64* K_df, cudaStream_t s);
// the n entries of an FP64 twiddle table (with any run-time plan tables) in double-float
void twiddles_to_df64(const double2* src, dfc* dst, int n);
cudaError_t setup_df64_kernels(const Grid& g, const Tiling& t);
cudaError_t setup_df64_yx_kernels(const Grid& g, const Tiling& t);     // kernels_df64_yx.cu
cudaError_t setup_df64_batch_kernels(const Grid& g, const Tiling& t);  // kernels_df64_batch.cu
cudaError_t launch_fwd_z_df(const Grid& g, const Tiling& t, int mode, const double* src, double* p, double* x,
                            const df64* K, const CgScalars* cg, dfc* S, const dfc* tw, cudaStream_t s);
cudaError_t launch_fwd_y_df(const Grid& g, const Tiling& t, dfc* S, const dfc* tw, const CgScalars* cg,
                            cudaStream_t s);
cudaError_t launch_x_ghat_df(const Grid& g, const Tiling& t, dfc* S, const dfc* tw, double scale,
                             const CgScalars* cg, cudaStream_t s);
cudaError_t launch_inv_y_df(const Grid& g, const Tiling& t, dfc* S, const dfc* tw, const CgScalars* cg,
                            cudaStream_t s);
cudaError_t launch_inv_z_df(const Grid& g, const Tiling& t, int mode, const dfc* S, double* out, const double* p,
                            double* partials, const dfc* tw, const CgScalars* cg, cudaStream_t s);

// batched double-float CG passes (kZCg / kZCgFirst forward, kIZDot inverse)
// over cells whose spectrum and tangent buffers hold double-float data; the
// tangents are converted in place for the cells not masked by newton_done
cudaError_t launch_tangent_to_df64_batch(const Grid& g, const CellState* cells, int n_cells, cudaStream_t s);
cudaError_t launch_fwd_z_batch_df(const Grid& g, const Tiling& t, int mode, const CellView* cells, int n_cells,
                                  const dfc* tw, cudaStream_t s);
cudaError_t launch_fwd_y_batch_df(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                                  const dfc* tw, cudaStream_t s);
cudaError_t launch_x_ghat_batch_df(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                                   const dfc* tw, double scale, cudaStream_t s);
cudaError_t launch_inv_y_batch_df(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                                  const dfc* tw, cudaStream_t s);
cudaError_t launch_inv_z_batch_df(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                                  const dfc* tw, cudaStream_t s);

cudaError_t launch_fwd_z_batch(const Grid& g, const Tiling& t, int mode, const CellView* cells, int n_cells,
                               const double2* tw, cudaStream_t s);
cudaError_t launch_fwd_y_batch(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                               const double2* tw, cudaStream_t s);
cudaError_t launch_x_ghat_batch(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                                const double2* tw, double scale, cudaStream_t s);
cudaError_t launch_inv_y_batch(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                               const double2* tw, cudaStream_t s);
cudaError_t launch_inv_z_batch(const Grid& g, const Tiling& t, int mode, const CellView* cells, int n_cells,
                               const double2* tw, cudaStream_t s);

// pointwise kernels (kernels_pointwise.cu)
long long constitutive_ctas(const Grid& g);
cudaError_t launch_constitutive(const Grid& g, const MatView& m, const double* F, double* P, double* K,
                                double* partials, int* flags, cudaStream_t s);
cudaError_t launch_jvp(const Grid& g, const MatView& m, const double* F, const double* src, double* p, double* x,
                       double* tau, int mode, const CgScalars* cg, int* flags, cudaStream_t s);
cudaError_t launch_sum_partials(const double* partials, int n_parts, int width, double* out, cudaStream_t s);
cudaError_t launch_field_sums(const Grid& g, const double* F, double* partials, cudaStream_t s);
cudaError_t launch_fill(const Grid& g, double* F, const double* value9, int add, cudaStream_t s);
cudaError_t launch_cg_init(CgScalars* cg, const double* partials, int n_parts, double tol, int max_it,
                           cudaStream_t s);
cudaError_t launch_cg_alpha(CgScalars* cg, const double* partials, int n_parts, cudaStream_t s);
long long cg_update_ctas(const Grid& g);
cudaError_t launch_cg_update(const Grid& g, CgScalars* cg, double* r, const double* y, double* partials,
                             cudaStream_t s);
cudaError_t launch_cg_finalize(const Grid& g, const CgScalars* cg, double* x, const double* p, cudaStream_t s);
cudaError_t launch_cg_beta(CgScalars* cg, const double* partials, int n_parts, cudaStream_t s);
cudaError_t launch_newton_update(const Grid& g, double* F, const double* dF, double* partials, cudaStream_t s);
long long newton_update_ctas(const Grid& g);
cudaError_t launch_constitutive_batch(const Grid& g, int kind, const double* params, const CellState* cells,
                                      int n_cells, int store_K, cudaStream_t s);
cudaError_t launch_cg_init_batch(const CellState* cells, int n_cells, int n_parts, double tol, int max_it,
                                 cudaStream_t s);
cudaError_t launch_cg_alpha_batch(const CellState* cells, int n_cells, int n_parts, cudaStream_t s);
cudaError_t launch_cg_update_batch(const Grid& g, const CellState* cells, int n_cells, cudaStream_t s);
cudaError_t launch_cg_beta_batch(const CellState* cells, int n_cells, int n_parts, cudaStream_t s);
cudaError_t launch_cg_finalize_batch(const Grid& g, const CellState* cells, int n_cells, cudaStream_t s);
cudaError_t launch_newton_update_batch(const Grid& g, const CellState* cells, int n_cells, cudaStream_t s);
cudaError_t launch_sum_partials_batch(const CellState* cells, int n_cells, int n_parts, int width, cudaStream_t s);
cudaError_t launch_fill_batch(const Grid& g, const CellState* cells, int n_cells, int field, const double* value9,
                              int add, cudaStream_t s);
long long kapply_sums_ctas(const Grid& g);
cudaError_t launch_j2_update(const Grid& g, const MatView& m, const double* H, double* history, cudaStream_t s);
cudaError_t launch_kapply_sums(const Grid& g, const double* K, const double* x, int cd, double* partials,
                               cudaStream_t s);
cudaError_t launch_stress_sensitivity(const Grid& g, const MatView& m, const double* F, const double* x, int ab,
                                      const double* dscale, double* out, cudaStream_t s);
cudaError_t launch_sensitivity(const Grid& g, const MatView& m, const double* xa, int ab, const double* xc, int cd,
                               const double* dscale, double* out, cudaStream_t s);

}  // namespace fh
