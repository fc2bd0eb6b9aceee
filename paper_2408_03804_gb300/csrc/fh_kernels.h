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
  int pad;
};

struct Tiling {
  int lines_z;   // z lines per CTA in the z passes
  int bk_y;      // kz columns per CTA in the y passes
  int bk_x;      // kz columns per CTA in the x pass
};

Tiling choose_tiling(const Grid& g);
size_t z_pass_smem(const Grid& g, const Tiling& t);
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
long long kapply_sums_ctas(const Grid& g);
cudaError_t launch_kapply_sums(const Grid& g, const double* K, const double* x, int cd, double* partials,
                               cudaStream_t s);
cudaError_t launch_sensitivity(const Grid& g, const MatView& m, const double* xa, int ab, const double* xc, int cd,
                               const double* dscale, double* out, cudaStream_t s);

}  // namespace fh
