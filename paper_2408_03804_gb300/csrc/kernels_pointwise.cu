// Voxel-wise kernels of the Newton-Krylov solve (Appendix A, Algorithm 1):
// the constitutive evaluation by automatic differentiation (Eqs. 2-3), the
// homogenized-stress reduction (Eq. 4), the conjugate-gradient scalar and
// vector updates, and the Newton update with its convergence norm.
//
// Every reduction is deterministic: each CTA writes one partial per output
// (a fixed shuffle tree inside the CTA), and a single CTA adds the partials
// in a fixed order, so repeated runs give bit-identical results.
#include <math.h>

#include "ad.cuh"
#include "fh_kernels.h"

namespace fh {

constexpr int kPointwiseCtas = 4 * 152;  // grid of the grid-stride voxel kernels

// P and packed K of one voxel for any law: energy laws by second-order AD of W,
// the J2 return map by first-order AD of the stress, from the voxel's history
template <class Law>
__device__ __forceinline__ double material_derivatives(const MatView& m, long long v, long long n, const double f[9],
                                                       double P[9], double K[45]) {
  double lam, mu;
  voxel_lame(m, v, lam, mu);
  if constexpr (std::is_same<Law, J2Law>::value) {
    J2State st;
#pragma unroll
    for (int c = 0; c < 9; ++c) st.ep[c] = m.history[c * n + v];
    st.p = m.history[9 * n + v];
    st.lam = lam;
    st.mu = mu;
    const int ph = m.phase[v];
    st.sy = m.plastic[2 * ph];
    st.h = m.plastic[2 * ph + 1];
    ad::stress_derivatives<J2Law>(f, st, P, K);
    return 0.0;
  } else {
    return ad::energy_derivatives<Law>(f, lam, mu, P, K);
  }
}

static unsigned pointwise_grid(const Grid& g) {
  long long b = (g.n + kThreads - 1) / kThreads;
  if (b > kPointwiseCtas) b = kPointwiseCtas;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// ---------------------------------------------------------------------------
// constitutive evaluation: P, packed K and per-CTA sums of P
// ---------------------------------------------------------------------------
template <class Law>
__device__ __forceinline__ void constitutive_body(Grid g, MatView m, const double* __restrict__ F,
                                                          double* __restrict__ P, double* __restrict__ K,
                                                          double* __restrict__ partials, int* __restrict__ flags) {
  __shared__ double red[32];
  double sum[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) sum[c] = 0.0;
  bool bad = false;
  const long long n = g.n;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    double f[9], pv[9], kv[45];
#pragma unroll
    for (int c = 0; c < 9; ++c) f[c] = F[c * n + v];
    const double w = material_derivatives<Law>(m, v, n, f, pv, kv);
    bool ok = isfinite(w);
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      ok = ok && isfinite(pv[c]);
      sum[c] += pv[c];
      if (P) P[c * n + v] = pv[c];
    }
    if (K) {
#pragma unroll
      for (int s = 0; s < 45; ++s) {
        ok = ok && isfinite(kv[s]);
        K[s * n + v] = kv[s];
      }
    }
    bad |= !ok;
  }
  if (bad) atomicOr(flags, kFlagNonPhysical);
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    const double s = block_sum(sum[c], red);
    if (threadIdx.x == 0) partials[c * gridDim.x + blockIdx.x] = s;
  }
}

template <class Law>
__global__ void __launch_bounds__(kThreads) k_constitutive(Grid g, MatView m, const double* __restrict__ F,
                                                          double* __restrict__ P, double* __restrict__ K,
                                                          double* __restrict__ partials, int* __restrict__ flags) {
  constitutive_body<Law>(g, m, F, P, K, partials, flags);
}

template <class Law>
__global__ void __launch_bounds__(kThreads) k_constitutive_b(Grid g, int kind, const double* __restrict__ params,
                                                            const CellState* __restrict__ cells, int store_K) {
  const CellState& c = cells[blockIdx.y];
  if (*c.newton_done) return;
  const MatView m{kind, c.phase, params, c.scale, nullptr, nullptr};
  constitutive_body<Law>(g, m, c.F, c.P, store_K ? c.K : nullptr, c.partials, c.flags);
}

long long constitutive_ctas(const Grid& g) { return pointwise_grid(g); }

cudaError_t launch_constitutive_batch(const Grid& g, int kind, const double* params, const CellState* cells,
                                      int n_cells, int store_K, cudaStream_t s) {
  const dim3 grid(pointwise_grid(g), (unsigned)n_cells);
  switch (kind) {
    case FH_LINEAR_ELASTIC:
      k_constitutive_b<LinearElasticLaw><<<grid, kThreads, 0, s>>>(g, kind, params, cells, store_K);
      break;
    case FH_NEO_HOOKEAN:
      k_constitutive_b<NeoHookeanLaw><<<grid, kThreads, 0, s>>>(g, kind, params, cells, store_K);
      break;
    case FH_SVK: k_constitutive_b<SVKLaw><<<grid, kThreads, 0, s>>>(g, kind, params, cells, store_K); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_constitutive(const Grid& g, const MatView& m, const double* F, double* P, double* K,
                                double* partials, int* flags, cudaStream_t s) {
  const unsigned grid = pointwise_grid(g);
  switch (m.kind) {
    case FH_LINEAR_ELASTIC:
      k_constitutive<LinearElasticLaw><<<grid, kThreads, 0, s>>>(g, m, F, P, K, partials, flags);
      break;
    case FH_NEO_HOOKEAN:
      k_constitutive<NeoHookeanLaw><<<grid, kThreads, 0, s>>>(g, m, F, P, K, partials, flags);
      break;
    case FH_SVK:
      k_constitutive<SVKLaw><<<grid, kThreads, 0, s>>>(g, m, F, P, K, partials, flags);
      break;
    case FH_J2:
      k_constitutive<J2Law><<<grid, kThreads, 0, s>>>(g, m, F, P, K, partials, flags);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// jvp form of the tangent apply (Listing 3): tau = K(F) : p with K re-derived
// by AD in every call. mode kZKApply: p = src ; kZCg: x += alpha p, then
// p = r + beta p ; kZCgFirst: p = r (p written back in the CG modes).
// ---------------------------------------------------------------------------
template <class Law, int MODE>
__global__ void __launch_bounds__(kThreads) k_jvp(Grid g, MatView m, const double* __restrict__ F,
                                                 const double* __restrict__ src, double* __restrict__ p,
                                                 double* __restrict__ x, double* __restrict__ tau,
                                                 const CgScalars* __restrict__ cg, int* __restrict__ flags) {
  if (cg != nullptr && cg->done) return;
  const long long n = g.n;
  double beta = 0.0, alpha = 0.0;
  if constexpr (MODE == kZCg) {
    beta = cg->beta;
    alpha = cg->alpha;
  }
  bool bad = false;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    double f[9], pv[9], kv[45], pd[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      f[c] = F[c * n + v];
      if constexpr (MODE == kZKApply) {
        pd[c] = src[c * n + v];
      } else if constexpr (MODE == kZCgFirst) {
        pd[c] = src[c * n + v];
        p[c * n + v] = pd[c];
      } else {
        const double po = p[c * n + v];
        x[c * n + v] = fma(alpha, po, x[c * n + v]);
        pd[c] = fma(beta, po, src[c * n + v]);
        p[c * n + v] = pd[c];
      }
    }
    const double w = material_derivatives<Law>(m, v, n, f, pv, kv);
    bad |= !isfinite(w);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      double acc = kv[sym_slot(a, 0)] * pd[0];
#pragma unroll
      for (int b = 1; b < 9; ++b) acc = fma(kv[sym_slot(a, b)], pd[b], acc);
      tau[a * n + v] = acc;
    }
  }
  if (bad) atomicOr(flags, kFlagNonPhysical);
}

template <class Law>
static void launch_jvp_law(unsigned grid, cudaStream_t s, const Grid& g, const MatView& m, const double* F,
                           const double* src, double* p, double* x, double* tau, int mode, const CgScalars* cg,
                           int* flags) {
  switch (mode) {
    case kZKApply: k_jvp<Law, kZKApply><<<grid, kThreads, 0, s>>>(g, m, F, src, p, x, tau, cg, flags); break;
    case kZCg: k_jvp<Law, kZCg><<<grid, kThreads, 0, s>>>(g, m, F, src, p, x, tau, cg, flags); break;
    default: k_jvp<Law, kZCgFirst><<<grid, kThreads, 0, s>>>(g, m, F, src, p, x, tau, cg, flags); break;
  }
}

cudaError_t launch_jvp(const Grid& g, const MatView& m, const double* F, const double* src, double* p, double* x,
                       double* tau, int mode, const CgScalars* cg, int* flags, cudaStream_t s) {
  const unsigned grid = pointwise_grid(g);
  switch (m.kind) {
    case FH_LINEAR_ELASTIC:
      launch_jvp_law<LinearElasticLaw>(grid, s, g, m, F, src, p, x, tau, mode, cg, flags);
      break;
    case FH_NEO_HOOKEAN: launch_jvp_law<NeoHookeanLaw>(grid, s, g, m, F, src, p, x, tau, mode, cg, flags); break;
    case FH_SVK: launch_jvp_law<SVKLaw>(grid, s, g, m, F, src, p, x, tau, mode, cg, flags); break;
    case FH_J2: launch_jvp_law<J2Law>(grid, s, g, m, F, src, p, x, tau, mode, cg, flags); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// single-CTA fixed-order sums of partials: out[w] = sum_b partials[w n_parts + b]
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sum_fixed(const double* __restrict__ a, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += a[i];
  return block_sum(s, red);
}

__global__ void __launch_bounds__(kThreads) k_sum_partials(const double* __restrict__ partials, int n_parts,
                                                          int width, double* __restrict__ out) {
  __shared__ double red[32];
  for (int w = 0; w < width; ++w) {
    const double s = sum_fixed(partials + (long long)w * n_parts, n_parts, red);
    if (threadIdx.x == 0) out[w] = s;
  }
}

cudaError_t launch_sum_partials(const double* partials, int n_parts, int width, double* out, cudaStream_t s) {
  k_sum_partials<<<1, kThreads, 0, s>>>(partials, n_parts, width, out);
  return cudaGetLastError();
}

// one CTA per cell: the cell's partials to its sums (cells whose mask is set are skipped)
__global__ void __launch_bounds__(kThreads) k_sum_partials_b(const CellState* __restrict__ cells, int n_parts,
                                                            int width) {
  __shared__ double red[32];
  const CellState& c = cells[blockIdx.x];
  if (*c.newton_done) return;
  for (int w = 0; w < width; ++w) {
    const double s = sum_fixed(c.partials + (long long)w * n_parts, n_parts, red);
    if (threadIdx.x == 0) c.sums[w] = s;
  }
}

cudaError_t launch_sum_partials_batch(const CellState* cells, int n_cells, int n_parts, int width, cudaStream_t s) {
  k_sum_partials_b<<<n_cells, kThreads, 0, s>>>(cells, n_parts, width);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// per-CTA sums of the nine components of a field (voxel mean of a start field)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_field_sums(Grid g, const double* __restrict__ F,
                                                        double* __restrict__ partials) {
  __shared__ double red[32];
  const long long n = g.n;
  for (int c = 0; c < 9; ++c) {
    double acc = 0.0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
      acc += F[c * n + v];
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[c * gridDim.x + blockIdx.x] = s;
  }
}

cudaError_t launch_field_sums(const Grid& g, const double* F, double* partials, cudaStream_t s) {
  k_field_sums<<<pointwise_grid(g), kThreads, 0, s>>>(g, F, partials);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// F = value (add = 0) or F += value (add = 1) in every voxel (load increment)
// ---------------------------------------------------------------------------
struct Nine {
  double v[9];
};

__global__ void __launch_bounds__(kThreads) k_fill(Grid g, double* __restrict__ F, Nine val, int add) {
  const long long n = g.n;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 9; ++c) F[c * n + v] = add ? F[c * n + v] + val.v[c] : val.v[c];
  }
}

// per cell: F (field 0), the CG solution x (field 1) or the CG direction p
// (field 2) set to / incremented by val (cells whose mask is set are skipped)
__global__ void __launch_bounds__(kThreads) k_fill_b(Grid g, const CellState* __restrict__ cells, int field, Nine val,
                                                    int add) {
  const CellState& c = cells[blockIdx.y];
  if (*c.newton_done) return;
  double* F = field == 0 ? c.F : (field == 1 ? c.x : c.p);
  const long long n = g.n;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k * n + v] = add ? F[k * n + v] + val.v[k] : val.v[k];
  }
}

cudaError_t launch_fill_batch(const Grid& g, const CellState* cells, int n_cells, int field, const double* value9,
                              int add, cudaStream_t s) {
  Nine val;
  for (int c = 0; c < 9; ++c) val.v[c] = value9[c];
  k_fill_b<<<dim3(pointwise_grid(g), n_cells), kThreads, 0, s>>>(g, cells, field, val, add);
  return cudaGetLastError();
}

cudaError_t launch_fill(const Grid& g, double* F, const double* value9, int add, cudaStream_t s) {
  Nine val;
  for (int c = 0; c < 9; ++c) val.v[c] = value9[c];
  k_fill<<<pointwise_grid(g), kThreads, 0, s>>>(g, F, val, add);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// conjugate-gradient scalars (single CTA each)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cg_init_body(CgScalars* cg, const double* __restrict__ partials, int n_parts,
                                                     double tol, int max_it) {
  __shared__ double red[32];
  const double bb = sum_fixed(partials, n_parts, red);
  if (threadIdx.x == 0) {
    cg->bb = bb;
    cg->rr = bb;
    cg->alpha = 0.0;
    cg->beta = 0.0;
    cg->tol = tol;
    cg->py = 0.0;
    cg->it = 0;
    cg->products = 0;
    cg->max_it = max_it;
    // the test of the loop head with r = b (converged at once only if b = 0 or tol >= 1)
    int done = 0;
    if (!(bb == bb)) done = 3;
    else if (sqrt(bb) <= tol * sqrt(bb)) done = 1;
    else if (max_it <= 0) done = 2;
    cg->done = done;
  }
}

__global__ void __launch_bounds__(kThreads) k_cg_init(CgScalars* cg, const double* __restrict__ partials,
                                                     int n_parts, double tol, int max_it) {
  cg_init_body(cg, partials, n_parts, tol, max_it);
}

// one CTA per cell; cells whose mask is set keep their CG state
__global__ void __launch_bounds__(kThreads) k_cg_init_b(const CellState* __restrict__ cells, int n_parts, double tol,
                                                       int max_it) {
  const CellState& c = cells[blockIdx.x];
  if (*c.newton_done) return;
  cg_init_body(c.cg, c.partials, n_parts, tol, max_it);
}

cudaError_t launch_cg_init(CgScalars* cg, const double* partials, int n_parts, double tol, int max_it,
                           cudaStream_t s) {
  k_cg_init<<<1, kThreads, 0, s>>>(cg, partials, n_parts, tol, max_it);
  return cudaGetLastError();
}

cudaError_t launch_cg_init_batch(const CellState* cells, int n_cells, int n_parts, double tol, int max_it,
                                 cudaStream_t s) {
  k_cg_init_b<<<n_cells, kThreads, 0, s>>>(cells, n_parts, tol, max_it);
  return cudaGetLastError();
}

__device__ __forceinline__ void cg_alpha_body(CgScalars* cg, const double* __restrict__ partials,
                                                      int n_parts) {
  __shared__ double red[32];
  if (cg->done) return;
  const double py = sum_fixed(partials, n_parts, red);
  if (threadIdx.x == 0) {
    cg->products += 1;
    cg->py = py;
    if (!(py > 0.0) || !isfinite(py)) {
      cg->done = 3;
      cg->alpha = 0.0;
    } else {
      cg->alpha = cg->rr / py;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_cg_alpha(CgScalars* cg, const double* __restrict__ partials,
                                                      int n_parts) {
  cg_alpha_body(cg, partials, n_parts);
}
__global__ void __launch_bounds__(kThreads) k_cg_alpha_b(const CellState* __restrict__ cells, int n_parts) {
  const CellState& c = cells[blockIdx.x];
  cg_alpha_body(c.cg, c.partials, n_parts);
}

cudaError_t launch_cg_alpha(CgScalars* cg, const double* partials, int n_parts, cudaStream_t s) {
  k_cg_alpha<<<1, kThreads, 0, s>>>(cg, partials, n_parts);
  return cudaGetLastError();
}
cudaError_t launch_cg_alpha_batch(const CellState* cells, int n_cells, int n_parts, cudaStream_t s) {
  k_cg_alpha_b<<<n_cells, kThreads, 0, s>>>(cells, n_parts);
  return cudaGetLastError();
}

// r -= alpha y and partial r . r. The matching x += alpha p is deferred to the
// next forward z pass (which reads p anyway) or to k_cg_finalize.
__device__ __forceinline__ void cg_update_body(Grid g, const CgScalars* __restrict__ cg,
                                                       double* __restrict__ r, const double* __restrict__ y,
                                                       double* __restrict__ partials) {
  __shared__ double red[32];
  if (cg->done) return;
  const double alpha = cg->alpha;
  const long long n9 = 9 * g.n;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n9; i += (long long)gridDim.x * blockDim.x) {
    const double rv = fma(-alpha, y[i], r[i]);
    r[i] = rv;
    acc = fma(rv, rv, acc);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_cg_update(Grid g, const CgScalars* __restrict__ cg,
                                                       double* __restrict__ r, const double* __restrict__ y,
                                                       double* __restrict__ partials) {
  cg_update_body(g, cg, r, y, partials);
}
__global__ void __launch_bounds__(kThreads) k_cg_update_b(Grid g, const CellState* __restrict__ cells) {
  const CellState& c = cells[blockIdx.y];
  cg_update_body(g, c.cg, c.r, c.y, c.partials);
}

long long cg_update_ctas(const Grid& g) { return pointwise_grid(g); }

cudaError_t launch_cg_update(const Grid& g, CgScalars* cg, double* r, const double* y, double* partials,
                             cudaStream_t s) {
  k_cg_update<<<pointwise_grid(g), kThreads, 0, s>>>(g, cg, r, y, partials);
  return cudaGetLastError();
}
cudaError_t launch_cg_update_batch(const Grid& g, const CellState* cells, int n_cells, cudaStream_t s) {
  k_cg_update_b<<<dim3(pointwise_grid(g), n_cells), kThreads, 0, s>>>(g, cells);
  return cudaGetLastError();
}

// the last deferred x += alpha p once CG has stopped (nothing if no product ran;
// alpha is 0 after a breakdown in k_cg_alpha)
__device__ __forceinline__ void cg_finalize_body(Grid g, const CgScalars* __restrict__ cg,
                                                         double* __restrict__ x, const double* __restrict__ p) {
  if (cg->it == 0) return;
  const double alpha = cg->alpha;
  const long long n9 = 9 * g.n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n9; i += (long long)gridDim.x * blockDim.x)
    x[i] = fma(alpha, p[i], x[i]);
}

__global__ void __launch_bounds__(kThreads) k_cg_finalize(Grid g, const CgScalars* __restrict__ cg,
                                                         double* __restrict__ x, const double* __restrict__ p) {
  cg_finalize_body(g, cg, x, p);
}
__global__ void __launch_bounds__(kThreads) k_cg_finalize_b(Grid g, const CellState* __restrict__ cells) {
  const CellState& c = cells[blockIdx.y];
  if (*c.newton_done) return;
  cg_finalize_body(g, c.cg, c.x, c.p);
}

cudaError_t launch_cg_finalize(const Grid& g, const CgScalars* cg, double* x, const double* p, cudaStream_t s) {
  k_cg_finalize<<<pointwise_grid(g), kThreads, 0, s>>>(g, cg, x, p);
  return cudaGetLastError();
}
cudaError_t launch_cg_finalize_batch(const Grid& g, const CellState* cells, int n_cells, cudaStream_t s) {
  k_cg_finalize_b<<<dim3(pointwise_grid(g), n_cells), kThreads, 0, s>>>(g, cells);
  return cudaGetLastError();
}

__device__ __forceinline__ void cg_beta_body(CgScalars* cg, const double* __restrict__ partials,
                                                     int n_parts) {
  __shared__ double red[32];
  if (cg->done) return;
  const double rr = sum_fixed(partials, n_parts, red);
  if (threadIdx.x == 0) {
    const double rr_old = cg->rr;
    cg->beta = rr / rr_old;
    cg->rr = rr;
    cg->it += 1;
    if (!isfinite(rr)) cg->done = 3;
    else if (sqrt(rr) <= cg->tol * sqrt(cg->bb)) cg->done = 1;
    else if (cg->it >= cg->max_it) cg->done = 2;
  }
}

__global__ void __launch_bounds__(kThreads) k_cg_beta(CgScalars* cg, const double* __restrict__ partials,
                                                     int n_parts) {
  cg_beta_body(cg, partials, n_parts);
}
__global__ void __launch_bounds__(kThreads) k_cg_beta_b(const CellState* __restrict__ cells, int n_parts) {
  const CellState& c = cells[blockIdx.x];
  cg_beta_body(c.cg, c.partials, n_parts);
}

cudaError_t launch_cg_beta(CgScalars* cg, const double* partials, int n_parts, cudaStream_t s) {
  k_cg_beta<<<1, kThreads, 0, s>>>(cg, partials, n_parts);
  return cudaGetLastError();
}
cudaError_t launch_cg_beta_batch(const CellState* cells, int n_cells, int n_parts, cudaStream_t s) {
  k_cg_beta_b<<<n_cells, kThreads, 0, s>>>(cells, n_parts);
  return cudaGetLastError();
}

// F += dF and partial ||dF||^2 (Algorithm 1 update and convergence test)
__device__ __forceinline__ void newton_update_body(Grid g, double* __restrict__ F,
                                                           const double* __restrict__ dF,
                                                           double* __restrict__ partials) {
  __shared__ double red[32];
  const long long n9 = 9 * g.n;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n9; i += (long long)gridDim.x * blockDim.x) {
    const double d = dF[i];
    F[i] += d;
    acc = fma(d, d, acc);
  }
  const double s = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_newton_update(Grid g, double* __restrict__ F,
                                                           const double* __restrict__ dF,
                                                           double* __restrict__ partials) {
  newton_update_body(g, F, dF, partials);
}
__global__ void __launch_bounds__(kThreads) k_newton_update_b(Grid g, const CellState* __restrict__ cells) {
  const CellState& c = cells[blockIdx.y];
  if (*c.newton_done) return;
  newton_update_body(g, c.F, c.x, c.partials);
}
cudaError_t launch_newton_update_batch(const Grid& g, const CellState* cells, int n_cells, cudaStream_t s) {
  k_newton_update_b<<<dim3(pointwise_grid(g), n_cells), kThreads, 0, s>>>(g, cells);
  return cudaGetLastError();
}

long long newton_update_ctas(const Grid& g) { return pointwise_grid(g); }

cudaError_t launch_newton_update(const Grid& g, double* F, const double* dF, double* partials, cudaStream_t s) {
  k_newton_update<<<pointwise_grid(g), kThreads, 0, s>>>(g, F, dF, partials);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// homogenized tangent column: per-CTA sums of K : (E_cd + x) (Eq. 4)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_kapply_sums(Grid g, const double* __restrict__ K,
                                                         const double* __restrict__ x, int cd,
                                                         double* __restrict__ partials) {
  __shared__ double red[32];
  double sum[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) sum[a] = 0.0;
  const long long n = g.n;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    double h[9];
#pragma unroll
    for (int b = 0; b < 9; ++b) h[b] = x[b * n + v] + (b == cd ? 1.0 : 0.0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      double acc = 0.0;
#pragma unroll
      for (int b = 0; b < 9; ++b) acc = fma(K[sym_slot(a, b) * n + v], h[b], acc);
      sum[a] += acc;
    }
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const double s = block_sum(sum[a], red);
    if (threadIdx.x == 0) partials[a * gridDim.x + blockIdx.x] = s;
  }
}

long long kapply_sums_ctas(const Grid& g) { return pointwise_grid(g); }

cudaError_t launch_kapply_sums(const Grid& g, const double* K, const double* x, int cd, double* partials,
                               cudaStream_t s) {
  k_kapply_sums<<<pointwise_grid(g), kThreads, 0, s>>>(g, K, x, cd, partials);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// voxel sensitivity of a homogenized linear modulus (self-adjoint form):
// out_v = (E_ab + xa)_v : C0_v : (E_cd + xc)_v * dscale_v / N, with C0 the
// tangent of the unscaled phase parameters, from the same AD as the solve
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_sensitivity(Grid g, MatView m, const double* __restrict__ xa, int ab,
                                                         const double* __restrict__ xc, int cd,
                                                         const double* __restrict__ dscale,
                                                         double* __restrict__ out) {
  const long long n = g.n;
  const double inv_n = 1.0 / (double)n;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    double zero[9], pv[9], kv[45], ha[9], hc[9];
#pragma unroll
    for (int b = 0; b < 9; ++b) {
      zero[b] = 0.0;
      ha[b] = xa[b * n + v] + (b == ab ? 1.0 : 0.0);
      hc[b] = xc[b * n + v] + (b == cd ? 1.0 : 0.0);
    }
    const int ph = m.phase[v];
    ad::energy_derivatives<LinearElasticLaw>(zero, m.params[2 * ph], m.params[2 * ph + 1], pv, kv);
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      double t = 0.0;
#pragma unroll
      for (int b = 0; b < 9; ++b) t = fma(kv[sym_slot(a, b)], hc[b], t);
      acc = fma(ha[a], t, acc);
    }
    out[v] = acc * dscale[v] * inv_n;
  }
}

cudaError_t launch_sensitivity(const Grid& g, const MatView& m, const double* xa, int ab, const double* xc, int cd,
                               const double* dscale, double* out, cudaStream_t s) {
  k_sensitivity<<<pointwise_grid(g), kThreads, 0, s>>>(g, m, xa, ab, xc, cd, dscale, out);
  return cudaGetLastError();
}

// Stress sensitivity dPbar_ab/drho_v = (1/N) (E_ab + d_ab)_v : P0(F_v) ds/drho_v:
// P0 by AD of the law with the unscaled moduli of the voxel's phase (m.scale
// is ignored), d_ab the unit response in x
template <class Law>
__global__ void __launch_bounds__(kThreads) k_stress_sensitivity(Grid g, MatView m, const double* __restrict__ F,
                                                                const double* __restrict__ x, int ab,
                                                                const double* __restrict__ dscale,
                                                                double* __restrict__ out) {
  const long long n = g.n;
  const double inv_n = 1.0 / (double)n;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    double f[9], pv[9], kv[45];
#pragma unroll
    for (int c = 0; c < 9; ++c) f[c] = F[c * n + v];
    const int ph = m.phase[v];
    ad::energy_derivatives<Law>(f, m.params[2 * ph], m.params[2 * ph + 1], pv, kv);
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < 9; ++c) acc = fma(x[c * n + v] + (c == ab ? 1.0 : 0.0), pv[c], acc);
    out[v] = acc * dscale[v] * inv_n;
  }
}

cudaError_t launch_stress_sensitivity(const Grid& g, const MatView& m, const double* F, const double* x, int ab,
                                      const double* dscale, double* out, cudaStream_t s) {
  const unsigned grid = pointwise_grid(g);
  switch (m.kind) {
    case FH_LINEAR_ELASTIC:
      k_stress_sensitivity<LinearElasticLaw><<<grid, kThreads, 0, s>>>(g, m, F, x, ab, dscale, out);
      break;
    case FH_NEO_HOOKEAN:
      k_stress_sensitivity<NeoHookeanLaw><<<grid, kThreads, 0, s>>>(g, m, F, x, ab, dscale, out);
      break;
    case FH_SVK: k_stress_sensitivity<SVKLaw><<<grid, kThreads, 0, s>>>(g, m, F, x, ab, dscale, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// J2 history after a converged increment: plastic strain and cumulative
// plastic strain of the return map at the converged total strain
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_j2_update(Grid g, MatView m, const double* __restrict__ H,
                                                       double* __restrict__ history) {
  const long long n = g.n;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    double lam, mu;
    voxel_lame(m, v, lam, mu);
    const int ph = m.phase[v];
    const double sy = m.plastic[2 * ph], h = m.plastic[2 * ph + 1];
    double e[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) e[c] = H[c * n + v];
    const double p = history[9 * n + v];
    // symmetric elastic trial strain, stored as a full 3x3
    double ee[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) ee[3 * i + j] = 0.5 * (e[3 * i + j] + e[3 * j + i]) - history[(3 * i + j) * n + v];
    const double tr = ee[0] + ee[4] + ee[8];
    double d[9], ss = 0.0;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      d[c] = 2.0 * mu * (ee[c] - ((c % 4 == 0) ? tr / 3.0 : 0.0));
      ss = fma(d[c], d[c], ss);
    }
    const double q = ::sqrt(1.5 * ss);
    const double phi = q - (sy + h * p);
    if (phi > 0.0) {
      const double dp = phi / (3.0 * mu + h);
      const double f = 1.5 * dp / q;
#pragma unroll
      for (int c = 0; c < 9; ++c) history[c * n + v] += f * d[c];
      history[9 * n + v] = p + dp;
    }
  }
}

cudaError_t launch_j2_update(const Grid& g, const MatView& m, const double* H, double* history, cudaStream_t s) {
  k_j2_update<<<pointwise_grid(g), kThreads, 0, s>>>(g, m, H, history);
  return cudaGetLastError();
}

}  // namespace fh
