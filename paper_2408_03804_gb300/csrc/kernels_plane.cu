// The y and x passes of the projection G (Eq. 1) on a plane cell, one voxel
// thick along z (nz = 1).
//
// Every field of such a cell is z-invariant, so xi_z = 0 on every frequency.
// The forward z pass is the identity and hands over the real field tau. The
// j = z column of Ghat's input is tau_iz xi_z = 0 and the j = z column of
// G(tau) is v_i xi_z = 0, so only the columns j = x, y of each row are
// transformed here, and the j = z column of the result is written as zero.
//
// Along y the transforms are real-to-complex. The columns of two x positions
// a and b are transformed together as z = a + i b; then
// 2 A_k = Z_k + conj Z_{-k} and 2 B_k = -i (Z_k - conj Z_{-k}) are the
// spectra of a and b, of which the half k = 0 .. ny/2 is kept (the rest is
// its conjugate). The x pass runs on that half only. The inverse y pass
// rebuilds the full spectra of two columns by conjugate symmetry (dropping
// the imaginary parts at k = 0 and, for even ny, k = ny/2, as any
// complex-to-real transform does), transforms Z_k = A_k + i B_k once and
// returns a as the real and b as the imaginary part. The factor 2 of the
// forward unpacking stands for the one every other grid's real-to-complex
// step along z carries, so the same scale c = 1 / (2 N) applies.
//
// Spectral layout: S[9][nx][ny] as for any grid with nzh = 1; the half
// spectrum of column x sits in S[c][x][0 .. ny/2]. Each CTA owns whole
// columns (y passes) or whole x lines (x pass) of the components it touches,
// so the in-place updates are race free.
#include "fft_core.cuh"
#include "fh_kernels.h"

namespace fh {

namespace {

size_t plane_smem(const FftPlan& p, int L) {
  // two buffers of two pencils (a Rader plan uses slot L of each pencil) and the axis tables
  return ((size_t)2 * 2 * (L + 1) + (p.L ? p.tw_len : L)) * sizeof(double2);
}

// CTA (row i, x pair x0 = 2 xp, x1 = x0 + 1): forward along y of the columns
// j = x, y of row i at x0 and x1 (x1 = nx is a zero column); writes T_ix and
// W_i = xi_y T_iy to the half spectra of x0 and x1
template <int L>
__global__ void __launch_bounds__(kThreads) k_plane_fwd_y(Grid g, double2* __restrict__ S,
                                                         const double2* __restrict__ tw,
                                                         const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  extern __shared__ double2 smem[];
  const int Ln = L > 0 ? L : g.ny;
  const int QS = Ln + 1;
  double2* bufA = smem;
  double2* bufB = smem + 2 * QS;
  double2* twL = bufB + 2 * QS;
  stage_axis_twiddles<L, 1>(twL, tw, g);
  const int i = blockIdx.x % 3;
  const int x0 = 2 * (blockIdx.x / 3);
  const bool has_b = x0 + 1 < g.nx;
  const long long ca = (long long)x0 * Ln, cb = ca + Ln;
  for (int t = threadIdx.x; t < 2 * Ln; t += blockDim.x) {
    const int f = t >= Ln, y = t - f * Ln;
    const double2* Sf = S + (3 * i + f) * g.nspec;
    bufA[f * QS + y] = make_double2(Sf[ca + y].x, has_b ? Sf[cb + y].x : 0.0);
  }
  const double2* R = fft_pencils_any<L, false, true>(bufA, bufB, PencilLayout{2, QS, 1, 2, 2}, twL, g.py);
  const int nyh = Ln / 2 + 1;
  double2* S0 = S + (3 * i + 0) * g.nspec;
  double2* S1 = S + (3 * i + 1) * g.nspec;
  for (int k = threadIdx.x; k < nyh; k += blockDim.x) {
    const int km = k == 0 ? 0 : Ln - k;
    const double xi_y = wave_int(k, Ln) * g.sy;
    const double2 zx = R[k], zxm = R[km];
    const double2 zy = R[QS + k], zym = R[QS + km];
    S0[ca + k] = make_double2(zx.x + zxm.x, zx.y - zxm.y);
    S1[ca + k] = make_double2(xi_y * (zy.x + zym.x), xi_y * (zy.y - zym.y));
    if (has_b) {
      S0[cb + k] = make_double2(zx.y + zxm.y, zxm.x - zx.x);
      S1[cb + k] = make_double2(xi_y * (zy.y + zym.y), xi_y * (zym.x - zy.x));
    }
  }
}

// CTA (row i, ky = 0 .. ny/2): forward along x of T_ix and W_i, Ghat on row i
// (v_i = s (xi_x T_ix + W_i), s = c / |xi|^2, 0 at xi = 0), inverse along x of
// A_i = xi_x v_i and B_i = v_i
template <int L>
__global__ void __launch_bounds__(kThreads) k_plane_x_ghat(Grid g, double2* __restrict__ S,
                                                          const double2* __restrict__ tw, double scale,
                                                          const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  extern __shared__ double2 smem[];
  const int Ln = L > 0 ? L : g.nx;
  const int QS = Ln + 1;
  double2* bufA = smem;
  double2* bufB = smem + 2 * QS;
  double2* twL = bufB + 2 * QS;
  stage_axis_twiddles<L, 0>(twL, tw, g);
  const int i = blockIdx.x % 3;
  const int ky = blockIdx.x / 3;
  const long long row = g.ny;  // stride of x in S
  for (int t = threadIdx.x; t < 2 * Ln; t += blockDim.x) {
    const int f = t >= Ln, x = t - f * Ln;
    bufA[f * QS + x] = S[(3 * i + f) * g.nspec + x * row + ky];
  }
  double2* R = fft_pencils_any<L, false, true>(bufA, bufB, PencilLayout{2, QS, 1, 2, 2}, twL, g.px);
  const double xi_y = wave_int(ky, g.ny) * g.sy;
  for (int kx = threadIdx.x; kx < Ln; kx += blockDim.x) {
    const double xi_x = wave_int(kx, Ln) * g.sx;
    const double d = fma(xi_x, xi_x, xi_y * xi_y);
    const double s = d > 0.0 ? scale / d : 0.0;
    const double2 X = R[kx], W = R[QS + kx];
    const double2 v = make_double2(s * fma(xi_x, X.x, W.x), s * fma(xi_x, X.y, W.y));
    R[kx] = cscale(v, xi_x);
    R[QS + kx] = v;
  }
  double2* other = (R == bufA) ? bufB : bufA;
  const double2* R2 = fft_pencils_any<L, true, true>(R, other, PencilLayout{2, QS, 1, 2, 2}, twL, g.px);
  for (int t = threadIdx.x; t < 2 * Ln; t += blockDim.x) {
    const int f = t >= Ln, x = t - f * Ln;
    S[(3 * i + f) * g.nspec + x * row + ky] = R2[f * QS + x];
  }
}

// CTA (row i, x pair): inverse along y of y_ix = A_i and y_iy = xi_y B_i at
// x0 and x1 from their half spectra; y_iz = xi_z B_i = 0. The real results
// are stored as (value, 0) for the inverse z pass.
template <int L>
__global__ void __launch_bounds__(kThreads) k_plane_inv_y(Grid g, double2* __restrict__ S,
                                                         const double2* __restrict__ tw,
                                                         const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  extern __shared__ double2 smem[];
  const int Ln = L > 0 ? L : g.ny;
  const int QS = Ln + 1;
  double2* bufA = smem;
  double2* bufB = smem + 2 * QS;
  double2* twL = bufB + 2 * QS;
  stage_axis_twiddles<L, 1>(twL, tw, g);
  const int i = blockIdx.x % 3;
  const int x0 = 2 * (blockIdx.x / 3);
  const bool has_b = x0 + 1 < g.nx;
  const long long ca = (long long)x0 * Ln, cb = ca + Ln;
  const int nyh = Ln / 2 + 1;
  for (int t = threadIdx.x; t < 2 * Ln; t += blockDim.x) {
    const int f = t >= Ln, k = t - f * Ln;
    const bool lo = k < nyh;
    const int ka = lo ? k : Ln - k;
    const double2* Sf = S + (3 * i + f) * g.nspec;
    double2 a = Sf[ca + ka];
    double2 b = has_b ? Sf[cb + ka] : make_double2(0.0, 0.0);
    if (f == 1) {
      const double xi_y = wave_int(ka, Ln) * g.sy;
      a = cscale(a, xi_y);
      b = cscale(b, xi_y);
    }
    if (ka == 0 || 2 * ka == Ln) {
      a.y = 0.0;
      b.y = 0.0;
    }
    if (!lo) {
      a.y = -a.y;
      b.y = -b.y;
    }
    bufA[f * QS + k] = make_double2(a.x - b.y, a.y + b.x);  // a + i b
  }
  const double2* R = fft_pencils_any<L, true, true>(bufA, bufB, PencilLayout{2, QS, 1, 2, 2}, twL, g.py);
  double2* S0 = S + (3 * i + 0) * g.nspec;
  double2* S1 = S + (3 * i + 1) * g.nspec;
  double2* S2 = S + (3 * i + 2) * g.nspec;
  const double2 zero = make_double2(0.0, 0.0);
  for (int y = threadIdx.x; y < Ln; y += blockDim.x) {
    const double2 u = R[y], w = R[QS + y];
    S0[ca + y] = make_double2(u.x, 0.0);
    S1[ca + y] = make_double2(w.x, 0.0);
    S2[ca + y] = zero;
    if (has_b) {
      S0[cb + y] = make_double2(u.y, 0.0);
      S1[cb + y] = make_double2(w.y, 0.0);
      S2[cb + y] = zero;
    }
  }
}

template <class Kern>
cudaError_t allow(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

#define FH_PLANE_LENGTHS(MACRO) \
  MACRO(1)                      \
  MACRO(2)                      \
  MACRO(3)                      \
  MACRO(4)                      \
  MACRO(6)                      \
  MACRO(8)                      \
  MACRO(12)                     \
  MACRO(16)                     \
  MACRO(24)                     \
  MACRO(32)                     \
  MACRO(48)                     \
  MACRO(64)                     \
  MACRO(96)                     \
  MACRO(128)                    \
  MACRO(192)                    \
  MACRO(256)

cudaError_t setup_plane_kernels(const Grid& g) {
  cudaError_t e = cudaSuccess;
  const size_t sy = plane_smem(g.py, g.ny), sx = plane_smem(g.px, g.nx);
#define YSET(V)                                                     \
  case V:                                                           \
    if ((e = allow(k_plane_fwd_y<V>, sy))) return e;                \
    if ((e = allow(k_plane_inv_y<V>, sy))) return e;                \
    break;
#define XSET(V)                                                     \
  case V:                                                           \
    if ((e = allow(k_plane_x_ghat<V>, sx))) return e;               \
    break;
  if (g.py.L) {
    if ((e = allow(k_plane_fwd_y<0>, sy))) return e;
    if ((e = allow(k_plane_inv_y<0>, sy))) return e;
  } else {
    switch (g.ny) {
      FH_PLANE_LENGTHS(YSET)
      default: return cudaErrorInvalidValue;
    }
  }
  if (g.px.L) {
    if ((e = allow(k_plane_x_ghat<0>, sx))) return e;
  } else {
    switch (g.nx) {
      FH_PLANE_LENGTHS(XSET)
      default: return cudaErrorInvalidValue;
    }
  }
#undef YSET
#undef XSET
  return cudaSuccess;
}

cudaError_t launch_plane_fwd_y(const Grid& g, double2* S, const double2* tw, const CgScalars* cg, cudaStream_t s) {
  const unsigned grid = 3u * (unsigned)((g.nx + 1) / 2);
  const size_t sm = plane_smem(g.py, g.ny);
#define YL(V)                                                        \
  case V:                                                            \
    k_plane_fwd_y<V><<<grid, kThreads, sm, s>>>(g, S, tw, cg);       \
    break;
  if (g.py.L) {
    k_plane_fwd_y<0><<<grid, kThreads, sm, s>>>(g, S, tw, cg);
  } else {
    switch (g.ny) {
      FH_PLANE_LENGTHS(YL)
      default: return cudaErrorInvalidValue;
    }
  }
#undef YL
  return cudaGetLastError();
}

cudaError_t launch_plane_x_ghat(const Grid& g, double2* S, const double2* tw, double scale, const CgScalars* cg,
                                cudaStream_t s) {
  const unsigned grid = 3u * (unsigned)(g.ny / 2 + 1);
  const size_t sm = plane_smem(g.px, g.nx);
#define XL(V)                                                               \
  case V:                                                                   \
    k_plane_x_ghat<V><<<grid, kThreads, sm, s>>>(g, S, tw, scale, cg);      \
    break;
  if (g.px.L) {
    k_plane_x_ghat<0><<<grid, kThreads, sm, s>>>(g, S, tw, scale, cg);
  } else {
    switch (g.nx) {
      FH_PLANE_LENGTHS(XL)
      default: return cudaErrorInvalidValue;
    }
  }
#undef XL
  return cudaGetLastError();
}

cudaError_t launch_plane_inv_y(const Grid& g, double2* S, const double2* tw, const CgScalars* cg, cudaStream_t s) {
  const unsigned grid = 3u * (unsigned)((g.nx + 1) / 2);
  const size_t sm = plane_smem(g.py, g.ny);
#define IYL(V)                                                       \
  case V:                                                            \
    k_plane_inv_y<V><<<grid, kThreads, sm, s>>>(g, S, tw, cg);       \
    break;
  if (g.py.L) {
    k_plane_inv_y<0><<<grid, kThreads, sm, s>>>(g, S, tw, cg);
  } else {
    switch (g.ny) {
      FH_PLANE_LENGTHS(IYL)
      default: return cudaErrorInvalidValue;
    }
  }
#undef IYL
  return cudaGetLastError();
}

}  // namespace fh
