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
#include "fft_df64.cuh"
#include "passes.cuh"

namespace fh {

namespace {

size_t plane_smem(const FftPlan& p, int L) {
  // two buffers of two pencils (a Rader plan uses slot L of each pencil) and
  // the axis tables; double2 and dfc entries are both 16 bytes
  return ((size_t)2 * 2 * (L + 1) + (p.L ? p.tw_len : L)) * sizeof(double2);
}

// (re a) + i (re b), and the imaginary part of u as a real entry
__device__ __forceinline__ double2 cpack_real(double2 a, double2 b) { return make_double2(a.x, b.x); }
__device__ __forceinline__ dfc cpack_real(dfc a, dfc b) { return dfc{a.re, b.re}; }
__device__ __forceinline__ double2 cimag_real(double2 u) { return make_double2(u.y, 0.0); }
__device__ __forceinline__ dfc cimag_real(dfc u) { return dfc{u.im, df64{0.f, 0.f}}; }

// CTA (row i, x pair x0 = 2 xp, x1 = x0 + 1): forward along y of the columns
// j = x, y of row i at x0 and x1 (x1 = nx is a zero column); writes T_ix and
// W_i = xi_y T_iy to the half spectra of x0 and x1
template <int L, class C>
__global__ void __launch_bounds__(kThreads) k_plane_fwd_y(Grid g, C* __restrict__ S, const C* __restrict__ tw,
                                                         const CgScalars* __restrict__ cg) {
  using R = typename RealOf<C>::type;
  if (cg_done(cg)) return;
  C* smem = pass_smem<C>();
  const int Ln = L > 0 ? L : g.ny;
  const int QS = Ln + 1;
  C* bufA = smem;
  C* bufB = smem + 2 * QS;
  C* twL = bufB + 2 * QS;
  stage_axis_twiddles<L, 1>(twL, tw, g);
  const int i = blockIdx.x % 3;
  const int x0 = 2 * (blockIdx.x / 3);
  const bool has_b = x0 + 1 < g.nx;
  const long long ca = (long long)x0 * Ln, cb = ca + Ln;
  C zero;
  czero(zero);
  for (int t = threadIdx.x; t < 2 * Ln; t += blockDim.x) {
    const int f = t >= Ln, y = t - f * Ln;
    const C* Sf = S + (3 * i + f) * g.nspec;
    bufA[f * QS + y] = cpack_real(Sf[ca + y], has_b ? Sf[cb + y] : zero);
  }
  const C* Rp = fft_pencils_any<L, false, true>(bufA, bufB, PencilLayout{2, QS, 1, 2, 2}, twL, g.py);
  const int nyh = Ln / 2 + 1;
  C* S0 = S + (3 * i + 0) * g.nspec;
  C* S1 = S + (3 * i + 1) * g.nspec;
  const R rsy = to_real(g.sy, (C*)nullptr);
  for (int k = threadIdx.x; k < nyh; k += blockDim.x) {
    const int km = k == 0 ? 0 : Ln - k;
    const R xi_y = wave_real(wave_int(k, Ln), rsy);
    const C zx = Rp[k], zxm = Rp[km];
    const C zy = Rp[QS + k], zym = Rp[QS + km];
    S0[ca + k] = cadd_conj(zx, zxm);                             // 2 A_k of column x0
    S1[ca + k] = cscale(cadd_conj(zy, zym), xi_y);
    if (has_b) {
      S0[cb + k] = mul_mi<false>(csub_conj(zx, zxm));            // 2 B_k = -i (Z_k - conj Z_-k)
      S1[cb + k] = cscale(mul_mi<false>(csub_conj(zy, zym)), xi_y);
    }
  }
}

// CTA (row i, ky = 0 .. ny/2): forward along x of T_ix and W_i, Ghat on row i
// (v_i = s (xi_x T_ix + W_i), s = c / |xi|^2, 0 at xi = 0), inverse along x of
// A_i = xi_x v_i and B_i = v_i
template <int L, class C>
__global__ void __launch_bounds__(kThreads) k_plane_x_ghat(Grid g, C* __restrict__ S, const C* __restrict__ tw,
                                                          double scale, const CgScalars* __restrict__ cg) {
  using R = typename RealOf<C>::type;
  if (cg_done(cg)) return;
  C* smem = pass_smem<C>();
  const int Ln = L > 0 ? L : g.nx;
  const int QS = Ln + 1;
  C* bufA = smem;
  C* bufB = smem + 2 * QS;
  C* twL = bufB + 2 * QS;
  stage_axis_twiddles<L, 0>(twL, tw, g);
  const int i = blockIdx.x % 3;
  const int ky = blockIdx.x / 3;
  const long long row = g.ny;  // stride of x in S
  for (int t = threadIdx.x; t < 2 * Ln; t += blockDim.x) {
    const int f = t >= Ln, x = t - f * Ln;
    bufA[f * QS + x] = S[(3 * i + f) * g.nspec + x * row + ky];
  }
  C* Rx = fft_pencils_any<L, false, true>(bufA, bufB, PencilLayout{2, QS, 1, 2, 2}, twL, g.px);
  const R rsx = to_real(g.sx, (C*)nullptr), rc = to_real(scale, (C*)nullptr);
  const R xi_y = wave_real(wave_int(ky, g.ny), to_real(g.sy, (C*)nullptr));
  const R xi_z = to_real(0.0, (C*)nullptr);
  for (int kx = threadIdx.x; kx < Ln; kx += blockDim.x) {
    const R xi_x = wave_real(wave_int(kx, Ln), rsx);
    const R s = ghat_scale(xi_x, xi_y, xi_z, rc);
    const C v = cscale(caxpy(xi_x, Rx[kx], Rx[QS + kx]), s);
    Rx[kx] = cscale(v, xi_x);
    Rx[QS + kx] = v;
  }
  C* other = (Rx == bufA) ? bufB : bufA;
  const C* R2 = fft_pencils_any<L, true, true>(Rx, other, PencilLayout{2, QS, 1, 2, 2}, twL, g.px);
  for (int t = threadIdx.x; t < 2 * Ln; t += blockDim.x) {
    const int f = t >= Ln, x = t - f * Ln;
    S[(3 * i + f) * g.nspec + x * row + ky] = R2[f * QS + x];
  }
}

// CTA (row i, x pair): inverse along y of y_ix = A_i and y_iy = xi_y B_i at
// x0 and x1 from their half spectra; y_iz = xi_z B_i = 0. The real results
// are stored as real entries for the inverse z pass.
template <int L, class C>
__global__ void __launch_bounds__(kThreads) k_plane_inv_y(Grid g, C* __restrict__ S, const C* __restrict__ tw,
                                                         const CgScalars* __restrict__ cg) {
  using R = typename RealOf<C>::type;
  if (cg_done(cg)) return;
  C* smem = pass_smem<C>();
  const int Ln = L > 0 ? L : g.ny;
  const int QS = Ln + 1;
  C* bufA = smem;
  C* bufB = smem + 2 * QS;
  C* twL = bufB + 2 * QS;
  stage_axis_twiddles<L, 1>(twL, tw, g);
  const int i = blockIdx.x % 3;
  const int x0 = 2 * (blockIdx.x / 3);
  const bool has_b = x0 + 1 < g.nx;
  const long long ca = (long long)x0 * Ln, cb = ca + Ln;
  const int nyh = Ln / 2 + 1;
  const R rsy = to_real(g.sy, (C*)nullptr);
  C zero;
  czero(zero);
  for (int t = threadIdx.x; t < 2 * Ln; t += blockDim.x) {
    const int f = t >= Ln, k = t - f * Ln;
    const bool lo = k < nyh;
    const int ka = lo ? k : Ln - k;
    const C* Sf = S + (3 * i + f) * g.nspec;
    C a = Sf[ca + ka];
    C b = has_b ? Sf[cb + ka] : zero;
    if (f == 1) {
      const R xi_y = wave_real(wave_int(ka, Ln), rsy);
      a = cscale(a, xi_y);
      b = cscale(b, xi_y);
    }
    if (ka == 0 || 2 * ka == Ln) {
      a = creal(a);
      b = creal(b);
    }
    if (!lo) {
      a = cconj(a);
      b = cconj(b);
    }
    bufA[f * QS + k] = cadd(a, mul_mi<true>(b));  // a + i b
  }
  const C* Rp = fft_pencils_any<L, true, true>(bufA, bufB, PencilLayout{2, QS, 1, 2, 2}, twL, g.py);
  C* S0 = S + (3 * i + 0) * g.nspec;
  C* S1 = S + (3 * i + 1) * g.nspec;
  C* S2 = S + (3 * i + 2) * g.nspec;
  for (int y = threadIdx.x; y < Ln; y += blockDim.x) {
    const C u = Rp[y], w = Rp[QS + y];
    S0[ca + y] = creal(u);
    S1[ca + y] = creal(w);
    S2[ca + y] = zero;
    if (has_b) {
      S0[cb + y] = cimag_real(u);
      S1[cb + y] = cimag_real(w);
      S2[cb + y] = zero;
    }
  }
}

template <class Kern>
cudaError_t allow(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

namespace {

template <class C>
cudaError_t setup_plane(const Grid& g) {
  cudaError_t e = cudaSuccess;
  const size_t sy = plane_smem(g.py, g.ny), sx = plane_smem(g.px, g.nx);
#define YSET(V)                                                     \
  case V:                                                           \
    if ((e = allow(k_plane_fwd_y<V, C>, sy))) return e;             \
    if ((e = allow(k_plane_inv_y<V, C>, sy))) return e;             \
    break;
#define XSET(V)                                                     \
  case V:                                                           \
    if ((e = allow(k_plane_x_ghat<V, C>, sx))) return e;            \
    break;
  if (g.py.L) {
    if ((e = allow(k_plane_fwd_y<0, C>, sy))) return e;
    if ((e = allow(k_plane_inv_y<0, C>, sy))) return e;
  } else {
    FH_SWITCH_LEN(g.ny, YSET)
  }
  if (g.px.L) {
    if ((e = allow(k_plane_x_ghat<0, C>, sx))) return e;
  } else {
    FH_SWITCH_LEN(g.nx, XSET)
  }
#undef YSET
#undef XSET
  return cudaSuccess;
}

template <class C>
cudaError_t plane_fwd_y(const Grid& g, C* S, const C* tw, const CgScalars* cg, cudaStream_t s) {
  const unsigned grid = 3u * (unsigned)((g.nx + 1) / 2);
  const size_t sm = plane_smem(g.py, g.ny);
#define YL(V)                                                        \
  case V:                                                            \
    k_plane_fwd_y<V, C><<<grid, kThreads, sm, s>>>(g, S, tw, cg);    \
    break;
  if (g.py.L) {
    k_plane_fwd_y<0, C><<<grid, kThreads, sm, s>>>(g, S, tw, cg);
  } else {
    FH_SWITCH_LEN(g.ny, YL)
  }
#undef YL
  return cudaGetLastError();
}

template <class C>
cudaError_t plane_x_ghat(const Grid& g, C* S, const C* tw, double scale, const CgScalars* cg, cudaStream_t s) {
  const unsigned grid = 3u * (unsigned)(g.ny / 2 + 1);
  const size_t sm = plane_smem(g.px, g.nx);
#define XL(V)                                                               \
  case V:                                                                   \
    k_plane_x_ghat<V, C><<<grid, kThreads, sm, s>>>(g, S, tw, scale, cg);   \
    break;
  if (g.px.L) {
    k_plane_x_ghat<0, C><<<grid, kThreads, sm, s>>>(g, S, tw, scale, cg);
  } else {
    FH_SWITCH_LEN(g.nx, XL)
  }
#undef XL
  return cudaGetLastError();
}

template <class C>
cudaError_t plane_inv_y(const Grid& g, C* S, const C* tw, const CgScalars* cg, cudaStream_t s) {
  const unsigned grid = 3u * (unsigned)((g.nx + 1) / 2);
  const size_t sm = plane_smem(g.py, g.ny);
#define IYL(V)                                                       \
  case V:                                                            \
    k_plane_inv_y<V, C><<<grid, kThreads, sm, s>>>(g, S, tw, cg);    \
    break;
  if (g.py.L) {
    k_plane_inv_y<0, C><<<grid, kThreads, sm, s>>>(g, S, tw, cg);
  } else {
    FH_SWITCH_LEN(g.ny, IYL)
  }
#undef IYL
  return cudaGetLastError();
}

}  // namespace

cudaError_t setup_plane_kernels(const Grid& g) {
  cudaError_t e = setup_plane<double2>(g);
  return e != cudaSuccess ? e : setup_plane<dfc>(g);
}
cudaError_t launch_plane_fwd_y(const Grid& g, double2* S, const double2* tw, const CgScalars* cg, cudaStream_t s) {
  return plane_fwd_y(g, S, tw, cg, s);
}
cudaError_t launch_plane_x_ghat(const Grid& g, double2* S, const double2* tw, double scale, const CgScalars* cg,
                                cudaStream_t s) {
  return plane_x_ghat(g, S, tw, scale, cg, s);
}
cudaError_t launch_plane_inv_y(const Grid& g, double2* S, const double2* tw, const CgScalars* cg, cudaStream_t s) {
  return plane_inv_y(g, S, tw, cg, s);
}
cudaError_t launch_plane_fwd_y(const Grid& g, dfc* S, const dfc* tw, const CgScalars* cg, cudaStream_t s) {
  return plane_fwd_y(g, S, tw, cg, s);
}
cudaError_t launch_plane_x_ghat(const Grid& g, dfc* S, const dfc* tw, double scale, const CgScalars* cg,
                                cudaStream_t s) {
  return plane_x_ghat(g, S, tw, scale, cg, s);
}
cudaError_t launch_plane_inv_y(const Grid& g, dfc* S, const dfc* tw, const CgScalars* cg, cudaStream_t s) {
  return plane_inv_y(g, S, tw, cg, s);
}

}  // namespace fh
