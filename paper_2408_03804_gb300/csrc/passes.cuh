// The five passes of one application of the compatibility projection G of
// Eq. 1 to a nine-component real field, with the stages of the CG
// matrix-vector product y = G(K : p) fused into the first and last pass.
//
// Spectral layout: one complex buffer S[9][nx][ny][nzh] (nzh = nz/2 + 1) that
// every pass updates in place. Ghat(xi)[Ahat] = v (x) xi with
// v = Ahat xi / |xi|^2, a rank structure that removes a third of the 1D
// transforms of the two outer passes:
//
//   z  (forward, real-to-complex): tau = K : p (or P), transform along z,
//      multiply the j = z column by xi_z                         9 transforms
//   y  (forward): transform the i-th row (j = x, y, z) along y, keep
//      T_ix and form W_i = xi_y T_iy + T_iz                      9 transforms
//   x  (forward + Ghat + inverse): transform T_ix, W_i along x,
//      v_i = s (xi_x T_ix + W_i), s = c / |xi|^2 (0 at xi = 0),
//      inverse-transform A_i = xi_x v_i and B_i = v_i along x   6 + 6 transforms
//   y  (inverse): y_ix <- A_i, y_iy <- xi_y B_i, y_iz <- B_i,
//      inverse transform along y, multiply y_iz by xi_z         9 transforms
//   z  (inverse, complex-to-real): back to the real field, optionally the
//      CG dot product p . y in the same pass                     9 transforms
//
// All transforms are unnormalised; the real-to-complex step skips its usual
// factor 1/2, so the constant c carries 1 / (2 N) together with the caller's
// scale. Each CTA owns a disjoint region of S in every pass, so in-place
// updates are race free.
//
// The bodies are templates over the element type C of the spectrum and of
// the shared-memory pencils: double2 (IEEE FP64, kernels_fft.cu) or dfc
// (double-float, kernels_df64.cu). The CG updates and the dot products
// work on the FP64 fields in both; the double-float form converts p (or the
// source field) to double-float in the z pass, forms K : p from a
// double-float copy of the tangent, and converts the result back in the
// inverse z pass. Both element types cover every grid: compile-time plans (L > 0),
// run-time plans (L = 0) and plane cells (M = 0).
#pragma once

#include "df64.cuh"
#include "fft_core.cuh"
#include "fh_kernels.h"

namespace fh {

// ---- the element types' scalar operations ---------------------------------
template <class C>
struct RealOf;
template <>
struct RealOf<double2> {
  using type = double;
};
template <>
struct RealOf<dfc> {
  using type = df64;
};

__device__ __forceinline__ double to_real(double x, double2*) { return x; }
__device__ __forceinline__ df64 to_real(double x, dfc*) { return to_df64(x); }

// wave number k * scale (scale already converted to the element's real type)
__device__ __forceinline__ double wave_real(int k, double sc) { return k * sc; }
__device__ __forceinline__ df64 wave_real(int k, df64 sc) { return dd_mul(df64{(float)k, 0.f}, sc); }


// a + conj(b), a - conj(b), conj(a), a with its imaginary part dropped
__device__ __forceinline__ double2 cadd_conj(double2 a, double2 b) { return make_double2(a.x + b.x, a.y - b.y); }
__device__ __forceinline__ double2 csub_conj(double2 a, double2 b) { return make_double2(a.x - b.x, a.y + b.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 creal(double2 a) { return make_double2(a.x, 0.0); }
__device__ __forceinline__ dfc cadd_conj(dfc a, dfc b) { return dfc{dd_add(a.re, b.re), dd_sub(a.im, b.im)}; }
__device__ __forceinline__ dfc csub_conj(dfc a, dfc b) { return dfc{dd_sub(a.re, b.re), dd_add(a.im, b.im)}; }
__device__ __forceinline__ dfc cconj(dfc a) { return dfc{a.re, dd_neg(a.im)}; }
__device__ __forceinline__ dfc creal(dfc a) { return dfc{a.re, df64{0.f, 0.f}}; }


// the real sequence packed two per complex entry (a real-to-complex step)
// a real value as a complex entry, and the real part of an entry as a double
__device__ __forceinline__ double2 cfrom_real(double v) { return make_double2(v, 0.0); }
__device__ __forceinline__ dfc cfrom_real(df64 v) { return dfc{v, df64{0.f, 0.f}}; }
__device__ __forceinline__ double creal_double(double2 a) { return a.x; }
__device__ __forceinline__ double creal_double(dfc a) { return join_df64(a.re); }

__device__ __forceinline__ void store_real(double2* buf, int i, double v) { reinterpret_cast<double*>(buf)[i] = v; }
__device__ __forceinline__ void store_real(dfc* buf, int i, df64 v) { reinterpret_cast<df64*>(buf)[i] = v; }
__device__ __forceinline__ double load_real(const double2* buf, int i) {
  return reinterpret_cast<const double*>(buf)[i];
}
__device__ __forceinline__ double load_real(const dfc* buf, int i) {
  return join_df64(reinterpret_cast<const df64*>(buf)[i]);
}

// s = c / |xi|^2, 0 at xi = 0
__device__ __forceinline__ double ghat_scale(double xx, double xy, double xz, double c) {
  const double d = fma(xx, xx, fma(xy, xy, xz * xz));
  return d > 0.0 ? c / d : 0.0;
}
__device__ __forceinline__ df64 ghat_scale(df64 xx, df64 xy, df64 xz, df64 c) {
  const df64 d = dd_fma(xx, xx, dd_fma(xy, xy, dd_mul(xz, xz)));
  if (!(d.hi > 0.f)) return df64{0.f, 0.f};
  // long division: q1 = c / d in FP32, then the FP32 quotient of the remainder
  const float q1 = c.hi / d.hi;
  const df64 r = dd_sub(c, dd_mul(df64{q1, 0.f}, d));
  const float q2 = r.hi / d.hi;
  return fast_two_sum(q1, q2);
}

// dynamic shared memory as pencils of C
template <class C>
__device__ __forceinline__ C* pass_smem() {
  extern __shared__ __align__(16) unsigned char fh_pass_smem[];
  return reinterpret_cast<C*>(fh_pass_smem);
}

// dispatch on the lengths with compile-time plans: the x and y extents, and
// the half extent nz/2 of the real-to-complex axis (up to 128; 0 for nz = 1,
// whose z passes are the identity)
#define FH_HALF_LENGTHS(MACRO) \
  MACRO(1) MACRO(2) MACRO(3) MACRO(4) MACRO(6) MACRO(8) MACRO(12) MACRO(16) MACRO(24) MACRO(32) MACRO(48) \
  MACRO(64) MACRO(96) MACRO(128)
#define FH_SWITCH_LEN(v, MACRO)        \
  switch (v) {                         \
    FH_HALF_LENGTHS(MACRO)             \
    MACRO(192)                         \
    MACRO(256)                         \
    default:                           \
      return cudaErrorInvalidValue;    \
  }
#define FH_SWITCH_HALF(v, MACRO)       \
  switch (v) {                         \
    MACRO(0)                           \
    FH_HALF_LENGTHS(MACRO)             \
    default:                           \
      return cudaErrorInvalidValue;    \
  }
#define FH_SWITCH_HALF_EVEN(v, MACRO)  \
  switch (v) {                         \
    FH_HALF_LENGTHS(MACRO)             \
    default:                           \
      return cudaErrorInvalidValue;    \
  }

// ---------------------------------------------------------------------------
// forward z pass: real-to-complex along z of LB consecutive z lines
// ---------------------------------------------------------------------------
// tau = K : p (or the source field) at voxel gi; the CG modes first advance
// x and p of the previous iteration at this voxel (FP64 in both forms). R is
// the real type of tau and of the packed tangent K: double, or df64 for the
// double-float passes, which read a double-float copy of K and form K : p
// with double-float fused multiply-adds.
__device__ __forceinline__ double real_from(double v, double*) { return v; }
__device__ __forceinline__ df64 real_from(double v, df64*) { return split_double(v); }
__device__ __forceinline__ double real_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ df64 real_fma(df64 a, df64 b, df64 c) { return dd_fma(a, b, c); }
__device__ __forceinline__ double real_mul(double a, double b) { return a * b; }
__device__ __forceinline__ df64 real_mul(df64 a, df64 b) { return dd_mul(a, b); }

template <int MODE, class R>
__device__ __forceinline__ void z_pass_tau(long long gi, long long n, const double* __restrict__ src,
                                           double* __restrict__ p, double* __restrict__ x,
                                           const R* __restrict__ K, double alpha, double beta, R tau[9]) {
  if constexpr (MODE == kZDirect) {
#pragma unroll
    for (int c = 0; c < 9; ++c) tau[c] = real_from(src[c * n + gi], (R*)nullptr);
  } else {
    R pv[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      double v;
      if constexpr (MODE == kZKApply) {
        v = src[c * n + gi];
      } else if constexpr (MODE == kZCgFirst) {
        v = src[c * n + gi];
        p[c * n + gi] = v;
      } else {
        // the previous iteration's x += alpha p, then p = r + beta p
        const double po = p[c * n + gi];
        x[c * n + gi] = fma(alpha, po, x[c * n + gi]);
        v = fma(beta, po, src[c * n + gi]);
        p[c * n + gi] = v;
      }
      pv[c] = real_from(v, (R*)nullptr);
    }
    R k[45];
#pragma unroll
    for (int s = 0; s < 45; ++s) k[s] = K[s * n + gi];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      R acc = real_mul(k[sym_slot(a, 0)], pv[0]);
#pragma unroll
      for (int b = 1; b < 9; ++b) acc = real_fma(k[sym_slot(a, b)], pv[b], acc);
      tau[a] = acc;
    }
  }
}

// M = nz / 2; M = 0 is a cell one voxel thick along z (nz = 1), whose
// transform along z is the identity
template <int M, int MODE, class C>
__device__ __forceinline__ void fwd_z_body(int cta, Grid g, int LB, const double* __restrict__ src,
                                           double* __restrict__ p, double* __restrict__ x,
                                           const typename RealOf<C>::type* __restrict__ K,
                                           const CgScalars* __restrict__ cg, C* __restrict__ S,
                                           const C* __restrict__ tw) {
  using R = typename RealOf<C>::type;
  const long long n = g.n;
  double beta = 0.0, alpha = 0.0;
  if constexpr (MODE == kZCg) {
    beta = cg->beta;
    alpha = cg->alpha;
  }
  if constexpr (M == 0) {
    // X_0 = tau, real (the plane y pass supplies the factor 2 of a
    // real-to-complex step); the j = z columns, multiplied by xi_z = 0, are
    // not read by the plane passes and are not written
    const long long v0 = (long long)cta * LB;
    for (int t = threadIdx.x; t < LB; t += blockDim.x) {
      const long long gi = v0 + t;
      R tau[9];
      z_pass_tau<MODE>(gi, n, src, p, x, K, alpha, beta, tau);
#pragma unroll
      for (int c = 0; c < 9; ++c)
        if (c % 3 != 2) S[c * g.nspec + gi] = cfrom_real(tau[c]);
    }
  } else {
    C* smem = pass_smem<C>();
    constexpr int NZ = 2 * M;
    C* bufA = smem;
    C* bufB = smem + 9 * LB * M;
    C* twM = bufB + 9 * LB * M;  // length-M table (half-length FFT)
    C* twN = twM + M;            // first M/2 + 1 entries of the length-NZ table (unpack; tangent form in FP64)
    stage_fft_twiddles<M>(twM, tw, M);
    stage_fft_twiddles<NZ>(twN, tw, M / 2 + 1);
    const long long line0 = (long long)cta * LB;
    const long long v0 = line0 * NZ;

    for (int t = threadIdx.x; t < LB * NZ; t += blockDim.x) {
      const long long gi = v0 + t;
      const int line = t / NZ, z = t % NZ;
      R tau[9];
      z_pass_tau<MODE>(gi, n, src, p, x, K, alpha, beta, tau);
#pragma unroll
      for (int c = 0; c < 9; ++c) store_real(bufA, (c * LB + line) * NZ + z, tau[c]);
    }

    C* Rz = fft_pencils<M, false, true>(bufA, bufB, PencilLayout{9 * LB, M, 1, 1, 1}, twM);

    // unpack the half-length transform Z of z_m = x_2m + i x_2m+1 into
    // 2 X_k = (Z_k + conj Z_{M-k}) - i w^k (Z_k - conj Z_{M-k}), k = 0..M
    const R rsz = to_real(g.sz, (C*)nullptr);
    constexpr int KH = M / 2 + 1;
    for (int t = threadIdx.x; t < 9 * LB * KH; t += blockDim.x) {
      const int q = t / KH, k = t % KH;
      const int c = q / LB, line = q % LB;
      const C* Zq = Rz + q * M;
      const C zk = Zq[k];
      const C zm = Zq[k == 0 ? 0 : M - k];
      const C e = cadd_conj(zk, zm);
      const C o = csub_conj(zk, zm);
      C xk, xm;
      if constexpr (IsFp64Complex<C>::value) {
        unpack_pair_tan(e, o, tan_twiddle<NZ, false>(twN, k), xk, xm);
      } else {
        const C tt = mul_mi<false>(cmul(o, twN[k]));  // -i w^k o
        xk = cadd(e, tt);
        xm = cconj(csub(e, tt));
      }
      C* out = S + (long long)c * g.nspec + (line0 + line) * g.nzh;
      if (c % 3 == 2) {
        xk = cscale(xk, wave_real(wave_int(k, NZ), rsz));
        xm = cscale(xm, wave_real(wave_int(M - k, NZ), rsz));
      }
      out[k] = xk;
      if (M - k != k) out[M - k] = xm;
    }
  }
}

// ---------------------------------------------------------------------------
// inverse z pass: complex-to-real along z, optional dot-product epilogue
// ---------------------------------------------------------------------------
template <int M, int MODE, class C>
__device__ __forceinline__ void inv_z_body(int cta, Grid g, int LB, const C* __restrict__ S,
                                           double* __restrict__ out, const double* __restrict__ p,
                                           double* __restrict__ partials, const C* __restrict__ tw,
                                           const CgScalars* __restrict__ cg) {
  __shared__ double red[32];
  const long long line0 = (long long)cta * LB;
  const long long n = g.n;
  double acc = 0.0;
  if constexpr (M == 0) {
    // nz = 1: the real part of X_0 (complex-to-real semantics)
    for (int t = threadIdx.x; t < LB; t += blockDim.x) {
      const long long gi = line0 + t;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const double yv = creal_double(S[c * g.nspec + gi]);
        out[c * n + gi] = yv;
        if constexpr (MODE == kIZDot) acc = fma(p[c * n + gi], yv, acc);
        if constexpr (MODE == kIZRhs) acc = fma(yv, yv, acc);
      }
    }
  } else {
    C* smem = pass_smem<C>();
    constexpr int NZ = 2 * M;
    C* bufA = smem;
    C* bufB = smem + 9 * LB * M;
    C* twM = bufB + 9 * LB * M;
    C* twN = twM + M;
    stage_fft_twiddles<M>(twM, tw, M);
    stage_fft_twiddles<NZ>(twN, tw, M / 2 + 1);
    __syncthreads();
    // pack Z_k = (X_k + conj X_{M-k}) + i w^-k (X_k - conj X_{M-k}); the
    // imaginary parts of X_0 and X_M are dropped (complex-to-real semantics)
    constexpr int KH = M / 2 + 1;
    for (int t = threadIdx.x; t < 9 * LB * KH; t += blockDim.x) {
      const int q = t / KH, k = t % KH;
      const int c = q / LB, line = q % LB;
      const C* in = S + (long long)c * g.nspec + (line0 + line) * g.nzh;
      C xk = in[k], xm = in[M - k];
      if (k == 0) {
        xk = creal(xk);
        xm = creal(xm);
      }
      const C a = cadd_conj(xk, xm);
      C zk, zm;
      if constexpr (IsFp64Complex<C>::value) {
        pack_pair_tan(a, csub_conj(xk, xm), tan_twiddle<NZ, true>(twN, k), zk, zm);
      } else {
        const C u = mul_mi<true>(cmulc(csub_conj(xk, xm), twN[k]));  // i w^-k b
        zk = cadd(a, u);
        zm = cconj(csub(a, u));
      }
      bufA[q * M + k] = zk;
      if (k != 0 && M - k != k) bufA[q * M + (M - k)] = zm;
    }
    const C* Rz = fft_pencils<M, true, true>(bufA, bufB, PencilLayout{9 * LB, M, 1, 1, 1}, twM);
    for (int t = threadIdx.x; t < LB * NZ; t += blockDim.x) {
      const int line = t / NZ, z = t % NZ;
      const long long gi = (line0 + line) * NZ + z;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        const double yv = load_real(Rz, (c * LB + line) * NZ + z);
        out[c * n + gi] = yv;
        if constexpr (MODE == kIZDot) acc = fma(p[c * n + gi], yv, acc);
        if constexpr (MODE == kIZRhs) acc = fma(yv, yv, acc);
      }
    }
  }
  if constexpr (MODE != kIZOut) {
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[cta] = s;
  }
}

// ---------------------------------------------------------------------------
// forward y pass: row i, columns j = x, y, z along y; combine W_i
// ---------------------------------------------------------------------------
template <int L, class C>
__device__ __forceinline__ void fwd_y_body(int cta, Grid g, int BK, C* __restrict__ S, const C* __restrict__ tw,
                                           const CgScalars* __restrict__ cg) {
  using R = typename RealOf<C>::type;
  C* smem = pass_smem<C>();
  const int Ln = L > 0 ? L : g.ny;
  const int QS = Ln + 1;
  const int np = 3 * BK;
  C* bufA = smem;
  C* bufB = smem + np * QS;
  C* twL = bufB + np * QS;
  stage_axis_twiddles<L, 1>(twL, tw, g);
  const int NC = (g.nzh + BK - 1) / BK;
  int b = cta;
  const int chunk = b % NC;
  b /= NC;
  const int i = b % 3;
  const int x = b / 3;
  const int kz0 = chunk * BK;
  const int valid = min(BK, g.nzh - kz0);
  for (int t = threadIdx.x; t < 3 * Ln * BK; t += blockDim.x) {
    const int kzl = t % BK, rest = t / BK;
    const int y = rest % Ln, f = rest / Ln;
    const int kz = kz0 + kzl;
    C v;
    czero(v);
    if (kz < g.nzh) v = S[(3 * i + f) * g.nspec + ((long long)x * Ln + y) * g.nzh + kz];
    bufA[(f * BK + kzl) * QS + y] = v;
  }
  C* Ry = fft_pencils_any<L, false, true>(bufA, bufB, PencilLayout{np, QS, 1, BK, valid}, twL, g.py);
  const R rsy = to_real(g.sy, (C*)nullptr);
  for (int t = threadIdx.x; t < Ln * BK; t += blockDim.x) {
    const int kzl = t % BK, y = t / BK;
    const int kz = kz0 + kzl;
    if (kz >= g.nzh) continue;
    const R xi_y = wave_real(wave_int(y, Ln), rsy);
    const C tx = Ry[(0 * BK + kzl) * QS + y];
    const C ty = Ry[(1 * BK + kzl) * QS + y];
    const C tz = Ry[(2 * BK + kzl) * QS + y];
    const long long o = ((long long)x * Ln + y) * g.nzh + kz;
    S[(3 * i + 0) * g.nspec + o] = tx;
    S[(3 * i + 1) * g.nspec + o] = caxpy(xi_y, ty, tz);
  }
}

// ---------------------------------------------------------------------------
// x pass: forward along x, Ghat, inverse along x
// ---------------------------------------------------------------------------
template <int L, class C>
__device__ __forceinline__ void x_ghat_body(int cta, Grid g, int BK, C* __restrict__ S, const C* __restrict__ tw,
                                            double scale, const CgScalars* __restrict__ cg) {
  using R = typename RealOf<C>::type;
  C* smem = pass_smem<C>();
  const int Ln = L > 0 ? L : g.nx;
  const int QS = Ln + 1;
  const int np = 6 * BK;
  C* bufA = smem;
  C* bufB = smem + np * QS;
  C* twL = bufB + np * QS;
  stage_axis_twiddles<L, 0>(twL, tw, g);
  const int NC = (g.nzh + BK - 1) / BK;
  const int chunk = cta % NC;
  const int ky = cta / NC;
  const int kz0 = chunk * BK;
  const int valid = min(BK, g.nzh - kz0);
  const long long row = (long long)g.ny * g.nzh;  // stride of x in S
  for (int t = threadIdx.x; t < 6 * Ln * BK; t += blockDim.x) {
    const int kzl = t % BK, rest = t / BK;
    const int x = rest % Ln, f = rest / Ln;
    const int kz = kz0 + kzl;
    const int comp = 3 * (f >> 1) + (f & 1);
    C v;
    czero(v);
    if (kz < g.nzh) v = S[comp * g.nspec + x * row + (long long)ky * g.nzh + kz];
    bufA[(f * BK + kzl) * QS + x] = v;
  }
  C* Rx = fft_pencils_any<L, false, true>(bufA, bufB, PencilLayout{np, QS, 1, BK, valid}, twL, g.px);
  const R rsx = to_real(g.sx, (C*)nullptr), rsz = to_real(g.sz, (C*)nullptr);
  const R rc = to_real(scale, (C*)nullptr);
  const R xi_y = wave_real(wave_int(ky, g.ny), to_real(g.sy, (C*)nullptr));
  for (int t = threadIdx.x; t < Ln * BK; t += blockDim.x) {
    const int kzl = t % BK, kx = t / BK;
    const int kz = kz0 + kzl;
    if (kzl >= valid) continue;
    const R xi_x = wave_real(wave_int(kx, Ln), rsx);
    const R xi_z = wave_real(wave_int(kz, g.nz), rsz);
    const R s = ghat_scale(xi_x, xi_y, xi_z, rc);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      C* pa = Rx + ((2 * i) * BK + kzl) * QS + kx;
      C* pb = Rx + ((2 * i + 1) * BK + kzl) * QS + kx;
      const C v = cscale(caxpy(xi_x, *pa, *pb), s);
      *pa = cscale(v, xi_x);
      *pb = v;
    }
  }
  C* other = (Rx == bufA) ? bufB : bufA;
  const C* R2 = fft_pencils_any<L, true, true>(Rx, other, PencilLayout{np, QS, 1, BK, valid}, twL, g.px);
  for (int t = threadIdx.x; t < 6 * Ln * BK; t += blockDim.x) {
    const int kzl = t % BK, rest = t / BK;
    const int x = rest % Ln, f = rest / Ln;
    const int kz = kz0 + kzl;
    if (kz >= g.nzh) continue;
    const int comp = 3 * (f >> 1) + (f & 1);
    S[comp * g.nspec + x * row + (long long)ky * g.nzh + kz] = R2[(f * BK + kzl) * QS + x];
  }
}

// ---------------------------------------------------------------------------
// inverse y pass: expand A_i, B_i to the three columns of row i
// ---------------------------------------------------------------------------
template <int L, class C>
__device__ __forceinline__ void inv_y_body(int cta, Grid g, int BK, C* __restrict__ S, const C* __restrict__ tw,
                                           const CgScalars* __restrict__ cg) {
  using R = typename RealOf<C>::type;
  C* smem = pass_smem<C>();
  const int Ln = L > 0 ? L : g.ny;
  const int QS = Ln + 1;
  const int np = 3 * BK;
  C* bufA = smem;
  C* bufB = smem + np * QS;
  C* twL = bufB + np * QS;
  stage_axis_twiddles<L, 1>(twL, tw, g);
  const int NC = (g.nzh + BK - 1) / BK;
  int b = cta;
  const int chunk = b % NC;
  b /= NC;
  const int i = b % 3;
  const int x = b / 3;
  const int kz0 = chunk * BK;
  const int valid = min(BK, g.nzh - kz0);
  const R rsy = to_real(g.sy, (C*)nullptr), rsz = to_real(g.sz, (C*)nullptr);
  for (int t = threadIdx.x; t < 2 * Ln * BK; t += blockDim.x) {
    const int kzl = t % BK, rest = t / BK;
    const int y = rest % Ln, h = rest / Ln;
    const int kz = kz0 + kzl;
    C v;
    czero(v);
    if (kz < g.nzh) v = S[(3 * i + h) * g.nspec + ((long long)x * Ln + y) * g.nzh + kz];
    if (h == 0) {
      bufA[(0 * BK + kzl) * QS + y] = v;
    } else {
      bufA[(1 * BK + kzl) * QS + y] = cscale(v, wave_real(wave_int(y, Ln), rsy));
      bufA[(2 * BK + kzl) * QS + y] = v;
    }
  }
  const C* Ry = fft_pencils_any<L, true, true>(bufA, bufB, PencilLayout{np, QS, 1, BK, valid}, twL, g.py);
  for (int t = threadIdx.x; t < Ln * BK; t += blockDim.x) {
    const int kzl = t % BK, y = t / BK;
    const int kz = kz0 + kzl;
    if (kz >= g.nzh) continue;
    const long long o = ((long long)x * Ln + y) * g.nzh + kz;
    S[(3 * i + 0) * g.nspec + o] = Ry[(0 * BK + kzl) * QS + y];
    S[(3 * i + 1) * g.nspec + o] = Ry[(1 * BK + kzl) * QS + y];
    S[(3 * i + 2) * g.nspec + o] = cscale(Ry[(2 * BK + kzl) * QS + y], wave_real(wave_int(kz, g.nz), rsz));
  }
}

}  // namespace fh
