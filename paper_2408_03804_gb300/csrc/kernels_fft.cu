// Kernels and launches of the five FP64 passes of the projection G (the pass
// bodies and the description of the passes are in passes.cuh), the
// batched-cell variants, and the host side of the transforms: twiddle
// tables, run-time plans and tiles.
#include <cmath>
#include <cstdio>
#include <vector>

#include "fft_core.cuh"
#include "fh_kernels.h"
#include "passes.cuh"

namespace fh {

// ---------------------------------------------------------------------------
// kernels: one cell (blockIdx.x = CTA of the pass) ...
// ---------------------------------------------------------------------------
template <int M, int MODE>
__global__ void __launch_bounds__(kThreads) k_fwd_z(Grid g, int LB, const double* __restrict__ src,
                                                   double* __restrict__ p, double* __restrict__ x,
                                                   const double* __restrict__ K, const CgScalars* __restrict__ cg,
                                                   double2* __restrict__ S, const double2* __restrict__ tw) {
  if (cg_done(cg)) return;
  fwd_z_body<M, MODE>(blockIdx.x, g, LB, src, p, x, K, cg, S, tw);
}
template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_fwd_y(Grid g, int BK, double2* __restrict__ S,
                                                      const double2* __restrict__ tw, const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  fwd_y_body<L>(blockIdx.x, g, BK, S, tw, cg);
}
template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_x_ghat(Grid g, int BK, double2* __restrict__ S,
                                                       const double2* __restrict__ tw, double scale,
                                                       const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  x_ghat_body<L>(blockIdx.x, g, BK, S, tw, scale, cg);
}
template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_inv_y(Grid g, int BK, double2* __restrict__ S,
                                                      const double2* __restrict__ tw, const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  inv_y_body<L>(blockIdx.x, g, BK, S, tw, cg);
}
template <int M, int MODE>
__global__ void __launch_bounds__(kThreads) k_inv_z(Grid g, int LB, const double2* __restrict__ S,
                                                   double* __restrict__ out, const double* __restrict__ p,
                                                   double* __restrict__ partials, const double2* __restrict__ tw,
                                                   const CgScalars* __restrict__ cg) {
  if (cg_done(cg)) return;
  inv_z_body<M, MODE>(blockIdx.x, g, LB, S, out, p, partials, tw, cg);
}

// ... and a group of cells of one grid shape (blockIdx.y = cell); a cell whose
// stop flag is set skips the launch
template <int M, int MODE>
__global__ void __launch_bounds__(kThreads) k_fwd_z_b(Grid g, int LB, const CellView* __restrict__ cells,
                                                     const double2* __restrict__ tw) {
  const CellView& c = cells[blockIdx.y];
  if (*c.stop) return;
  fwd_z_body<M, MODE>(blockIdx.x, g, LB, c.src, c.p, c.x, c.K, c.cg, c.S, tw);
}
template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_fwd_y_b(Grid g, int BK, const CellView* __restrict__ cells,
                                                        const double2* __restrict__ tw) {
  const CellView& c = cells[blockIdx.y];
  if (*c.stop) return;
  fwd_y_body<L>(blockIdx.x, g, BK, c.S, tw, c.cg);
}
template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_x_ghat_b(Grid g, int BK, const CellView* __restrict__ cells,
                                                         const double2* __restrict__ tw, double scale) {
  const CellView& c = cells[blockIdx.y];
  if (*c.stop) return;
  x_ghat_body<L>(blockIdx.x, g, BK, c.S, tw, scale, c.cg);
}
template <int L>
__global__ void __launch_bounds__(kThreads, 3) k_inv_y_b(Grid g, int BK, const CellView* __restrict__ cells,
                                                        const double2* __restrict__ tw) {
  const CellView& c = cells[blockIdx.y];
  if (*c.stop) return;
  inv_y_body<L>(blockIdx.x, g, BK, c.S, tw, c.cg);
}
template <int M, int MODE>
__global__ void __launch_bounds__(kThreads) k_inv_z_b(Grid g, int LB, const CellView* __restrict__ cells,
                                                     const double2* __restrict__ tw) {
  const CellView& c = cells[blockIdx.y];
  if (*c.stop) return;
  inv_z_body<M, MODE>(blockIdx.x, g, LB, c.S, c.out, c.p, c.partials, tw, c.cg);
}

// ---------------------------------------------------------------------------
// host side: twiddle tables, tiling, dispatch on the compile-time lengths
// ---------------------------------------------------------------------------
void fill_twiddle_table(double2* t) {
  for (int i = 0; i < kTwiddleTables; ++i) t[i] = make_double2(0.0, 0.0);
  for (int L = 1; L <= kMaxN; ++L) {
    if (!fft_length_ok(L)) continue;
    fill_twiddles_of_length(t + twiddle_offset(L), L);
    fill_tangent_twiddles_of_length(t + kTwiddleTotal + twiddle_offset(L), L);
  }
}

// w_L^m = i^Q rho (1 + i tau) with qr the nearest quarter turn of 2 pi m / L
// (halves rounded up), Q = -qr mod 4 (computed again by the kernels from m and
// L), phi = 2 pi m / L - qr pi / 2 in [-pi/4, pi/4), rho = cos phi,
// tau = -tan phi; entry m holds (rho, tau)
void fill_tangent_twiddles_of_length(double2* t, int L) {
  const long double half_pi = 1.570796326794896619231321691639751442L;
  for (int m = 0; m < L; ++m) {
    const int qr = (8 * m + L) / (2 * L);
    const int n4 = 4 * m - qr * L;  // phi = (pi / 2) n4 / L, |n4| <= L / 2
    double rho, tau;
    if (n4 == 0) {
      rho = 1.0;
      tau = 0.0;
    } else if (2 * n4 == L || 2 * n4 == -L) {
      rho = (double)sqrtl(0.5L);
      tau = n4 > 0 ? -1.0 : 1.0;
    } else {
      const long double phi = half_pi * (long double)n4 / (long double)L;
      rho = (double)cosl(phi);
      tau = (double)-tanl(phi);
    }
    t[m] = make_double2(rho, tau);
  }
}

void fill_twiddles_of_length(double2* t, int L) {
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int m = 0; m < L; ++m) {
    double c, sn;
    if ((4 * m) % L == 0) {
      const int q = (4 * m) / L;
      c = (q == 0) ? 1.0 : (q == 2) ? -1.0 : 0.0;
      sn = (q == 1) ? -1.0 : (q == 3) ? 1.0 : 0.0;
    } else {
      const long double a = two_pi * (long double)m / (long double)L;
      c = (double)cosl(a);
      sn = (double)-sinl(a);
    }
    t[m] = make_double2(c, sn);
  }
}

// stage radices of a length: powers of two as radix-16 stages and one radix-8/4/2
// stage, then radix-3 stages, then the other prime factors in increasing order
static int plan_radices(int L, int* r) {
  int n = 0, rest = L, twos = 0;
  while (rest % 2 == 0) {
    rest /= 2;
    ++twos;
  }
  while (twos >= 4) {
    r[n++] = 16;
    twos -= 4;
  }
  if (twos > 0) r[n++] = 1 << twos;
  while (rest % 3 == 0) {
    r[n++] = 3;
    rest /= 3;
  }
  for (int f = 5; rest > 1; f += 2) {
    while (rest % f == 0) {
      r[n++] = f;
      rest /= f;
    }
  }
  return n;
}

static bool is_prime(int L) {
  if (L < 2) return false;
  for (int f = 2; f * f <= L; ++f)
    if (L % f == 0) return false;
  return true;
}

// primes from this length on use Rader's algorithm; shorter ones a direct stage
constexpr int kRaderMin = 37;

FftPlan make_fft_plan(int L, int tw_off) {
  FftPlan p{};
  if (fft_length_ok(L)) return p;  // compile-time plan
  p.L = L;
  p.tw_off = tw_off;
  if (L >= kRaderMin && is_prime(L)) {
    p.rader = 1;
    p.tw_len = 4 * (L - 1);
    p.in_n = plan_radices(L - 1, p.in_r);
  } else {
    p.tw_len = L;
    p.n = plan_radices(L, p.r);
  }
  return p;
}

static long long pow_mod(long long b, long long e, long long m) {
  long long r = 1 % m;
  b %= m;
  while (e > 0) {
    if (e & 1) r = r * b % m;
    b = b * b % m;
    e >>= 1;
  }
  return r;
}

// smallest primitive root of the prime L
static int primitive_root(int L) {
  int f[16], nf = 0, m = L - 1;
  for (int q = 2; q * q <= m; ++q)
    if (m % q == 0) {
      f[nf++] = q;
      while (m % q == 0) m /= q;
    }
  if (m > 1) f[nf++] = m;
  for (int g = 2; g < L; ++g) {
    bool ok = true;
    for (int i = 0; i < nf && ok; ++i) ok = pow_mod(g, (L - 1) / f[i], L) != 1;
    if (ok) return g;
  }
  return 1;
}

void fill_plan_tables(double2* t, const FftPlan& p) {
  if (!p.rader) {
    fill_twiddles_of_length(t, p.L);
    return;
  }
  const int L = p.L, M = L - 1;
  const long double two_pi = 6.283185307179586476925286766559005768L;
  fill_twiddles_of_length(t, M);
  const long long g = primitive_root(L), ginv = pow_mod(g, L - 2, L);
  // b_s = exp(-2 pi i g^-s / L); Bhat_k = (1/M) sum_s b_s exp(-2 pi i s k / M) (and with conj b)
  std::vector<long double> br(M), bi(M);
  long long e = 1;
  for (int s = 0; s < M; ++s) {
    const long double a = two_pi * (long double)e / (long double)L;
    br[s] = cosl(a);
    bi[s] = -sinl(a);
    e = e * ginv % L;
  }
  for (int k = 0; k < M; ++k) {
    long double fr = 0, fi = 0, ir = 0, ii = 0;
    for (int s = 0; s < M; ++s) {
      const long double a = two_pi * (long double)(((long long)s * k) % M) / (long double)M;
      const long double c = cosl(a), sn = -sinl(a);
      fr += br[s] * c - bi[s] * sn;
      fi += br[s] * sn + bi[s] * c;
      ir += br[s] * c + bi[s] * sn;  // conj(b) times the same root
      ii += br[s] * sn - bi[s] * c;
    }
    t[M + k] = make_double2((double)(fr / M), (double)(fi / M));
    t[2 * M + k] = make_double2((double)(ir / M), (double)(ii / M));
  }
  long long gr = 1, gi = 1;
  for (int r = 0; r < M; ++r) {
    t[3 * M + r] = make_double2((double)gr, (double)gi);
    gr = gr * g % L;
    gi = gi * ginv % L;
  }
}

Tiling choose_tiling(const Grid& g, long long min_ctas) {
  Tiling t;
  const long long lines = (long long)g.nx * g.ny;
  // z lines per CTA: the largest divisor of nx*ny not above 512 / nz that
  // leaves at least min_ctas CTAs (one line per CTA if none does; a plane
  // cell keeps its full tile: one voxel per line)
  int lb = 512 / g.nz;
  if (lb < 1) lb = 1;
  if (lb > lines) lb = (int)lines;
  while (lines % lb) --lb;
  while (g.nz > 1 && lb > 1 && lines / lb < min_ctas) {
    --lb;
    while (lines % lb) --lb;
  }
  t.lines_z = lb;
  // the double-float z passes on long z lines: half the lines per CTA (half
  // the shared memory, more resident CTAs to stream the tangent); measured
  // faster at 128^3 (4 -> 2 lines), slower at one line per CTA (256^3) and on
  // the short lines of the batched grids, which keep lines_z
  int ld = lb;
  if (g.nz >= 128 && lb >= 4) {
    ld = lb / 2;
    while (lines % ld) --ld;
  }
  t.lines_z_df = ld;
  // kz columns per CTA of the y and x passes, likewise
  auto chunks = [&](int bk) { return (long long)((g.nzh + bk - 1) / bk); };
  int by = 512 / g.ny;
  if (by < 1) by = 1;
  if (by > g.nzh) by = g.nzh;
  while (by > 1 && 3LL * g.nx * chunks(by) < min_ctas) --by;
  t.bk_y = by;
  int bx = 256 / g.nx;
  if (bx < 1) bx = 1;
  if (bx > g.nzh) bx = g.nzh;
  while (bx > 1 && (long long)g.ny * chunks(bx) < min_ctas) --bx;
  t.bk_x = bx;
  return t;
}

size_t z_pass_smem(const Grid& g, const Tiling& t) {
  if (g.nz == 1) return 0;  // identity along z: no staging
  const int M = g.nz / 2;
  return ((size_t)9 * t.lines_z * g.nz + M + M / 2 + 1) * sizeof(double2);
}
long long z_pass_ctas(const Grid& g, const Tiling& t) { return (long long)g.nx * g.ny / t.lines_z; }
size_t y_smem(int L, int bk, int fields) {
  return ((size_t)2 * fields * bk * (L + 1) + L) * sizeof(double2);
}
// shared memory of a pass along an axis with a run-time plan (its tables may exceed L entries)
size_t y_smem_rt(const FftPlan& p, int bk, int fields) {
  return ((size_t)2 * fields * bk * (p.L + 1) + p.tw_len) * sizeof(double2);
}

template <class Kern>
static cudaError_t allow_smem(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t setup_fft_kernels(const Grid& g, const Tiling& t) {
  cudaError_t e = cudaSuccess;
  if (g.nz == 1) {
    // plane cell: the z passes need no shared memory, the y and x passes are kernels_plane.cu's
    return setup_plane_kernels(g);
  }
  const size_t zs = z_pass_smem(g, t);
  const int M = g.nz / 2;
#define ZCASE(V)                                                      \
  case V:                                                             \
    if ((e = allow_smem(k_fwd_z<V, kZDirect>, zs))) return e;         \
    if ((e = allow_smem(k_fwd_z<V, kZKApply>, zs))) return e;         \
    if ((e = allow_smem(k_fwd_z<V, kZCg>, zs))) return e;             \
    if ((e = allow_smem(k_fwd_z<V, kZCgFirst>, zs))) return e;        \
    if ((e = allow_smem(k_inv_z<V, kIZOut>, zs))) return e;           \
    if ((e = allow_smem(k_inv_z<V, kIZDot>, zs))) return e;           \
    if ((e = allow_smem(k_inv_z<V, kIZRhs>, zs))) return e;           \
    if ((e = allow_smem(k_fwd_z_b<V, kZDirect>, zs))) return e;       \
    if ((e = allow_smem(k_fwd_z_b<V, kZCg>, zs))) return e;           \
    if ((e = allow_smem(k_fwd_z_b<V, kZCgFirst>, zs))) return e;      \
    if ((e = allow_smem(k_inv_z_b<V, kIZDot>, zs))) return e;         \
    if ((e = allow_smem(k_inv_z_b<V, kIZRhs>, zs))) return e;         \
    break;
  FH_SWITCH_HALF(M, ZCASE)
#undef ZCASE
#define YCASE(V)                                                           \
  case V:                                                                  \
    if ((e = allow_smem(k_fwd_y<V>, y_smem(V, t.bk_y, 3)))) return e;      \
    if ((e = allow_smem(k_inv_y<V>, y_smem(V, t.bk_y, 3)))) return e;      \
    if ((e = allow_smem(k_fwd_y_b<V>, y_smem(V, t.bk_y, 3)))) return e;    \
    if ((e = allow_smem(k_inv_y_b<V>, y_smem(V, t.bk_y, 3)))) return e;    \
    break;
  if (g.py.L) {
    if ((e = allow_smem(k_fwd_y<0>, y_smem_rt(g.py, t.bk_y, 3)))) return e;
    if ((e = allow_smem(k_inv_y<0>, y_smem_rt(g.py, t.bk_y, 3)))) return e;
  } else {
    FH_SWITCH_LEN(g.ny, YCASE)
  }
#undef YCASE
#define XCASE(V)                                                           \
  case V:                                                                  \
    if ((e = allow_smem(k_x_ghat<V>, y_smem(V, t.bk_x, 6)))) return e;     \
    if ((e = allow_smem(k_x_ghat_b<V>, y_smem(V, t.bk_x, 6)))) return e;   \
    break;
  if (g.px.L) {
    if ((e = allow_smem(k_x_ghat<0>, y_smem_rt(g.px, t.bk_x, 6)))) return e;
  } else {
    FH_SWITCH_LEN(g.nx, XCASE)
  }
#undef XCASE
  // the double-float kernels take the same tiles and shared memory
  return setup_df64_kernels(g, t);
}

cudaError_t launch_fwd_z(const Grid& g, const Tiling& t, int mode, const double* src, double* p, double* x,
                         const double* K, const CgScalars* cg, double2* S, const double2* tw, cudaStream_t s) {
  const size_t smem = z_pass_smem(g, t);
  const unsigned grid = (unsigned)z_pass_ctas(g, t);
  const int M = g.nz / 2;
#define ZL(V)                                                                                              \
  case V:                                                                                                  \
    switch (mode) {                                                                                        \
      case kZDirect: k_fwd_z<V, kZDirect><<<grid, kThreads, smem, s>>>(g, t.lines_z, src, p, x, K, cg, S, tw); break; \
      case kZKApply: k_fwd_z<V, kZKApply><<<grid, kThreads, smem, s>>>(g, t.lines_z, src, p, x, K, cg, S, tw); break; \
      case kZCg: k_fwd_z<V, kZCg><<<grid, kThreads, smem, s>>>(g, t.lines_z, src, p, x, K, cg, S, tw); break;         \
      case kZCgFirst: k_fwd_z<V, kZCgFirst><<<grid, kThreads, smem, s>>>(g, t.lines_z, src, p, x, K, cg, S, tw); break; \
      default: return cudaErrorInvalidValue;                                                               \
    }                                                                                                      \
    break;
  FH_SWITCH_HALF(M, ZL)
#undef ZL
  return cudaGetLastError();
}

cudaError_t launch_fwd_y(const Grid& g, const Tiling& t, double2* S, const double2* tw, const CgScalars* cg,
                         cudaStream_t s) {
  if (g.nz == 1) return launch_plane_fwd_y(g, S, tw, cg, s);
  const int NC = (g.nzh + t.bk_y - 1) / t.bk_y;
  const unsigned grid = (unsigned)((long long)g.nx * 3 * NC);
#define YL(V)                                                                               \
  case V:                                                                                   \
    k_fwd_y<V><<<grid, kThreads, y_smem(V, t.bk_y, 3), s>>>(g, t.bk_y, S, tw, cg);          \
    break;
  if (g.py.L) k_fwd_y<0><<<grid, kThreads, y_smem_rt(g.py, t.bk_y, 3), s>>>(g, t.bk_y, S, tw, cg);
  else FH_SWITCH_LEN(g.ny, YL)
#undef YL
  return cudaGetLastError();
}

cudaError_t launch_x_ghat(const Grid& g, const Tiling& t, double2* S, const double2* tw, double scale,
                          const CgScalars* cg, cudaStream_t s) {
  if (g.nz == 1) return launch_plane_x_ghat(g, S, tw, scale, cg, s);
  const int NC = (g.nzh + t.bk_x - 1) / t.bk_x;
  const unsigned grid = (unsigned)((long long)g.ny * NC);
#define XL(V)                                                                                      \
  case V:                                                                                          \
    k_x_ghat<V><<<grid, kThreads, y_smem(V, t.bk_x, 6), s>>>(g, t.bk_x, S, tw, scale, cg);         \
    break;
  if (g.px.L) k_x_ghat<0><<<grid, kThreads, y_smem_rt(g.px, t.bk_x, 6), s>>>(g, t.bk_x, S, tw, scale, cg);
  else FH_SWITCH_LEN(g.nx, XL)
#undef XL
  return cudaGetLastError();
}

cudaError_t launch_inv_y(const Grid& g, const Tiling& t, double2* S, const double2* tw, const CgScalars* cg,
                         cudaStream_t s) {
  if (g.nz == 1) return launch_plane_inv_y(g, S, tw, cg, s);
  const int NC = (g.nzh + t.bk_y - 1) / t.bk_y;
  const unsigned grid = (unsigned)((long long)g.nx * 3 * NC);
#define IYL(V)                                                                              \
  case V:                                                                                   \
    k_inv_y<V><<<grid, kThreads, y_smem(V, t.bk_y, 3), s>>>(g, t.bk_y, S, tw, cg);          \
    break;
  if (g.py.L) k_inv_y<0><<<grid, kThreads, y_smem_rt(g.py, t.bk_y, 3), s>>>(g, t.bk_y, S, tw, cg);
  else FH_SWITCH_LEN(g.ny, IYL)
#undef IYL
  return cudaGetLastError();
}

cudaError_t launch_inv_z(const Grid& g, const Tiling& t, int mode, const double2* S, double* out, const double* p,
                         double* partials, const double2* tw, const CgScalars* cg, cudaStream_t s) {
  const size_t smem = z_pass_smem(g, t);
  const unsigned grid = (unsigned)z_pass_ctas(g, t);
  const int M = g.nz / 2;
#define IZL(V)                                                                                                  \
  case V:                                                                                                       \
    switch (mode) {                                                                                             \
      case kIZOut: k_inv_z<V, kIZOut><<<grid, kThreads, smem, s>>>(g, t.lines_z, S, out, p, partials, tw, cg); break; \
      case kIZDot: k_inv_z<V, kIZDot><<<grid, kThreads, smem, s>>>(g, t.lines_z, S, out, p, partials, tw, cg); break; \
      case kIZRhs: k_inv_z<V, kIZRhs><<<grid, kThreads, smem, s>>>(g, t.lines_z, S, out, p, partials, tw, cg); break; \
      default: return cudaErrorInvalidValue;                                                                    \
    }                                                                                                           \
    break;
  FH_SWITCH_HALF(M, IZL)
#undef IZL
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// batched launches: one pass over every cell of a group of equal grids
// ---------------------------------------------------------------------------
cudaError_t launch_fwd_z_batch(const Grid& g, const Tiling& t, int mode, const CellView* cells, int n_cells,
                               const double2* tw, cudaStream_t s) {
  const size_t smem = z_pass_smem(g, t);
  const dim3 grid((unsigned)z_pass_ctas(g, t), (unsigned)n_cells);
  const int M = g.nz / 2;
#define ZB(V)                                                                                          \
  case V:                                                                                              \
    switch (mode) {                                                                                    \
      case kZDirect: k_fwd_z_b<V, kZDirect><<<grid, kThreads, smem, s>>>(g, t.lines_z, cells, tw); break; \
      case kZCg: k_fwd_z_b<V, kZCg><<<grid, kThreads, smem, s>>>(g, t.lines_z, cells, tw); break;         \
      case kZCgFirst: k_fwd_z_b<V, kZCgFirst><<<grid, kThreads, smem, s>>>(g, t.lines_z, cells, tw); break; \
      default: return cudaErrorInvalidValue;                                                           \
    }                                                                                                  \
    break;
  FH_SWITCH_HALF(M, ZB)
#undef ZB
  return cudaGetLastError();
}

cudaError_t launch_fwd_y_batch(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                               const double2* tw, cudaStream_t s) {
  const int NC = (g.nzh + t.bk_y - 1) / t.bk_y;
  const dim3 grid((unsigned)((long long)g.nx * 3 * NC), (unsigned)n_cells);
#define YB(V)                                                                         \
  case V:                                                                             \
    k_fwd_y_b<V><<<grid, kThreads, y_smem(V, t.bk_y, 3), s>>>(g, t.bk_y, cells, tw);  \
    break;
  FH_SWITCH_LEN(g.ny, YB)
#undef YB
  return cudaGetLastError();
}

cudaError_t launch_x_ghat_batch(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                                const double2* tw, double scale, cudaStream_t s) {
  const int NC = (g.nzh + t.bk_x - 1) / t.bk_x;
  const dim3 grid((unsigned)((long long)g.ny * NC), (unsigned)n_cells);
#define XB(V)                                                                                \
  case V:                                                                                    \
    k_x_ghat_b<V><<<grid, kThreads, y_smem(V, t.bk_x, 6), s>>>(g, t.bk_x, cells, tw, scale); \
    break;
  FH_SWITCH_LEN(g.nx, XB)
#undef XB
  return cudaGetLastError();
}

cudaError_t launch_inv_y_batch(const Grid& g, const Tiling& t, const CellView* cells, int n_cells,
                               const double2* tw, cudaStream_t s) {
  const int NC = (g.nzh + t.bk_y - 1) / t.bk_y;
  const dim3 grid((unsigned)((long long)g.nx * 3 * NC), (unsigned)n_cells);
#define IYB(V)                                                                        \
  case V:                                                                             \
    k_inv_y_b<V><<<grid, kThreads, y_smem(V, t.bk_y, 3), s>>>(g, t.bk_y, cells, tw);  \
    break;
  FH_SWITCH_LEN(g.ny, IYB)
#undef IYB
  return cudaGetLastError();
}

cudaError_t launch_inv_z_batch(const Grid& g, const Tiling& t, int mode, const CellView* cells, int n_cells,
                               const double2* tw, cudaStream_t s) {
  const size_t smem = z_pass_smem(g, t);
  const dim3 grid((unsigned)z_pass_ctas(g, t), (unsigned)n_cells);
  const int M = g.nz / 2;
#define IZB(V)                                                                                      \
  case V:                                                                                           \
    switch (mode) {                                                                                 \
      case kIZDot: k_inv_z_b<V, kIZDot><<<grid, kThreads, smem, s>>>(g, t.lines_z, cells, tw); break; \
      case kIZRhs: k_inv_z_b<V, kIZRhs><<<grid, kThreads, smem, s>>>(g, t.lines_z, cells, tw); break; \
      default: return cudaErrorInvalidValue;                                                        \
    }                                                                                               \
    break;
  FH_SWITCH_HALF(M, IZB)
#undef IZB
  return cudaGetLastError();
}

}  // namespace fh
