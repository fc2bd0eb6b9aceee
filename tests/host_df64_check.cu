// Host check of the double-float arithmetic (df64.cuh) and butterflies
// (fft_df64.cuh) of the FH_ARITH_DF64 option, both host-and-device code,
// against long double, driven by tests/test_fft_tables_cpu.py. Prints one
// line "<case> <worst error / bound>" per case; every ratio must stay <= 1.
#include <cmath>
#include <cstdio>

#include "../paper_2408_03804_gb300/csrc/fft_df64.cuh"

using namespace fh;

namespace {

const long double kPi = 3.141592653589793238462643383279502884L;
const long double kEps = 1.0L / (1LL << 47);  // 2^-47: the double-float unit of one operation
unsigned g_seed = 2024u;

double urand() {
  g_seed = g_seed * 1664525u + 1013904223u;
  return (g_seed >> 8) * (2.0 / 16777216.0) - 1.0;
}

// a double-float value with a full low part, of magnitude about 2^e
df64 rand_df(int e) {
  const double x = std::ldexp(urand(), e) + std::ldexp(urand(), e - 30);
  return to_df64(x);
}

long double val(df64 a) { return (long double)a.hi + (long double)a.lo; }

// dd_add: |error| <= 4 eps (|a| + |b|); dd_mul, dd_fma: |error| <= 4 eps |a b| (+ 4 eps |c|)
void check_scalar_ops() {
  long double add = 0, mul = 0, fma_ = 0;
  for (int i = 0; i < 200000; ++i) {
    const df64 a = rand_df((int)(urand() * 20)), b = rand_df((int)(urand() * 20)), c = rand_df((int)(urand() * 20));
    const long double A = val(a), B = val(b), C = val(c);
    add = fmaxl(add, fabsl(val(dd_add(a, b)) - (A + B)) / (4 * kEps * (fabsl(A) + fabsl(B))));
    mul = fmaxl(mul, fabsl(val(dd_mul(a, b)) - A * B) / (4 * kEps * fabsl(A * B)));
    fma_ = fmaxl(fma_, fabsl(val(dd_fma(a, b, c)) - (A * B + C)) / (4 * kEps * (fabsl(A * B) + fabsl(C))));
  }
  printf("dd_add %.3Le\ndd_mul %.3Le\ndd_fma %.3Le\n", add, mul, fma_);
}

dfc rand_c() { return dfc{rand_df(0), rand_df(0)}; }

// untwiddled R-point butterflies: |error| <= 4 eps R max(|re| + |im|) of the inputs (normwise)
template <int R, bool INV>
void check_dft() {
  long double worst = 0;
  for (int rep = 0; rep < 2000; ++rep) {
    dfc v[R];
    long double xr[R], xi[R], norm = 0;
    for (int r = 0; r < R; ++r) {
      v[r] = rand_c();
      xr[r] = val(v[r].re);
      xi[r] = val(v[r].im);
      norm = fmaxl(norm, fabsl(xr[r]) + fabsl(xi[r]));
    }
    dft_r<R, INV>(v);
    const long double sg = INV ? 1.0L : -1.0L;
    for (int s = 0; s < R; ++s) {
      long double re = 0, im = 0;
      for (int r = 0; r < R; ++r) {
        const long double a = sg * 2 * kPi * (long double)(r * s % R) / R;
        re += xr[r] * cosl(a) - xi[r] * sinl(a);
        im += xr[r] * sinl(a) + xi[r] * cosl(a);
      }
      const long double err = fmaxl(fabsl(val(v[s].re) - re), fabsl(val(v[s].im) - im));
      worst = fmaxl(worst, err / (4 * kEps * R * norm));
    }
  }
  printf("dfc_dft%d_%s %.3Le\n", R, INV ? "inv" : "fwd", worst);
}

// the twiddle products of the twiddled stages, w from an FP64 root split into double-float
void check_twiddle_products() {
  long double worst = 0;
  for (int L : {8, 48, 128, 192, 256}) {
    for (int m = 0; m < L; ++m) {
      const long double a = 2 * kPi * m / L;
      const dfc w{to_df64((double)cosl(a)), to_df64((double)-sinl(a))};
      const dfc x = rand_c();
      const long double xr = val(x.re), xi = val(x.im), c = cosl(a), s = -sinl(a);
      const dfc p = cmul(x, w), q = cmulc(x, w);
      // w carries the FP64 rounding of cos and sin (2^-53) besides the products' own error
      const long double bound = 8 * kEps * (fabsl(xr) + fabsl(xi));
      worst = fmaxl(worst, fabsl(val(p.re) - (xr * c - xi * s)) / bound);
      worst = fmaxl(worst, fabsl(val(p.im) - (xr * s + xi * c)) / bound);
      worst = fmaxl(worst, fabsl(val(q.re) - (xr * c + xi * s)) / bound);
      worst = fmaxl(worst, fabsl(val(q.im) - (xi * c - xr * s)) / bound);
    }
  }
  printf("dfc_twiddle_products %.3Le\n", worst);
}

}  // namespace

int main() {
  check_scalar_ops();
  check_dft<2, false>(), check_dft<2, true>();
  check_dft<3, false>(), check_dft<3, true>();
  check_dft<4, false>(), check_dft<4, true>();
  check_dft<8, false>(), check_dft<8, true>();
  check_dft<16, false>(), check_dft<16, true>();
  check_twiddle_products();
  return 0;
}
