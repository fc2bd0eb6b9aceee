// Host check of the FP64 FFT butterflies of fft_core.cuh (they are
// host-and-device code) against a direct DFT in long double, driven by
// tests/test_fft_tables_cpu.py. Reads the library's twiddle tables (written
// by the test from fh_twiddle_tables: 2 T complex entries, T given on the
// command line) and prints one line "<case> <max error / max |output|>" per
// case.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_2408_03804_gb300/csrc/fft_core.cuh"

using namespace fh;

namespace {

const long double kPi = 3.141592653589793238462643383279502884L;
std::vector<double2> g_tab;
int g_total = 0;
unsigned g_seed = 12345u;

double urand() {
  g_seed = g_seed * 1664525u + 1013904223u;
  return (g_seed >> 8) * (2.0 / 16777216.0) - 1.0;
}

// Y_s = sum_r v_r omega^r w_R^(r s), omega = w_L^(m1) (conjugates for the inverse)
void direct(const double2* v, double2* y, int R, int L, int m1, bool inv) {
  const long double sg = inv ? 1.0L : -1.0L;
  for (int s = 0; s < R; ++s) {
    long double re = 0, im = 0;
    for (int r = 0; r < R; ++r) {
      const long double a = sg * 2 * kPi * ((long double)r * m1 / L + (long double)r * s / R);
      re += v[r].x * cosl(a) - v[r].y * sinl(a);
      im += v[r].x * sinl(a) + v[r].y * cosl(a);
    }
    y[s] = make_double2((double)re, (double)im);
  }
}

double rel_err(const double2* a, const double2* b, int n) {
  double e = 0, m = 0;
  for (int i = 0; i < n; ++i) {
    e = fmax(e, fmax(fabs(a[i].x - b[i].x), fabs(a[i].y - b[i].y)));
    m = fmax(m, fmax(fabs(b[i].x), fabs(b[i].y)));
  }
  return m > 0 ? e / m : e;
}

const double2* tangent_table(int L) { return g_tab.data() + g_total + twiddle_offset(L); }

// a twiddled radix-2^P stage of length L, every twiddle index m1 < L / R
template <int L, int R, bool INV>
void check_pow2() {
  double worst = 0;
  for (int m1 = 0; m1 < L / R; ++m1) {
    double2 v[R], y[R];
    for (int r = 0; r < R; ++r) v[r] = make_double2(urand(), urand());
    direct(v, y, R, L, m1, INV);
    dft_pow2_twiddled<L, R, INV>(v, tangent_table(L), m1);
    worst = fmax(worst, rel_err(v, y, R));
  }
  printf("radix%d_L%d_%s %.3e\n", R, L, INV ? "inv" : "fwd", worst);
}

// a twiddled radix-3 stage: two products in the tangent form, then the radix-3 butterfly
template <int L, bool INV>
void check_r3() {
  double worst = 0;
  for (int m1 = 0; m1 < L / 3; ++m1) {
    double2 v[3], y[3];
    for (int r = 0; r < 3; ++r) v[r] = make_double2(urand(), urand());
    direct(v, y, 3, L, m1, INV);
    v[1] = mul_tan(v[1], tan_twiddle<L, INV>(tangent_table(L), m1));
    v[2] = mul_tan(v[2], tan_twiddle<L, INV>(tangent_table(L), 2 * m1));
    dft3<INV>(v);
    worst = fmax(worst, rel_err(v, y, 3));
  }
  printf("radix3_L%d_%s %.3e\n", L, INV ? "inv" : "fwd", worst);
}

template <int R, bool INV>
void check_untwiddled() {
  double worst = 0;
  for (int rep = 0; rep < 64; ++rep) {
    double2 v[R], y[R];
    for (int r = 0; r < R; ++r) v[r] = make_double2(urand(), urand());
    direct(v, y, R, R, 0, INV);
    dft_r<R, INV>(v);
    worst = fmax(worst, rel_err(v, y, R));
  }
  printf("dft%d_%s %.3e\n", R, INV ? "inv" : "fwd", worst);
}

// the pair steps of the real-to-complex transform along z (NZ = 2M) against
// their definition with w = w_NZ^k from the (cos, -sin) table:
// unpack (e + t, conj(e - t)), t = -i w o; pack (a + u, conj(a - u)), u = i conj(w) b
template <int NZ>
void check_pairs() {
  double worst = 0;
  for (int k = 0; k <= NZ / 4; ++k) {
    const double2 e = make_double2(urand(), urand()), o = make_double2(urand(), urand());
    double2 got[4];
    unpack_pair_tan(e, o, tan_twiddle<NZ, false>(tangent_table(NZ), k), got[0], got[1]);
    pack_pair_tan(e, o, tan_twiddle<NZ, true>(tangent_table(NZ), k), got[2], got[3]);
    const long double a = 2 * kPi * k / NZ, c = cosl(a), s = sinl(a);
    // w o with w = c - i s; t = -i w o
    const long double wr = c * o.x + s * o.y, wi = c * o.y - s * o.x;
    const long double tr = wi, ti = -wr;
    // conj(w) b = (c + i s) o; u = i conj(w) b
    const long double vr = c * o.x - s * o.y, vi = c * o.y + s * o.x;
    const long double ur = -vi, ui = vr;
    const double2 ref[4] = {make_double2((double)(e.x + tr), (double)(e.y + ti)),
                            make_double2((double)(e.x - tr), (double)-(e.y - ti)),
                            make_double2((double)(e.x + ur), (double)(e.y + ui)),
                            make_double2((double)(e.x - ur), (double)-(e.y - ui))};
    worst = fmax(worst, rel_err(got, ref, 4));
  }
  printf("pairs_NZ%d %.3e\n", NZ, worst);
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s tables.bin T\n", argv[0]);
    return 2;
  }
  g_total = atoi(argv[2]);
  if (g_total != kTwiddleTotal) {
    fprintf(stderr, "table length %d, expected %d\n", g_total, kTwiddleTotal);
    return 3;
  }
  g_tab.resize(2 * g_total);
  FILE* f = fopen(argv[1], "rb");
  if (!f || fread(g_tab.data(), sizeof(double2), g_tab.size(), f) != g_tab.size()) {
    fprintf(stderr, "cannot read %s\n", argv[1]);
    return 4;
  }
  fclose(f);
  // the twiddled stages of the compile-time plans (32 = 8x4, 64 = 8x8, 128 = 16x8,
  // 256 = 16x4x4, 96 = 8x4x3, 192 = 16x4x3, 24 = 8x3, 48 = 16x3, 12 = 4x3, 6 = 2x3)
  check_pow2<32, 4, false>(), check_pow2<32, 4, true>();
  check_pow2<64, 8, false>(), check_pow2<64, 8, true>();
  check_pow2<128, 8, false>(), check_pow2<128, 8, true>();
  check_pow2<256, 4, false>(), check_pow2<256, 4, true>();
  check_pow2<256, 16, false>(), check_pow2<256, 16, true>();
  check_pow2<96, 4, false>(), check_pow2<96, 4, true>();
  check_pow2<192, 4, false>(), check_pow2<192, 4, true>();
  check_pow2<16, 2, false>(), check_pow2<16, 2, true>();
  check_r3<6, false>(), check_r3<6, true>();
  check_r3<12, false>(), check_r3<12, true>();
  check_r3<24, false>(), check_r3<24, true>();
  check_r3<48, false>(), check_r3<48, true>();
  check_r3<96, false>(), check_r3<96, true>();
  check_r3<192, false>(), check_r3<192, true>();
  check_untwiddled<2, false>(), check_untwiddled<2, true>();
  check_untwiddled<3, false>(), check_untwiddled<3, true>();
  check_untwiddled<4, false>(), check_untwiddled<4, true>();
  check_untwiddled<8, false>(), check_untwiddled<8, true>();
  check_untwiddled<16, false>(), check_untwiddled<16, true>();
  check_pairs<2>(), check_pairs<4>(), check_pairs<6>(), check_pairs<8>(), check_pairs<12>(), check_pairs<16>();
  check_pairs<24>(), check_pairs<32>(), check_pairs<48>(), check_pairs<64>(), check_pairs<96>();
  check_pairs<128>(), check_pairs<192>(), check_pairs<256>();
  return 0;
}
