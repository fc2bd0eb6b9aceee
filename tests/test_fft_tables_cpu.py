"""The FFT twiddle tables and the FP64 butterflies of the transforms of Eq. 1, on the host.

The library's tables (fh_twiddle_tables, no device needed) hold every root
w_L^m = exp(-2 pi i m / L) of the compile-time plans twice: as (cos, -sin) and
in the tangent form (rho, tau) of the FP64 stages, w = (-i)^qr rho (1 + i tau)
with qr the nearest quarter turn. The butterflies themselves are
host-and-device code: tests/host_fft_check.cu compiles them for the host and
compares every twiddled stage, the radix-16 butterfly and the real-to-complex
pair steps with a direct DFT in long double; tests/host_df64_check.cu does the
same for the double-float arithmetic and butterflies of the FH_ARITH_DF64
option against the error bounds of df64.cuh.
"""

import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2408_03804_gb300 import _binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LENGTHS = [1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256]


@pytest.fixture(scope="module")
def tables():
    build.build()
    t = _binding.fh_twiddle_tables()
    total = sum(LENGTHS)
    assert t.shape == (2 * total,)
    return t, total


PI_LD = np.longdouble("3.14159265358979323846264338327950288")


def _roots(L):
    """exp(-2 pi i m / L), m < L, in extended precision, rounded to float64 parts."""
    a = 2 * PI_LD * np.arange(L, dtype=np.longdouble) / np.longdouble(L)
    return np.cos(a).astype(np.float64) - 1j * np.sin(a).astype(np.float64)


def _offsets():
    off, o = {}, 0
    for L in LENGTHS:
        off[L] = o
        o += L
    return off


def test_cos_sin_tables_are_the_roots_of_unity(tables):
    t, _ = tables
    off = _offsets()
    for L in LENGTHS:
        m = np.arange(L)
        w = t[off[L]:off[L] + L]
        ref = _roots(L)
        assert np.abs(w - ref).max() <= 1.2e-16, L
        quarter = (4 * m) % L == 0  # exact at multiples of pi/2
        np.testing.assert_array_equal(w[quarter], np.round(ref[quarter].real) + 1j * np.round(ref[quarter].imag))


def test_tangent_form_gives_each_root(tables):
    t, total = tables
    off = _offsets()
    for L in LENGTHS:
        m = np.arange(L)
        e = t[total + off[L]:total + off[L] + L]
        rho, tau = e.real, e.imag
        qr = (8 * m + L) // (2 * L)
        assert np.all(np.abs(tau) <= 1.0), L
        assert np.all(rho >= np.cos(np.pi / 4) - 1e-16) and np.all(rho <= 1.0), L
        w = (-1j) ** qr * rho * (1 + 1j * tau)
        assert np.abs(w - _roots(L)).max() <= 4e-16, L
        exact = (4 * m) % L == 0
        np.testing.assert_array_equal(rho[exact], 1.0)
        np.testing.assert_array_equal(tau[exact], 0.0)


def _host_program(name, tmp_path):
    """Compile tests/<name>.cu (host code only) with nvcc; returns the executable."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = tmp_path / name
    src = os.path.join(ROOT, "tests", name + ".cu")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-o", str(exe), src],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


def _results(stdout):
    out = {}
    for line in stdout.splitlines():
        name, err = line.rsplit(" ", 1)
        out[name] = float(err)
    return out


def test_fp64_butterflies_match_a_direct_dft_on_the_host(tables, tmp_path):
    exe = _host_program("host_fft_check", tmp_path)
    t, total = tables
    table_file = tmp_path / "tables.bin"
    np.stack([t.real, t.imag], axis=1).astype(np.float64).tofile(table_file)
    r = subprocess.run([str(exe), str(table_file), str(total)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    worst = _results(r.stdout)
    assert len(worst) >= 40
    # relative to the largest output; rounding of a few operations per point
    bad = {k: v for k, v in worst.items() if not v <= 1e-15}
    assert not bad, bad


def test_double_float_arithmetic_and_butterflies_within_their_bounds_on_the_host(tmp_path):
    exe = _host_program("host_df64_check", tmp_path)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    ratio = _results(r.stdout)
    # each line: worst error / its bound (dd_add 4 eps (|a| + |b|), products 4 eps |a b|, an R-point
    # butterfly 4 eps R max(|re| + |im|), eps = 2^-47)
    assert {"dd_add", "dd_mul", "dd_fma", "dfc_dft16_fwd", "dfc_dft16_inv", "dfc_twiddle_products"} <= set(ratio)
    bad = {k: v for k, v in ratio.items() if not v <= 1.0}
    assert not bad, bad
