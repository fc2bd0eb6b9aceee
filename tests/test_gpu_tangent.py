"""Homogenized tangent and voxel sensitivities on the GPU (Section 3.3, Section 4.4.2).

* the 9x9 tangent of fft_homog_tangent against the oracle's linear solves
  (relative 1e-9 of the largest entry) for a neo-Hookean state and the 16^3
  linear elastic sphere, with major symmetry;
* sensitivities dCbar_ijkl/drho of fft_homog_sensitivity against the
  oracle's field (1e-8 max-relative) on a 32^3 SIMP density field;
* the 64^3 SIMP workload (rho in [0.01, 1], E = rho^3, nu = 0.3): the 6x6
  Voigt tangent and dCbar_1212/drho of every voxel, checked against central
  finite differences with step 1e-6 at 64 random voxels. Each perturbed solve
  starts from the converged unperturbed field, so CG resolves only the O(h)
  correction, to a tolerance relative to it; a cold solve would have to reach
  a relative accuracy of about 1e-14 in Cbar for a 1e-6 step to resolve a
  per-voxel sensitivity of order Cbar/N.
"""

import numpy as np
import pytest

from gpu_helpers import dev, field_maxrel, host, require_gpu
from oracle import homogenize, materials as omat, solver as osolver
from rve_inputs import random_spheres, shear_macro, simp_config, small_strain_config, two_phase_table

pytestmark = pytest.mark.gpu

TOL = 1e-9
VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def voigt(C9):
    return np.array([[C9[3 * i + j, 3 * k + l] for (k, l) in VOIGT] for (i, j) in VOIGT])


@pytest.fixture(scope="module")
def fh():
    require_gpu()
    import paper_2408_03804_gb300 as fh

    return fh


def test_tangent_matches_oracle_neo_hookean(fh):
    import torch

    shape = (8, 8, 16)
    phase = random_spheres(shape, seed=3, r_min=1.5, r_max=2.5)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.05, finite=True)
    ref_state = osolver.solve(phase, params, 1, Fbar, n_increments=2, newton_tol=1e-12)
    C_ref = homogenize.tangent(phase, params, 1, ref_state.F, cg_tol=1e-13)
    with fh.Context(*shape) as ctx:
        mat = fh.Material(1, phase, params)
        F = dev(ref_state.F)
        C = ctx.fft_homog_tangent(mat, F, options=fh.default_options(cg_tol=1e-13))
    assert np.abs(C - C_ref).max() < TOL * np.abs(C_ref).max()
    assert np.abs(C - C.T).max() < 1e-10 * np.abs(C).max()


def test_tangent_matches_oracle_small_strain_sphere(fh):
    phase, params, _ = small_strain_config(16)
    zero = np.zeros((9, 16, 16, 16))
    C_ref = homogenize.tangent(phase, params, 0, zero, cg_tol=1e-13)
    with fh.Context(16, 16, 16) as ctx:
        C = ctx.fft_homog_tangent(fh.Material(0, phase, params), dev(zero), options=fh.default_options(cg_tol=1e-13))
    assert np.abs(C - C_ref).max() < TOL * np.abs(C_ref).max()
    Cv = voigt(C)
    assert np.abs(Cv - Cv.T).max() < 1e-10 * np.abs(Cv).max()
    # cubic symmetry of a centred sphere in a cube
    np.testing.assert_allclose(np.diag(Cv)[:3], Cv[0, 0], rtol=1e-9)
    np.testing.assert_allclose(np.diag(Cv)[3:], Cv[3, 3], rtol=1e-9)


@pytest.mark.parametrize("ijkl", [(0, 1, 0, 1), (0, 0, 1, 1)])
def test_sensitivity_matches_oracle(fh, ijkl):
    import torch

    phase, params, rho, scale, dscale = simp_config(32, seed=1)
    i, j, k, l = ijkl
    ref = homogenize.sensitivity(phase, params, scale, dscale, 3 * i + j, 3 * k + l, cg_tol=1e-13)
    with fh.Context(32, 32, 32) as ctx:
        mat = fh.Material(0, phase, params, scale=scale)
        out = torch.empty((32, 32, 32), dtype=torch.float64, device="cuda")
        ctx.fft_homog_sensitivity(mat, ijkl, dev(dscale), out, options=fh.default_options(cg_tol=1e-13))
    assert field_maxrel(host(out)[None], ref[None]) < 1e-8


def test_simp_64_voigt_tangent_and_sensitivity_vs_finite_differences(fh):
    import torch

    n = 64
    phase, params, rho, scale, dscale = simp_config(n, seed=0)
    shape = (n, n, n)
    opts = fh.default_options(cg_tol=1e-13)
    with fh.Context(*shape) as ctx:
        mat = fh.Material(0, phase, params, scale=scale)
        C = ctx.fft_homog_tangent(mat, torch.zeros((9,) + shape, dtype=torch.float64, device="cuda"), options=opts)
        Cv = voigt(C)
        assert np.abs(Cv - Cv.T).max() < 1e-10 * np.abs(Cv).max()
        assert np.all(np.linalg.eigvalsh(0.5 * (Cv + Cv.T)) > 0)
        sens = torch.empty(shape, dtype=torch.float64, device="cuda")
        ctx.fft_homog_sensitivity(mat, (0, 1, 0, 1), dev(dscale), sens, options=opts)
        s = host(sens)
        # Euler's identity for a degree-one dependence on the modulus scale rho^3
        np.testing.assert_allclose((s * rho / 3.0).sum(), C[1, 1], rtol=1e-9)
        # central differences: Cbar_xyxy = Pbar_xy of a linear solve with Hbar = e_x (x) e_y,
        # each perturbed solve warm-started from the converged unperturbed field H0
        Hbar = np.zeros(9)
        Hbar[1] = 1.0
        H0 = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        ctx.fft_homog_solve(mat, Hbar, H0, options=fh.default_options(newton_tol=1e-12, cg_tol=1e-13))
        fd_opts = fh.default_options(newton_tol=1e-30, cg_tol=1e-12, max_newton=1, init=fh.INIT_GIVEN)
        rng = np.random.default_rng(7)
        vox = rng.integers(0, n, size=(64, 3))
        h = 1e-6
        F = torch.empty_like(H0)
        errs = []
        for v in vox:
            v = tuple(int(t) for t in v)
            vals = []
            for sgn in (1, -1):
                r = rho.copy()
                r[v] += sgn * h
                m = fh.Material(0, phase, params, scale=r ** 3)
                F.copy_(H0)
                pbar, _, rc = ctx.fft_homog_solve(m, Hbar, F, options=fd_opts, allow=(fh.FH_ERR_NOT_CONVERGED,))
                vals.append(pbar[1])
            fd = (vals[0] - vals[1]) / (2 * h)
            errs.append(abs(fd - s[v]) / abs(s[v]))
        assert max(errs) < 1e-4, (max(errs), float(np.median(errs)))


@pytest.mark.parametrize("n,nz", [(192, 2), (199, 2), (199, 1)])
def test_eshelby_2d_mode_matches_oracle_and_table1(fh, n, nz):
    """2D plane strain as a z-invariant n x n x nz cell (Section 4.2.1, Table 1; the paper's grid is 199^2)."""
    import json

    from test_oracle_eshelby import GOLDEN, TABLE1_RTOL, dilute_estimate, eshelby_cell

    phase, f = eshelby_cell(n, nz=nz)
    params = np.array([[2.0, 1.0], [10.0, 5.0]])
    zero = np.zeros((9,) + phase.shape)
    C_ref = homogenize.tangent(phase, params, 0, zero, cg_tol=1e-12)
    with fh.Context(*phase.shape) as ctx:
        C = ctx.fft_homog_tangent(fh.Material(0, phase, params), dev(zero), options=fh.default_options(cg_tol=1e-12))
    assert np.abs(C - C_ref).max() < TOL * np.abs(C_ref).max()
    with open(GOLDEN) as fp:
        num = json.load(fp)["numerical"]
    np.testing.assert_allclose([C[0, 0], C[4, 4], C[1, 1]], [num["Cxxxx"], num["Cyyyy"], num["Cxyxy"]],
                               rtol=TABLE1_RTOL)
    np.testing.assert_allclose([C[0, 0], C[1, 1]], dilute_estimate(f), rtol=2e-4)


@pytest.mark.parametrize("kind,ij", [(1, (0, 1)), (2, (1, 1)), (0, (0, 1))])
def test_stress_sensitivity_matches_oracle_euler_and_finite_differences(fh, kind, ij):
    """dPbar_ij/drho per voxel at a converged finite-strain (or small-strain) state of a SIMP cell
    (modulus scale rho^3): against the oracle's adjoint formula (1e-9), Euler's identity
    sum_v rho_v dPbar/drho_v = 3 Pbar_ij, and central differences of two GPU solves (step 1e-4, whose
    truncation error is of order (h/rho)^2 ~ 1e-7) on eight voxels (1e-5)."""
    import torch

    n = 12
    rho = 0.35 + 0.65 * simp_config(n, seed=11)[2]  # densities in [0.35, 1]: modulus contrast 23
    scale, dscale = rho ** 3, 3.0 * rho ** 2
    phase = np.zeros((n, n, n), np.uint8)
    params = np.array([[1.5, 1.0]])
    if kind == 0:
        Fbar = np.zeros(9)
        Fbar[1] = Fbar[3] = 0.01
        Fbar[0] = 0.005
    else:
        Fbar = shear_macro(0.05, finite=True)
        Fbar[8] += 0.01
    ab = 3 * ij[0] + ij[1]
    opts = fh.default_options(newton_tol=1e-12, cg_tol=1e-13)
    with fh.Context(n, n, n) as ctx:
        def solve(sc):
            F = torch.zeros((9, n, n, n), dtype=torch.float64, device="cuda")
            pbar, _, _ = ctx.fft_homog_solve(fh.Material(kind, phase, params, scale=dev(sc)), Fbar, F, options=opts)
            return pbar, F

        pbar, F = solve(scale)
        out = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
        ctx.fft_homog_stress_sensitivity(fh.Material(kind, phase, params, scale=dev(scale)), F, ij, dev(dscale), out,
                                         options=opts)
        s = host(out)
        ref = homogenize.stress_sensitivity(phase, params, kind, host(F), scale, dscale, ab, cg_tol=1e-13)
        assert np.abs(s - ref).max() < TOL * np.abs(ref).max()
        np.testing.assert_allclose((s * rho).sum(), 3.0 * pbar[ab], rtol=1e-9)
        h = 1e-4
        rng = np.random.default_rng(5)
        for v in rng.integers(0, n, size=(8, 3)):
            v = tuple(int(t) for t in v)
            rp = rho.copy(); rp[v] += h
            rm = rho.copy(); rm[v] -= h
            fd = (solve(rp ** 3)[0][ab] - solve(rm ** 3)[0][ab]) / (2 * h)
            assert abs(fd - s[v]) <= 1e-5 * abs(s[v]) + 1e-7 * np.abs(s).max(), (v, fd, s[v])
