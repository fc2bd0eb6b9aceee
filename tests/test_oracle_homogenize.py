"""Pins of the oracle's homogenized tangent (Eq. 4, Listing 5) and sensitivities.

* the tangent equals central finite differences of the homogenized stress of
  two full solves, column by column;
* it has major symmetry, equals K(Fbar) for a homogeneous cell, reproduces
  the Reuss and Voigt shear moduli of a laminate, and lies between the Reuss
  and Voigt bounds for a random two-phase linear cell;
* the voxel sensitivities equal central finite differences of the tangent in
  the voxel density, and satisfy Euler's identity for a modulus scale rho^3
  (the tangent is homogeneous of degree one in the moduli);
* the finite-strain stress sensitivities (neo-Hookean and SVK) equal central
  finite differences of the homogenized stress of two full solves in the
  voxel density, and satisfy Euler's identity sum_v rho_v dPbar/drho_v =
  3 Pbar for a modulus scale rho^3 (the equilibrium field does not change when
  every modulus is scaled alike, so Pbar is homogeneous of degree three in rho).
"""

import numpy as np
import pytest

from oracle import homogenize, laminate, materials as mat, solver
from rve_inputs import laminate as laminate_map, simp_config, two_phase_table


def _two_phase(shape, seed, frac=0.4):
    rng = np.random.default_rng(seed)
    return (rng.uniform(size=shape) < frac).astype(np.uint8)


def test_tangent_matches_finite_differences_of_pbar():
    shape = (4, 4, 4)
    phase = _two_phase(shape, 1)
    params = two_phase_table(1.5, 1.0, 6.0)
    Fbar = np.eye(3).reshape(9) + np.array([0.02, 0.04, 0.0, -0.01, 0.03, 0.01, 0.0, 0.02, -0.02])
    r = solver.solve(phase, params, mat.NEO_HOOKEAN, Fbar, newton_tol=1e-13)
    C = homogenize.tangent(phase, params, mat.NEO_HOOKEAN, r.F)
    h = 1e-5
    for cd in range(9):
        Fp = Fbar.copy(); Fp[cd] += h
        Fm = Fbar.copy(); Fm[cd] -= h
        Pp = solver.solve(phase, params, mat.NEO_HOOKEAN, Fp, newton_tol=1e-13).Pbar
        Pm = solver.solve(phase, params, mat.NEO_HOOKEAN, Fm, newton_tol=1e-13).Pbar
        np.testing.assert_allclose(C[:, cd], (Pp - Pm) / (2 * h), rtol=1e-6, atol=1e-7)


def test_tangent_major_symmetry_and_homogeneous_cell():
    shape = (6, 4, 4)
    phase = _two_phase(shape, 2)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = np.eye(3).reshape(9) + np.array([0.0, 0.05, 0.0, 0.0, 0.02, 0.0, 0.01, 0.0, 0.0])
    r = solver.solve(phase, params, mat.NEO_HOOKEAN, Fbar, newton_tol=1e-12)
    C = homogenize.tangent(phase, params, mat.NEO_HOOKEAN, r.F)
    np.testing.assert_allclose(C, C.T, atol=1e-10 * np.abs(C).max())
    one = np.zeros(shape, np.uint8)
    Fh = np.broadcast_to(Fbar.reshape(9, 1, 1, 1), (9,) + shape).copy()
    Ch = homogenize.tangent(one, params, mat.NEO_HOOKEAN, Fh)
    np.testing.assert_allclose(Ch, mat.tangent(1, Fbar.reshape(9, 1), 1.5, 1.0)[:, :, 0], atol=1e-13)


def test_linear_laminate_tangent_has_reuss_and_voigt_shear():
    shape = (8, 4, 4)
    phase = laminate_map(shape, 4, axis=0)
    params = two_phase_table(0.6, 0.4, 10.0)
    C = homogenize.tangent(phase, params, mat.LINEAR_ELASTIC, np.zeros((9,) + shape))
    mu_across, mu_along = laminate.linear_shear_moduli(params, 0.5)
    np.testing.assert_allclose(C[1, 1], mu_across, rtol=1e-11)   # d sigma_xy / d H_xy
    np.testing.assert_allclose(C[5, 5], mu_along, rtol=1e-11)    # d sigma_yz / d H_yz


def test_linear_tangent_between_reuss_and_voigt_bounds():
    shape = (6, 6, 6)
    phase = _two_phase(shape, 3, 0.3)
    params = two_phase_table(0.6, 0.4, 10.0)
    C = homogenize.tangent(phase, params, mat.LINEAR_ELASTIC, np.zeros((9,) + shape))
    lam, mu = params[phase, 0], params[phase, 1]
    Kv = mat.tangent(0, np.zeros((9,) + shape), lam, mu).reshape(9, 9, -1)
    # restrict to symmetric strains through an orthonormal basis of them
    B = []
    for i in range(3):
        for j in range(i, 3):
            e = np.zeros((3, 3)); e[i, j] = e[j, i] = 1.0
            B.append((e / np.linalg.norm(e)).reshape(9))
    B = np.array(B).T  # 9 x 6
    Cs = B.T @ C @ B
    Cv = B.T @ Kv.mean(axis=2) @ B
    Cr = np.linalg.inv(np.mean([np.linalg.inv(B.T @ Kv[:, :, v] @ B) for v in range(Kv.shape[2])], axis=0))
    assert np.linalg.eigvalsh(Cv - Cs).min() > -1e-12
    assert np.linalg.eigvalsh(Cs - Cr).min() > -1e-12
    np.testing.assert_allclose(Cs, Cs.T, atol=1e-12)


@pytest.mark.parametrize("ab,cd", [(1, 1), (0, 4)])
def test_sensitivity_matches_finite_differences_and_euler_identity(ab, cd):
    phase, params, rho, scale, dscale = simp_config(4, seed=5)
    zero = np.zeros((9,) + phase.shape)
    s = homogenize.sensitivity(phase, params, scale, dscale, ab, cd)
    C = homogenize.tangent(phase, params, mat.LINEAR_ELASTIC, zero, scale=scale)
    # Euler: C is homogeneous of degree one in the moduli scale rho^3
    np.testing.assert_allclose((s * rho / 3.0).sum(), C[ab, cd], rtol=1e-10)
    h = 1e-4
    for v in [(0, 0, 0), (1, 2, 3), (3, 1, 0)]:
        rp = rho.copy(); rp[v] += h
        rm = rho.copy(); rm[v] -= h
        Cp = homogenize.tangent(phase, params, 0, zero, scale=rp ** 3)[ab, cd]
        Cm = homogenize.tangent(phase, params, 0, zero, scale=rm ** 3)[ab, cd]
        np.testing.assert_allclose(s[v], (Cp - Cm) / (2 * h), rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("kind,ab", [(mat.NEO_HOOKEAN, 1), (mat.NEO_HOOKEAN, 0), (mat.SVK, 3)])
def test_stress_sensitivity_matches_finite_differences_and_euler_identity(kind, ab):
    shape = (4, 4, 4)
    phase, params, rho, scale, dscale = simp_config(4, seed=7)
    params = two_phase_table(1.5, 1.0, 5.0)[:1]
    phase = np.zeros(shape, np.uint8)
    Fbar = np.eye(3).reshape(9) + np.array([0.02, 0.05, 0.0, -0.01, 0.01, 0.02, 0.0, 0.01, -0.02])

    def pbar(r):
        return solver.solve(phase, params, kind, Fbar, newton_tol=1e-13, cg_tol=1e-14, scale=r ** 3).Pbar

    ref = solver.solve(phase, params, kind, Fbar, newton_tol=1e-13, cg_tol=1e-14, scale=scale)
    s = homogenize.stress_sensitivity(phase, params, kind, ref.F, scale, dscale, ab, cg_tol=1e-14)
    np.testing.assert_allclose((s * rho).sum(), 3.0 * ref.Pbar[ab], rtol=1e-9)
    h = 1e-5
    for v in [(0, 0, 0), (1, 2, 3), (3, 1, 0)]:
        rp = rho.copy(); rp[v] += h
        rm = rho.copy(); rm[v] -= h
        fd = (pbar(rp)[ab] - pbar(rm)[ab]) / (2 * h)
        np.testing.assert_allclose(s[v], fd, rtol=1e-6, atol=1e-11)
