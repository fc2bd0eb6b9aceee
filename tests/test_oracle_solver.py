"""Pins of the oracle's Newton-Krylov solve (Algorithm 1) against independent results.

* homogeneous material: the fluctuation is zero and Pbar = P(Fbar);
* laminates: the exact piecewise-constant solution (traction continuity and a
  rank-one jump, solved by a 3-unknown Newton iteration) and, for linear
  elasticity, the Reuss and Voigt shear moduli in closed form;
* tiny grids: dense minimisation of the discrete energy with derivative
  matrices from the explicit DFT sum and least-squares Newton steps;
* mean(F) = Fbar, linear problems converge in two Newton iterations, and the
  final state does not depend on how the load is split into increments.
"""

import numpy as np
import pytest

from oracle import brute, laminate, materials as mat, solver
from rve_inputs import laminate as laminate_map, shear_macro, two_phase_table


def _fbar(kind, seed=0, scale=0.04):
    rng = np.random.default_rng(seed)
    F = rng.uniform(-scale, scale, 9)
    if mat.FINITE_STRAIN[kind]:
        F[[0, 4, 8]] += 1.0
    else:
        F = 0.5 * (F.reshape(3, 3) + F.reshape(3, 3).T).reshape(9)
    return F


@pytest.mark.parametrize("kind", [mat.LINEAR_ELASTIC, mat.NEO_HOOKEAN, mat.SVK])
def test_homogeneous_material_has_no_fluctuation(kind):
    shape = (6, 5, 4)
    phase = (np.arange(np.prod(shape)) % 2).astype(np.uint8).reshape(shape)
    params = np.array([[1.5, 1.0], [1.5, 1.0]])
    Fbar = _fbar(kind)
    r = solver.solve(phase, params, kind, Fbar, newton_tol=1e-12)
    assert np.abs(r.F - Fbar.reshape(9, 1, 1, 1)).max() < 1e-14
    Pref = mat.stress(kind, Fbar.reshape(9, 1), 1.5, 1.0)[:, 0]
    np.testing.assert_allclose(r.Pbar, Pref, atol=1e-14)


@pytest.mark.parametrize("kind", [mat.NEO_HOOKEAN, mat.SVK, mat.LINEAR_ELASTIC])
@pytest.mark.parametrize("axis", [0, 2])
def test_laminate_matches_exact_piecewise_constant_solution(kind, axis):
    shape = [4, 4, 4]
    shape[axis] = 8
    shape = tuple(shape)
    phase = laminate_map(shape, 2, axis=axis)  # phase 1 on two layers: f_A = 1/4
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = _fbar(kind, seed=3, scale=0.05)
    r = solver.solve(phase, params, kind, Fbar, newton_tol=1e-12, n_increments=2)
    FA, FB = laminate.laminate_states(kind, params, 0.25, Fbar, axis=axis)
    F = r.F.reshape(9, -1)
    ph = phase.reshape(-1)
    assert np.abs(F[:, ph == 1] - FA[:, None]).max() < 1e-11
    assert np.abs(F[:, ph == 0] - FB[:, None]).max() < 1e-11


def test_linear_laminate_shear_moduli_reuss_and_voigt():
    shape = (8, 4, 4)
    phase = laminate_map(shape, 4, axis=0)  # f_A = 1/2
    params = two_phase_table(0.6, 0.4, 10.0)
    mu_across, mu_along = laminate.linear_shear_moduli(params, 0.5)
    g = 0.01
    r = solver.solve(phase, params, mat.LINEAR_ELASTIC, shear_macro(g, finite=False), newton_tol=1e-12)
    np.testing.assert_allclose(r.Pbar[1], 2 * g * mu_across, rtol=1e-12)
    E = np.zeros(9); E[5] = E[7] = g  # shear in the layer plane (yz)
    r = solver.solve(phase, params, mat.LINEAR_ELASTIC, E, newton_tol=1e-12)
    np.testing.assert_allclose(r.Pbar[5], 2 * g * mu_along, rtol=1e-12)


@pytest.mark.parametrize("kind,shape", [(mat.NEO_HOOKEAN, (4, 4, 4)), (mat.LINEAR_ELASTIC, (4, 4, 4)),
                                        (mat.NEO_HOOKEAN, (3, 3, 3)), (mat.SVK, (3, 4, 2))])
def test_matches_dense_energy_minimisation(kind, shape):
    rng = np.random.default_rng(7)
    phase = (rng.uniform(size=shape) < 0.4).astype(np.uint8)
    params = two_phase_table(1.5, 1.0, 5.0)
    Fbar = _fbar(kind, seed=5, scale=0.05)
    r = solver.solve(phase, params, kind, Fbar, newton_tol=1e-13)
    Fb = brute.minimise(phase, params, kind, Fbar)
    assert np.abs(r.F - Fb).max() < 1e-11


def test_mean_strain_equals_macro_and_linear_takes_two_newton_steps():
    rng = np.random.default_rng(9)
    shape = (6, 6, 6)
    phase = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    params = two_phase_table(0.6, 0.4, 10.0)
    Ebar = shear_macro(0.01, finite=False)
    r = solver.solve(phase, params, mat.LINEAR_ELASTIC, Ebar, newton_tol=1e-10)
    np.testing.assert_allclose(r.F.reshape(9, -1).mean(axis=1), Ebar, atol=1e-16)
    assert len(r.newton_residuals) == 2


def test_increments_reach_the_same_state():
    rng = np.random.default_rng(11)
    shape = (6, 6, 6)
    phase = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.05, finite=True)
    r1 = solver.solve(phase, params, mat.NEO_HOOKEAN, Fbar, n_increments=1, newton_tol=1e-12)
    r5 = solver.solve(phase, params, mat.NEO_HOOKEAN, Fbar, n_increments=5, newton_tol=1e-12)
    assert np.abs(r1.F - r5.F).max() < 1e-11
    np.testing.assert_allclose(r1.F.reshape(9, -1).mean(axis=1), Fbar, atol=1e-15)
    # Newton converges quadratically once close: the last residual is far below tol
    assert r5.newton_residuals[-1] < 1e-12


def test_warm_start_continues_from_given_field():
    rng = np.random.default_rng(12)
    shape = (4, 6, 4)
    phase = (rng.uniform(size=shape) < 0.3).astype(np.uint8)
    params = two_phase_table(1.5, 1.0, 10.0)
    r_a = solver.solve(phase, params, mat.NEO_HOOKEAN, shear_macro(0.02, True), newton_tol=1e-12)
    r_b = solver.solve(phase, params, mat.NEO_HOOKEAN, shear_macro(0.05, True), newton_tol=1e-12,
                       F_init=r_a.F, n_increments=3)
    r_c = solver.solve(phase, params, mat.NEO_HOOKEAN, shear_macro(0.05, True), newton_tol=1e-12)
    assert np.abs(r_b.F - r_c.F).max() < 1e-11
