"""Pins of the oracle's closed-form stresses and tangents (Eqs. 2-3).

P must be the derivative of W and K the derivative of P (checked by central
finite differences of the energy, which is the definition written out), K must
have major symmetry, and both finite-strain laws must reduce to linear
elasticity at F = I.
"""

import numpy as np
import pytest

from oracle import materials as mat
from rve_inputs import random_deformation

KINDS = [mat.LINEAR_ELASTIC, mat.NEO_HOOKEAN, mat.SVK]


def _F(kind, n=6, seed=0):
    return random_deformation(n, seed, scale=0.15, identity=mat.FINITE_STRAIN[kind])


@pytest.mark.parametrize("kind", KINDS)
def test_stress_is_energy_gradient(kind):
    F = _F(kind)
    lam, mu = 1.3, 0.7
    P = mat.stress(kind, F, lam, mu)
    h = 1e-6
    for a in range(9):
        Fp = F.copy(); Fp[a] += h
        Fm = F.copy(); Fm[a] -= h
        fd = (mat.energy(kind, Fp, lam, mu) - mat.energy(kind, Fm, lam, mu)) / (2 * h)
        np.testing.assert_allclose(P[a], fd, rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("kind", KINDS)
def test_tangent_is_stress_gradient_and_major_symmetric(kind):
    F = _F(kind, seed=1)
    lam, mu = 1.3, 0.7
    K = mat.tangent(kind, F, lam, mu)
    h = 1e-6
    for b in range(9):
        Fp = F.copy(); Fp[b] += h
        Fm = F.copy(); Fm[b] -= h
        fd = (mat.stress(kind, Fp, lam, mu) - mat.stress(kind, Fm, lam, mu)) / (2 * h)
        np.testing.assert_allclose(K[:, b], fd, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(K, K.transpose(1, 0, 2), atol=1e-13)


@pytest.mark.parametrize("kind", [mat.NEO_HOOKEAN, mat.SVK])
def test_finite_strain_laws_reduce_to_linear_elasticity_at_identity(kind):
    I = np.eye(3).reshape(9, 1)
    lam, mu = 1.5, 1.0
    np.testing.assert_allclose(mat.stress(kind, I, lam, mu), 0.0, atol=1e-15)
    np.testing.assert_allclose(mat.tangent(kind, I, lam, mu),
                               mat.tangent(mat.LINEAR_ELASTIC, np.zeros((9, 1)), lam, mu), atol=1e-14)


def test_linear_elastic_stress_is_hooke():
    eps = np.array([[0.01, 0.002, 0.0], [0.002, -0.003, 0.004], [0.0, 0.004, 0.005]])
    lam, mu = 0.6, 0.4
    H = eps + np.array([[0, 0.3, -0.1], [-0.3, 0, 0.2], [0.1, -0.2, 0]])  # add a rotation
    P = mat.stress(mat.LINEAR_ELASTIC, H.reshape(9, 1), lam, mu).reshape(3, 3)
    np.testing.assert_allclose(P, lam * np.trace(eps) * np.eye(3) + 2 * mu * eps, atol=1e-15)


def test_neo_hookean_uniaxial_closed_form():
    """Stretch F = diag(s, 1, 1): P_11 = mu (s - 1/s) + lam ln(s)/s, P_22 = lam ln(s), P_12 = 0."""
    s = 1.2
    lam, mu = 1.5, 1.0
    P = mat.stress(mat.NEO_HOOKEAN, np.diag([s, 1.0, 1.0]).reshape(9, 1), lam, mu).reshape(3, 3)
    np.testing.assert_allclose(P[0, 0], mu * (s - 1 / s) + lam * np.log(s) / s, rtol=1e-15)
    np.testing.assert_allclose(P[1, 1], lam * np.log(s), rtol=1e-15)
    np.testing.assert_allclose(P[0, 1], 0.0, atol=1e-15)


def test_non_physical_state_raises():
    F = np.diag([-1.0, 1.0, 1.0]).reshape(9, 1)
    with pytest.raises(mat.NonPhysicalState):
        mat.stress(mat.NEO_HOOKEAN, F, 1.0, 1.0)
