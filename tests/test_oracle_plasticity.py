"""Pins of the oracle's J2 return mapping (Section 4.1.2, Appendix B).

* the consistent tangent equals central finite differences of the stress, in
  the elastic and in the plastic regime, and has major symmetry;
* a plastic state returned by the map lies on the updated yield surface;
* uniaxial-strain loading of one voxel follows the closed-form elastoplastic
  response (stiffness lambda + 2 mu, then the plastic modulus);
* an elastic trial state is left untouched.
"""

import numpy as np
import pytest

from oracle import plasticity as pl

LAM, MU, SY, HH = 1.2, 0.8, 0.01, 0.3


def _H(seed, scale):
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=(9, 5))


@pytest.mark.parametrize("scale", [1e-3, 0.05])
def test_tangent_is_stress_derivative(scale):
    H = _H(1, scale)
    ep = _H(2, 0.2 * scale)
    ep = 0.5 * (ep.reshape(3, 3, -1) + ep.reshape(3, 3, -1).swapaxes(0, 1)).reshape(9, -1)
    p = np.full(5, 0.002)
    K = pl.tangent(H, ep, p, LAM, MU, SY, HH)
    h = 1e-7
    for b in range(9):
        Hp = H.copy(); Hp[b] += h
        Hm = H.copy(); Hm[b] -= h
        fd = (pl.stress(Hp, ep, p, LAM, MU, SY, HH) - pl.stress(Hm, ep, p, LAM, MU, SY, HH)) / (2 * h)
        np.testing.assert_allclose(K[:, b], fd, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(K, K.transpose(1, 0, 2), atol=1e-12)


def test_plastic_state_lies_on_updated_yield_surface():
    H = _H(3, 0.05)
    ep = np.zeros((9, 5))
    p = np.zeros(5)
    sig = pl.stress(H, ep, p, LAM, MU, SY, HH).reshape(3, 3, -1)
    ep2, p2 = pl.update(H, ep, p, LAM, MU, SY, HH)
    assert np.all(p2 > 0)
    s = sig - np.trace(sig)[None, None] / 3.0 * np.eye(3)[:, :, None]
    q = np.sqrt(1.5 * np.einsum("ij...,ij...->...", s, s))
    np.testing.assert_allclose(q, SY + HH * p2, rtol=1e-12)
    # the stress is the elastic response to the remaining elastic strain
    eps = 0.5 * (H.reshape(3, 3, -1) + H.reshape(3, 3, -1).swapaxes(0, 1)) - ep2.reshape(3, 3, -1)
    ref = LAM * np.trace(eps)[None, None] * np.eye(3)[:, :, None] + 2 * MU * eps
    np.testing.assert_allclose(sig, ref, atol=1e-14)


def test_uniaxial_strain_closed_form():
    """eps = diag(e, 0, 0): elastic slope lambda + 2 mu, plastic slope from the return map."""
    e_y = SY / (2 * MU)  # q_tr = 2 mu e at yield for uniaxial strain
    slope_pl = LAM + 2 * MU - 4 * MU ** 2 / (3 * MU + HH)
    for e in [0.5 * e_y, 3 * e_y]:
        H = np.zeros((9, 1)); H[0] = e
        sig = pl.stress(H, np.zeros((9, 1)), np.zeros(1), LAM, MU, SY, HH)[0, 0]
        if e <= e_y:
            np.testing.assert_allclose(sig, (LAM + 2 * MU) * e, rtol=1e-14)
        else:
            np.testing.assert_allclose(sig, (LAM + 2 * MU) * e_y + slope_pl * (e - e_y), rtol=1e-12)


def test_elastic_trial_is_untouched():
    H = _H(4, 1e-4)
    ep = np.zeros((9, 5)); p = np.zeros(5)
    K = pl.tangent(H, ep, p, LAM, MU, SY, HH)
    ep2, p2 = pl.update(H, ep, p, LAM, MU, SY, HH)
    assert np.all(p2 == 0) and np.all(ep2 == 0)
    d = np.eye(3)
    Ce = (LAM * np.einsum("ij,kl->ijkl", d, d) + MU * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))).reshape(9, 9)
    np.testing.assert_allclose(K[:, :, 0], Ce, atol=1e-14)
