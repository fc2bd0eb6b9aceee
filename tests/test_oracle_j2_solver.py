"""Pins of the oracle's J2 solve with history (Section 4.1.2, Appendix B, Alg. 1).

* a one-phase cell under uniaxial strain is homogeneous: after any number of
  increments its stress and cumulative plastic strain follow the closed-form
  elastoplastic response, and partial unloading is elastic;
* a two-layer laminate whose layers yield at different stresses matches the
  exact laminate solution advanced increment by increment with each layer's
  own return map and history (traction continuity across the layers);
* the stress reported after a converged increment equals the elastic
  response to the strain minus the updated plastic strain.
"""

import numpy as np
import pytest

from oracle import laminate, materials as mat, plasticity as pl, solver
from rve_inputs import j2_config, laminate as laminate_map

LAM, MU = 1.2, 0.8


@pytest.mark.parametrize("n_inc", [1, 4])
def test_homogeneous_uniaxial_strain_closed_form_and_unloading(n_inc):
    sy, hh = 0.01, 0.3
    phase = np.zeros((4, 4, 2), dtype=np.uint8)
    params = np.array([[LAM, MU]])
    plastic = np.array([[sy, hh]])
    e_y = sy / (2 * MU)
    e = 3 * e_y
    Ebar = np.zeros(9)
    Ebar[0] = e
    r = solver.solve(phase, params, mat.J2, Ebar, n_increments=n_inc, newton_tol=1e-12,
                     plastic=plastic)
    slope_pl = LAM + 2 * MU - 4 * MU ** 2 / (3 * MU + hh)
    s_peak = (LAM + 2 * MU) * e_y + slope_pl * (e - e_y)
    np.testing.assert_allclose(r.Pbar[0], s_peak, rtol=1e-12)
    # cumulative plastic strain: q = 2 mu (e - e_p11 * 3/2) on the updated surface
    p_exact = 2 * MU * (e - e_y) / (3 * MU + hh)
    np.testing.assert_allclose(r.history[9], p_exact, rtol=1e-12)
    # unloading by 1.5 e_y stays elastic (reverse yield needs more than 2 e_y)
    Eun = Ebar.copy()
    Eun[0] = e - 1.5 * e_y
    r2 = solver.solve(phase, params, mat.J2, Eun, n_increments=2, newton_tol=1e-12, F_init=r.F,
                      plastic=plastic, history=r.history)
    np.testing.assert_allclose(r2.Pbar[0], s_peak - (LAM + 2 * MU) * 1.5 * e_y, rtol=1e-12)
    np.testing.assert_array_equal(r2.history, r.history)


def test_two_layer_laminate_matches_exact_incremental_solution():
    shape = (8, 4, 2)
    phase = laminate_map(shape, 4, axis=0)  # f_A = 1/2, layers 4 voxels thick
    params = np.array([[LAM, MU], [1.5 * LAM, 1.5 * MU]])
    plastic = np.array([[0.01, 0.2], [0.02, 0.4]])
    Ebar = np.zeros(9)
    Ebar[0] = 0.02
    Ebar[4] = 0.01
    Ebar[1] = Ebar[3] = 0.015
    n_inc = 5
    r = solver.solve(phase, params, mat.J2, Ebar, n_increments=n_inc, newton_tol=1e-13, plastic=plastic)
    # exact laminate, advanced increment by increment with each layer's history
    hist = {0: (np.zeros(9), 0.0), 1: (np.zeros(9), 0.0)}

    def law(ph, fn):
        (lam, mu), (sy, hh) = params[ph], plastic[ph]
        ep, p = hist[ph]
        return lambda F: fn(F[:, None], ep[:, None], np.array([p]), lam, mu, sy, hh)[..., 0]

    for n in range(1, n_inc + 1):
        En = Ebar * n / n_inc
        FA, FB = laminate.laminate_states_law(law(1, pl.stress), law(1, pl.tangent), law(0, pl.stress),
                                              law(0, pl.tangent), 0.5, En, axis=0)
        for ph, F in ((1, FA), (0, FB)):
            (lam, mu), (sy, hh) = params[ph], plastic[ph]
            ep, p = hist[ph]
            ep2, p2 = pl.update(F[:, None], ep[:, None], np.array([p]), lam, mu, sy, hh)
            hist[ph] = (ep2[:, 0], float(p2[0]))
    assert hist[0][1] > 0 and hist[1][1] > 0, "both layers should have yielded"
    assert hist[0][1] != pytest.approx(hist[1][1], rel=1e-3)
    for ph, F in ((1, FA), (0, FB)):
        sel = phase == ph
        for c in range(9):
            np.testing.assert_allclose(r.F[c][sel], F[c], rtol=0, atol=1e-12)
        for c in range(9):
            np.testing.assert_allclose(r.history[c][sel], hist[ph][0][c], rtol=0, atol=1e-12)
        np.testing.assert_allclose(r.history[9][sel], hist[ph][1], rtol=1e-10)


def test_reported_stress_is_elastic_response_to_remaining_strain():
    phase, params, plastic, Ebar = j2_config(24, 0, nz=1)
    r = solver.solve(phase, params, mat.J2, Ebar, n_increments=3, newton_tol=1e-10, plastic=plastic)
    assert r.history[9].max() > 0
    H = r.F.reshape(3, 3, -1)
    eps = 0.5 * (H + H.swapaxes(0, 1)) - r.history[:9].reshape(3, 3, -1)
    lam, mu = params[phase.reshape(-1), 0], params[phase.reshape(-1), 1]
    ref = lam * np.trace(eps)[None, None] * np.eye(3)[:, :, None] + 2 * mu * eps
    np.testing.assert_allclose(r.P.reshape(3, 3, -1), ref, atol=1e-12)
