"""Exact solutions of two-phase laminates (an independent pin of the solver).

For a cell whose phase depends only on the coordinate along e_a, the discrete
Fourier-Galerkin solution is piecewise constant when each layer spans an even
number of voxels (so that the fluctuation has no Nyquist content, which the
projection of Eq. 1 cannot represent on an even axis):

    F_A = Fbar + f_B c (x) e_a,   F_B = Fbar - f_A c (x) e_a,

so that f_A F_A + f_B F_B = Fbar and F_A - F_B = c (x) e_a is a rank-one jump,
with traction continuity P_A(F_A) e_a = P_B(F_B) e_a. The unknown jump vector
c (3 entries) solves that equation by Newton's method with the closed-form
tangents; for linear elasticity the homogenized shear moduli follow in closed
form (Reuss across the layers, Voigt along them).
"""

from __future__ import annotations

import numpy as np

from . import materials as mat


def laminate_states(kind: int, params: np.ndarray, f_A: float, Fbar, axis: int = 0,
                    tol: float = 1e-15, max_iter: int = 50):
    """Return (F_A, F_B) for phase A = row 1, phase B = row 0 of ``params``.

    ``f_A`` is the volume fraction of phase A (row 1, the layered phase).
    """
    lA, mA = params[1]
    lB, mB = params[0]
    return laminate_states_law(
        lambda F: mat.stress(kind, F[:, None], lA, mA)[:, 0],
        lambda F: mat.tangent(kind, F[:, None], lA, mA)[:, :, 0],
        lambda F: mat.stress(kind, F[:, None], lB, mB)[:, 0],
        lambda F: mat.tangent(kind, F[:, None], lB, mB)[:, :, 0],
        f_A, Fbar, axis, tol, max_iter)


def laminate_states_law(stress_A, tangent_A, stress_B, tangent_B, f_A: float, Fbar, axis: int = 0,
                        tol: float = 1e-15, max_iter: int = 50):
    """Laminate states for any pair of stress laws given as callables.

    ``stress_X(F)`` returns the 9 stress entries of one voxel state F (9,),
    ``tangent_X(F)`` the 9x9 derivative. Used for path-dependent laws, whose
    callables close over the layer's history.
    """
    Fbar = np.asarray(Fbar, dtype=np.float64).reshape(9)
    f_B = 1.0 - f_A
    e = np.zeros(3)
    e[axis] = 1.0
    c = np.zeros(3)
    for _ in range(max_iter):
        FA = Fbar + f_B * np.outer(c, e).reshape(9)
        FB = Fbar - f_A * np.outer(c, e).reshape(9)
        PA = stress_A(FA).reshape(3, 3)
        PB = stress_B(FB).reshape(3, 3)
        R = PA[:, axis] - PB[:, axis]
        KA = tangent_A(FA).reshape(3, 3, 3, 3)
        KB = tangent_B(FB).reshape(3, 3, 3, 3)
        Jac = f_B * KA[:, axis, :, axis] + f_A * KB[:, axis, :, axis]
        dc = np.linalg.solve(Jac, -R)
        c += dc
        if np.linalg.norm(dc) <= tol * max(1.0, np.linalg.norm(c)):
            break
    FA = Fbar + f_B * np.outer(c, e).reshape(9)
    FB = Fbar - f_A * np.outer(c, e).reshape(9)
    return FA, FB


def linear_shear_moduli(params: np.ndarray, f_A: float):
    """Effective shear moduli of a linear elastic laminate.

    Returns (mu_across, mu_along): the Reuss mean (f_A/mu_A + f_B/mu_B)^-1 for
    shear in a plane containing the normal, and the Voigt mean
    f_A mu_A + f_B mu_B for shear in the layer plane.
    """
    mA, mB = params[1, 1], params[0, 1]
    f_B = 1.0 - f_A
    return 1.0 / (f_A / mA + f_B / mB), f_A * mA + f_B * mB
