"""Homogenized tangent and its sensitivity to a voxel modulus field (oracle).

Section 3.3 defines the homogenized stiffness as the derivative of the volume
mean stress with respect to the macroscopic strain (Eq. 4) and obtains it by
forward-mode differentiation of the whole solve (Listing 5). At a converged
state that derivative is the solution of the linearised cell problem: for
each unit macroscopic perturbation E_cd (one entry of the 3x3 tensor set to
1), the fluctuation d solves

    G(K : (E_cd + d)) = 0,  d compatible (in the range of G),

by conjugate gradients with the converged tangent K, and column cd of the
homogenized tangent is mean(K : (E_cd + d)). This is the reading taken for
"jacfwd through the solver": the forward derivative of the converged state,
not of the iterates' rounding.

For linear elasticity the response to E_cd is linear in the moduli, and the
homogenized entry is the mutual energy  C_ab,cd = mean((E_ab + d_ab) : C :
(E_cd + d_cd)). Its derivative with respect to a voxel's modulus scale s_v
(the topology-optimisation sensitivity of Section 4.4.2, with C_v = s_v C0)
follows without an extra adjoint solve, because the cell problem is
self-adjoint and d_ab, d_cd are stationary:

    dC_ab,cd / d rho_v = (1/N) (E_ab + d_ab)_v : C0_v : (E_cd + d_cd)_v * ds_v/d rho_v.

For a hyperelastic law (finite strain) whose moduli a voxel scale multiplies,
P = s(rho) P0(F), the first-order quantity of Section 4.4 is the sensitivity
of the homogenized stress at the converged state. Differentiating the
equilibrium G(P) = 0 gives the fluctuation response dF/d rho_v, and with the
unit response d_ab of the linearised problem (K symmetric, d_ab compatible,
K : (E_ab + d_ab) equilibrated) the adjoint argument leaves

    dPbar_ab / d rho_v = (1/N) (E_ab + d_ab)_v : P0(F_v) * ds_v/d rho_v,

one linear CG solve per component ab.
"""

from __future__ import annotations

import numpy as np

from . import materials as mat
from .solver import cg, voxel_lame
from .spectral import project


def unit_response(K, cd: int, cg_tol: float, max_cg: int, lengths):
    """The strain field E_cd + d for a unit macroscopic entry cd, given the tangent K."""
    shape = K.shape[2:]
    E = np.zeros((9,) + shape)
    E[cd] = 1.0
    b = -project(mat.apply_tangent(K, E), lengths)
    d, it, ok = cg(lambda p: project(mat.apply_tangent(K, p), lengths), b, cg_tol, max_cg)
    if not ok:
        raise RuntimeError("tangent CG did not converge")
    return E + d, it


def tangent(phase, params, kind: int, F, scale=None, cg_tol: float = 1e-12, max_cg: int = 5000,
            lengths=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Homogenized tangent dPbar/dFbar (9x9, column cd = response to entry cd) at state F."""
    lam, mu = voxel_lame(phase, params, scale)
    K = mat.tangent(kind, F, lam, mu)
    C = np.zeros((9, 9))
    for cd in range(9):
        H, _ = unit_response(K, cd, cg_tol, max_cg, lengths)
        C[:, cd] = mat.apply_tangent(K, H).reshape(9, -1).mean(axis=1)
    return C


def sensitivity(phase, params, scale, dscale, ab: int, cd: int, cg_tol: float = 1e-12, max_cg: int = 5000,
                lengths=(1.0, 1.0, 1.0)) -> np.ndarray:
    """dC_ab,cd / d rho at every voxel for small-strain linear elasticity.

    scale: per-voxel modulus multiplier s(rho); dscale: ds/d rho per voxel.
    """
    shape = phase.shape
    lam, mu = voxel_lame(phase, params, scale)
    K = mat.tangent(mat.LINEAR_ELASTIC, np.zeros((9,) + shape), lam, mu)
    Ha, _ = unit_response(K, ab, cg_tol, max_cg, lengths)
    Hc = Ha if cd == ab else unit_response(K, cd, cg_tol, max_cg, lengths)[0]
    lam0, mu0 = voxel_lame(phase, params, None)
    K0 = mat.tangent(mat.LINEAR_ELASTIC, np.zeros((9,) + shape), lam0, mu0)
    return np.einsum("a...,a...->...", Ha, mat.apply_tangent(K0, Hc)) * dscale / phase.size


def stress_sensitivity(phase, params, kind: int, F, scale, dscale, ab: int, cg_tol: float = 1e-12,
                       max_cg: int = 5000, lengths=(1.0, 1.0, 1.0)) -> np.ndarray:
    """dPbar_ab / d rho at every voxel at the converged state F (any hyperelastic law, or linear elasticity).

    scale: per-voxel modulus multiplier s(rho); dscale: ds/d rho per voxel.
    """
    lam, mu = voxel_lame(phase, params, scale)
    K = mat.tangent(kind, F, lam, mu)
    H, _ = unit_response(K, ab, cg_tol, max_cg, lengths)
    lam0, mu0 = voxel_lame(phase, params, None)
    P0 = mat.stress(kind, F, lam0, mu0)
    return np.einsum("a...,a...->...", H, P0) * dscale / phase.size
