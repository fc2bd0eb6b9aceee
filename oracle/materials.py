"""Closed-form energies, stresses and tangents (the oracle side of Eqs. 2-3).

The paper obtains the stress as the derivative of an energy density (Eq. 2)
and the tangent K = dP/dF as its second derivative (Eq. 3) by automatic
differentiation. The oracle instead writes out the textbook closed forms, so
that it shares nothing with the GPU's dual-number arithmetic; the closed forms
are pinned against central finite differences of W in the tests.

Fields are float64 arrays of shape (9, ...) with component 3*i + j; a tangent
is (9, 9, ...) with K[3i+j, 3k+l] = dP_ij / dF_kl. ``lam`` and ``mu`` are
arrays broadcastable to the voxel shape.

Materials (kind codes shared with the C-ABI by value only):
  0  small-strain linear elastic, unknown = displacement gradient H,
     eps = sym(H), W = lam/2 tr(eps)^2 + mu eps:eps. The paper prints
     lam tr(eps)^2 + mu tr(eps:eps) (Section 3.2, Section 4.2.1); the factor 1/2
     on lambda is the reading taken, so that sigma = lam tr(eps) I + 2 mu eps.
  1  compressible neo-Hookean, W = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2.
  2  St. Venant-Kirchhoff, W = lam/2 tr(E)^2 + mu E:E with the Green-Lagrange
     strain E = (F^T F - I)/2 (Eq. 6; the paper's "F F^T - I" is read as this).
"""

from __future__ import annotations

import numpy as np

LINEAR_ELASTIC = 0
NEO_HOOKEAN = 1
SVK = 2
J2 = 3  # small-strain J2 plasticity; stress and tangent in ``plasticity`` (no energy)
FINITE_STRAIN = {LINEAR_ELASTIC: False, NEO_HOOKEAN: True, SVK: True, J2: False}


class NonPhysicalState(ValueError):
    """Raised when det F <= 0 (ln J undefined) or a value is not finite."""


def _t(F):
    return F.reshape((3, 3) + F.shape[1:])


def _flat(A):
    return A.reshape((9,) + A.shape[2:])


def _inv_det(F3):
    """Inverse and determinant of 3x3 tensors stored as (3, 3, ...)."""
    a = np.moveaxis(F3, (0, 1), (-2, -1))
    det = np.linalg.det(a)
    if not np.all(np.isfinite(det)) or np.any(det <= 0):
        raise NonPhysicalState("det F <= 0 or non-finite deformation")
    inv = np.linalg.inv(a)
    return np.moveaxis(inv, (-2, -1), (0, 1)), det


def energy(kind: int, F: np.ndarray, lam, mu) -> np.ndarray:
    """Stored energy density W per voxel."""
    F3 = _t(F)
    if kind == LINEAR_ELASTIC:
        eps = 0.5 * (F3 + F3.swapaxes(0, 1))
        tr = eps[0, 0] + eps[1, 1] + eps[2, 2]
        return 0.5 * lam * tr ** 2 + mu * np.einsum("ij...,ij...->...", eps, eps)
    if kind == NEO_HOOKEAN:
        _, J = _inv_det(F3)
        lnJ = np.log(J)
        I1 = np.einsum("ij...,ij...->...", F3, F3)
        return 0.5 * mu * (I1 - 3.0) - mu * lnJ + 0.5 * lam * lnJ ** 2
    if kind == SVK:
        E = _green(F3)
        tr = E[0, 0] + E[1, 1] + E[2, 2]
        return 0.5 * lam * tr ** 2 + mu * np.einsum("ij...,ij...->...", E, E)
    raise ValueError(f"unknown material kind {kind}")


def _green(F3):
    C = np.einsum("ki...,kj...->ij...", F3, F3)
    eye = np.eye(3).reshape((3, 3) + (1,) * (F3.ndim - 2))
    return 0.5 * (C - eye)


def stress(kind: int, F: np.ndarray, lam, mu) -> np.ndarray:
    """First derivative of W: the stress P = dW/dF (Eq. 2), shape (9, ...)."""
    F3 = _t(F)
    eye = np.eye(3).reshape((3, 3) + (1,) * (F3.ndim - 2))
    if kind == LINEAR_ELASTIC:
        eps = 0.5 * (F3 + F3.swapaxes(0, 1))
        tr = eps[0, 0] + eps[1, 1] + eps[2, 2]
        return _flat(lam * tr * eye + 2.0 * mu * eps)
    if kind == NEO_HOOKEAN:
        Finv, J = _inv_det(F3)
        FinvT = Finv.swapaxes(0, 1)
        return _flat(mu * (F3 - FinvT) + lam * np.log(J) * FinvT)
    if kind == SVK:
        E = _green(F3)
        tr = E[0, 0] + E[1, 1] + E[2, 2]
        S = lam * tr * eye + 2.0 * mu * E
        return _flat(np.einsum("im...,mj...->ij...", F3, S))
    raise ValueError(f"unknown material kind {kind}")


def tangent(kind: int, F: np.ndarray, lam, mu) -> np.ndarray:
    """Second derivative of W: K[3i+j, 3k+l] = dP_ij/dF_kl (Eq. 3), shape (9, 9, ...)."""
    F3 = _t(F)
    shape = F3.shape[2:]
    d = np.eye(3)
    lam = np.broadcast_to(lam, shape)
    mu = np.broadcast_to(mu, shape)
    if kind == LINEAR_ELASTIC:
        K = (np.einsum("ij,kl->ijkl", d, d)[..., None] * lam.reshape(-1)
             + (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))[..., None] * mu.reshape(-1))
        return K.reshape((9, 9) + shape)
    if kind == NEO_HOOKEAN:
        Finv, J = _inv_det(F3)
        lnJ = np.log(J)
        # mu d_ik d_jl + (mu - lam ln J) Finv_li Finv_jk + lam Finv_ji Finv_lk
        K = (np.einsum("ik,jl->ijkl", d, d).reshape((3, 3, 3, 3) + (1,) * len(shape)) * mu
             + np.einsum("li...,jk...->ijkl...", Finv, Finv) * (mu - lam * lnJ)
             + np.einsum("ji...,lk...->ijkl...", Finv, Finv) * lam)
        return K.reshape((9, 9) + shape)
    if kind == SVK:
        E = _green(F3)
        tr = E[0, 0] + E[1, 1] + E[2, 2]
        eye = d.reshape((3, 3) + (1,) * len(shape))
        S = lam * tr * eye + 2.0 * mu * E
        FFt = np.einsum("im...,km...->ik...", F3, F3)
        # d_ik S_lj + lam F_ij F_kl + mu F_il F_kj + mu (F F^T)_ik d_jl
        K = (np.einsum("ik,lj...->ijkl...", d, S)
             + lam * np.einsum("ij...,kl...->ijkl...", F3, F3)
             + mu * np.einsum("il...,kj...->ijkl...", F3, F3)
             + mu * np.einsum("ik...,jl->ijkl...", FFt, d))
        return K.reshape((9, 9) + shape)
    raise ValueError(f"unknown material kind {kind}")


def apply_tangent(K: np.ndarray, dF: np.ndarray) -> np.ndarray:
    """Incremental stress dP = K : dF per voxel (Eq. 3)."""
    return np.einsum("ab...,b...->a...", K, dF)
