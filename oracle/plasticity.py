"""Small-strain J2 plasticity with linear isotropic hardening (oracle).

Section 4.1.2 and Appendix B of the paper: an elastic predictor, the von Mises
yield check, a radial return and the cumulative plastic strain, evaluated at
the total strain of the current increment from the history of the last
converged one. Written here in the plastic-strain form:

    eps      = sym(H),             eps_p, p : history (plastic strain, cumulative plastic strain)
    sig_tr   = C : (eps - eps_p),  s_tr = dev(sig_tr),  q_tr = sqrt(3/2 s_tr : s_tr)
    Phi      = q_tr - (sigma_y + H_iso p)
    dp       = <Phi>_+ / (3 mu + H_iso)
    sig      = sig_tr - 3 mu dp s_tr / q_tr
    eps_p'   = eps_p + (3/2) dp s_tr / q_tr,   p' = p + dp

Readings of garbled passages: Appendix B writes the return as
"- 2 mu dp s_tr / q_tr" and the elastic-strain update without the factor 3/2;
with dp = Phi/(3 mu + H_iso) only the factor 3 mu = (3/2)(2 mu) brings the
corrected stress onto the updated yield surface, so that factor is used. The
closed-form consistent tangent printed in Section 4.1.2 is garbled (its second
coefficient reads 4 mu^2); the one derived from the return above is

    K = C - (6 mu^2 dp / q_tr) I_dev + 6 mu^2 (dp / q_tr - 1/(3 mu + H_iso)) N (x) N,

N = s_tr / |s_tr|, and the elastic C when Phi <= 0. The tests pin it against
finite differences of the stress.

Fields: H (9, ...) displacement gradient; eps_p (9, ...) symmetric; p (...).
Parameters per voxel: lam, mu, sigma_y, h (hardening modulus H_iso).
"""

from __future__ import annotations

import numpy as np


def _t(A):
    return A.reshape((3, 3) + A.shape[1:])


def _sym(A3):
    return 0.5 * (A3 + A3.swapaxes(0, 1))


def trial(H, eps_p, lam, mu):
    eps = _sym(_t(H)) - _t(eps_p)
    tr = eps[0, 0] + eps[1, 1] + eps[2, 2]
    eye = np.eye(3).reshape((3, 3) + (1,) * (eps.ndim - 2))
    sig = lam * tr * eye + 2.0 * mu * eps
    s = sig - (sig[0, 0] + sig[1, 1] + sig[2, 2]) / 3.0 * eye
    q = np.sqrt(1.5 * np.einsum("ij...,ij...->...", s, s))
    return sig, s, q


def stress(H, eps_p, p, lam, mu, sigma_y, h):
    """Stress (9, ...) at total strain sym(H) from the history (eps_p, p)."""
    sig, s, q = trial(H, eps_p, lam, mu)
    phi = q - (sigma_y + h * p)
    dp = np.maximum(phi, 0.0) / (3.0 * mu + h)
    safe_q = np.where(q > 0, q, 1.0)
    sig = sig - 3.0 * mu * dp / safe_q * s
    return sig.reshape((9,) + sig.shape[2:])


def update(H, eps_p, p, lam, mu, sigma_y, h):
    """History (eps_p', p') after the increment that ends at total strain sym(H)."""
    sig, s, q = trial(H, eps_p, lam, mu)
    phi = q - (sigma_y + h * p)
    dp = np.maximum(phi, 0.0) / (3.0 * mu + h)
    safe_q = np.where(q > 0, q, 1.0)
    ep = _t(eps_p) + 1.5 * dp / safe_q * s
    return ep.reshape((9,) + ep.shape[2:]), p + dp


def tangent(H, eps_p, p, lam, mu, sigma_y, h):
    """Consistent tangent K[3i+j, 3k+l] = d sig_ij / d H_kl, shape (9, 9, ...)."""
    sig, s, q = trial(H, eps_p, lam, mu)
    shape = q.shape
    lam = np.broadcast_to(lam, shape)
    mu = np.broadcast_to(mu, shape)
    h = np.broadcast_to(h, shape)
    phi = q - (sigma_y + h * p)
    dp = np.maximum(phi, 0.0) / (3.0 * mu + h)
    d = np.eye(3)
    I_sym = 0.5 * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))
    I_dev = I_sym - np.einsum("ij,kl->ijkl", d, d) / 3.0
    ex = (1,) * len(shape)
    C = (np.einsum("ij,kl->ijkl", d, d).reshape((3, 3, 3, 3) + ex) * lam + 2.0 * mu * I_sym.reshape((3, 3, 3, 3) + ex))
    plastic = phi > 0
    safe_q = np.where(q > 0, q, 1.0)
    snorm = np.sqrt(np.einsum("ij...,ij...->...", s, s))
    N = s / np.where(snorm > 0, snorm, 1.0)
    a = np.where(plastic, 6.0 * mu ** 2 * dp / safe_q, 0.0)
    b = np.where(plastic, 6.0 * mu ** 2 * (dp / safe_q - 1.0 / (3.0 * mu + h)), 0.0)
    K = C - a * I_dev.reshape((3, 3, 3, 3) + ex) + b * np.einsum("ij...,kl...->ijkl...", N, N)
    return K.reshape((9, 9) + shape)
