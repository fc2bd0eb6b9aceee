"""Dense energy minimisation on tiny grids (an independent pin of the solver).

The Fourier-Galerkin solution of Eq. 1 is the minimiser of the discrete
energy sum_x W(Fbar + grad u (x)) over periodic displacement fluctuations u,
where grad is the spectral first derivative: the fields G keeps are exactly
the spectral gradients, so G(P) = 0 is the stationarity condition
grad^T P = 0. This module rebuilds that minimiser by a route that shares
nothing with ``solver``: the derivative matrices come from the explicit DFT
sum (no FFT library, no projection operator), and the minimisation is a
dense Newton iteration with least-squares steps (no conjugate gradients).

Wave numbers: k in FFT order; the Nyquist index of an even axis differentiates
to zero (the same convention as the projection, restated here).
"""

from __future__ import annotations

import numpy as np

from . import materials as mat


def derivative_matrix(n: int, length: float = 1.0) -> np.ndarray:
    """Real n x n matrix D with (D u)_m = spectral derivative of u at point m.

    D[m, p] = (1/n) sum_j (i xi_j) exp(2 pi i k_j (m - p) / n), written as an
    explicit sum over the n wave numbers.
    """
    D = np.zeros((n, n), dtype=np.complex128)
    m = np.arange(n)
    for j in range(n):
        k = j if 2 * j < n else j - n
        if 2 * j == n:
            continue  # the Nyquist mode has zero derivative
        xi = 2.0 * np.pi * k / length
        ph = np.exp(2j * np.pi * k * (m[:, None] - m[None, :]) / n)
        D += (1j * xi / n) * ph
    assert np.max(np.abs(D.imag)) < 1e-10
    return D.real.copy()


def gradient_operator(shape, lengths=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Dense (9N, 3N) matrix mapping u (3, nx, ny, nz) to H_ij = d u_i / d x_j."""
    nx, ny, nz = shape
    N = nx * ny * nz
    Ds = [
        np.kron(np.kron(derivative_matrix(nx, lengths[0]), np.eye(ny)), np.eye(nz)),
        np.kron(np.kron(np.eye(nx), derivative_matrix(ny, lengths[1])), np.eye(nz)),
        np.kron(np.kron(np.eye(nx), np.eye(ny)), derivative_matrix(nz, lengths[2])),
    ]
    Gr = np.zeros((9 * N, 3 * N))
    for i in range(3):
        for j in range(3):
            Gr[(3 * i + j) * N:(3 * i + j + 1) * N, i * N:(i + 1) * N] = Ds[j]
    return Gr


def minimise(phase: np.ndarray, params: np.ndarray, kind: int, Fbar, lengths=(1.0, 1.0, 1.0),
             tol: float = 1e-14, max_iter: int = 40) -> np.ndarray:
    """Minimise sum_x W(Fbar + grad u) by dense Newton steps; return F (9, nx, ny, nz)."""
    shape = phase.shape
    N = phase.size
    lam = params[phase.reshape(-1), 0]
    mu = params[phase.reshape(-1), 1]
    Gr = gradient_operator(shape, lengths)
    Fbar = np.asarray(Fbar, dtype=np.float64).reshape(9, 1)
    u = np.zeros(3 * N)
    for _ in range(max_iter):
        F = Fbar + (Gr @ u).reshape(9, N)
        P = mat.stress(kind, F, lam, mu)
        K = mat.tangent(kind, F, lam, mu)          # (9, 9, N)
        g = Gr.T @ P.reshape(-1)
        KG = np.einsum("abn,bnc->anc", K, Gr.reshape(9, N, 3 * N)).reshape(9 * N, 3 * N)
        H = Gr.T @ KG
        du = np.linalg.lstsq(H, -g, rcond=1e-12)[0]
        u += du
        if np.linalg.norm(du) <= tol * max(1.0, np.linalg.norm(u)):
            break
    return (Fbar + (Gr @ u).reshape(9, N)).reshape((9,) + shape)
