"""Wave vectors and the compatibility projection G of the Fourier-Galerkin method.

Eq. 1 (Section 3) writes equilibrium as IFFT{ Ghat(xi) : FFT{P} } = 0, where G
maps an arbitrary tensor field to its compatible (periodic, curl-free) part;
its explicit form is delegated to the cited literature. The form used here is
the standard one for a 3x3 field A with Fourier coefficients Ahat(xi):

    Ghat(xi)[Ahat] = (Ahat xi) (x) xi / (xi . xi)   for xi != 0,
    Ghat(0)        = 0,

i.e. entry (i, j) of the result is sum_l Ahat_il xi_l xi_j / |xi|^2. Per
frequency this is right-multiplication by the projector xi xi^T/|xi|^2, so it
is symmetric and idempotent under the Frobenius product, it keeps gradients
(a (x) xi) and removes divergence-free rows (Ahat xi = 0).

Reading for even grids (the paper uses odd grids only, Section 4.1.1): on an
axis with an even number of points the Nyquist index k = n/2 gets the wave
number xi = 0, the usual convention for a first spectral derivative. Then
xi(-k) = -xi(k) on every index, Ghat preserves Hermitian symmetry, G maps real
fields to real fields and stays an orthogonal projection.

Layout: fields are float64 arrays of shape (9, nx, ny, nz), component 3*i + j.
"""

from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft

_WORKERS = os.cpu_count() or 1


def wave_integers(n: int, half: bool = False) -> np.ndarray:
    """Signed wave integers k of an n-point axis in FFT order, Nyquist set to 0.

    ``half`` gives the non-negative half used by a real-to-complex transform
    (n // 2 + 1 entries).
    """
    m = n // 2 + 1 if half else n
    j = np.arange(m)
    k = np.where(j <= (n - 1) // 2, j, j - n).astype(np.float64)
    if n % 2 == 0:
        k[j == n // 2] = 0.0
    return k


def wave_vectors(shape: tuple[int, int, int], lengths=(1.0, 1.0, 1.0)):
    """Broadcastable wave-vector components (xi_x, xi_y, xi_z) on the half spectrum.

    xi_a = 2 pi k_a / L_a with k_a from :func:`wave_integers`; the last axis is
    the half axis of ``scipy.fft.rfftn``.
    """
    nx, ny, nz = shape
    xx = 2 * np.pi * wave_integers(nx) / lengths[0]
    xy = 2 * np.pi * wave_integers(ny) / lengths[1]
    xz = 2 * np.pi * wave_integers(nz, half=True) / lengths[2]
    return xx[:, None, None], xy[None, :, None], xz[None, None, :]


def apply_ghat(Ahat: np.ndarray, xi) -> np.ndarray:
    """Apply Ghat(xi) to a spectrum of shape (9, ...) (Eq. 1).

    Returns (Ahat xi) (x) xi / |xi|^2 per frequency and 0 where xi = 0.
    """
    xs = np.broadcast_arrays(*xi)
    xi2 = xs[0] ** 2 + xs[1] ** 2 + xs[2] ** 2
    inv = np.zeros_like(xi2)
    nz = xi2 > 0
    inv[nz] = 1.0 / xi2[nz]
    A = Ahat.reshape((3, 3) + Ahat.shape[1:])
    out = np.empty_like(A)
    for i in range(3):
        v = (A[i, 0] * xs[0] + A[i, 1] * xs[1] + A[i, 2] * xs[2]) * inv
        for j in range(3):
            out[i, j] = v * xs[j]
    return out.reshape(Ahat.shape)


def project(A: np.ndarray, lengths=(1.0, 1.0, 1.0), workers: int | None = None) -> np.ndarray:
    """G(A) = IFFT{ Ghat : FFT{A} } for a real field A of shape (9, nx, ny, nz) (Eq. 1)."""
    shape = A.shape[1:]
    w = workers or _WORKERS
    Ahat = sfft.rfftn(A, axes=(1, 2, 3), workers=w)
    Ahat = apply_ghat(Ahat, wave_vectors(shape, lengths))
    return sfft.irfftn(Ahat, s=shape, axes=(1, 2, 3), workers=w)
