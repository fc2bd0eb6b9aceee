"""Pins of the oracle's projection G (Eq. 1) against properties it must have.

None of these re-derives the projection formula: they check algebraic
identities of an orthogonal projection onto compatible fields, analytic
gradients of trigonometric displacement fields, divergence-free fields and
the rank the projection must have on small grids.
"""

import numpy as np
import pytest

from oracle import spectral


def test_wave_integers_fft_order_and_nyquist():
    assert spectral.wave_integers(8).tolist() == [0, 1, 2, 3, 0, -3, -2, -1]
    assert spectral.wave_integers(7).tolist() == [0, 1, 2, 3, -3, -2, -1]
    assert spectral.wave_integers(8, half=True).tolist() == [0, 1, 2, 3, 0]
    assert spectral.wave_integers(7, half=True).tolist() == [0, 1, 2, 3]


def _grid(shape, lengths):
    axes = [(np.arange(n) + 0.5) * L / n for n, L in zip(shape, lengths)]
    return np.meshgrid(*axes, indexing="ij")


@pytest.mark.parametrize("shape,lengths", [((6, 8, 5), (1, 1, 1)), ((4, 4, 4), (1, 1, 1)),
                                           ((5, 6, 8), (1.0, 2.0, 0.5))])
def test_projection_idempotent_and_symmetric(shape, lengths):
    rng = np.random.default_rng(1)
    A = rng.standard_normal((9,) + shape)
    B = rng.standard_normal((9,) + shape)
    GA = spectral.project(A, lengths)
    GB = spectral.project(B, lengths)
    np.testing.assert_allclose(spectral.project(GA, lengths), GA, atol=1e-13)
    assert abs(np.vdot(GA, B) - np.vdot(A, GB)) < 1e-11 * np.linalg.norm(A) * np.linalg.norm(B)
    # the complement is orthogonal to the range
    assert abs(np.vdot(GA, A - GA)) < 1e-11 * np.vdot(A, A)


@pytest.mark.parametrize("shape,lengths", [((8, 8, 8), (1, 1, 1)), ((6, 7, 8), (1.0, 2.0, 0.5))])
def test_projection_keeps_analytic_gradients(shape, lengths):
    """u_i = a_i sin(2 pi m.x/L + phi) has grad u = a (x) (2 pi m / L) cos(...): G keeps it."""
    X = _grid(shape, lengths)
    rng = np.random.default_rng(2)
    H = np.zeros((3, 3) + shape)
    for m in [(1, 0, 0), (1, -2, 3), (0, 2, -1), (2, 1, 1)]:
        a = rng.standard_normal(3)
        phi = rng.uniform(0, 2 * np.pi)
        q = [2 * np.pi * m[d] / lengths[d] for d in range(3)]
        arg = q[0] * X[0] + q[1] * X[1] + q[2] * X[2] + phi
        for i in range(3):
            for j in range(3):
                H[i, j] += a[i] * q[j] * np.cos(arg)
    H = H.reshape((9,) + shape)
    np.testing.assert_allclose(spectral.project(H, lengths), H, atol=1e-12 * np.abs(H).max())


def test_projection_removes_constants_and_divergence_free_rows():
    shape = (8, 6, 7)
    X = _grid(shape, (1, 1, 1))
    A = np.zeros((3, 3) + shape)
    rng = np.random.default_rng(3)
    A += rng.standard_normal((3, 3))[:, :, None, None, None]  # constant part
    for m in [(1, 2, 0), (0, 1, 3), (2, -1, 1)]:
        m = np.array(m, dtype=float)
        c = np.cross(m, rng.standard_normal(3))  # c . m = 0: each row is divergence free
        b = rng.standard_normal(3)
        arg = 2 * np.pi * (m[0] * X[0] + m[1] * X[1] + m[2] * X[2])
        A += np.einsum("i,j->ij", b, c)[:, :, None, None, None] * np.sin(arg)
    A = A.reshape((9,) + shape)
    assert np.abs(spectral.project(A)).max() < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("shape,zero_modes", [((4, 4, 4), 8), ((3, 3, 3), 1), ((4, 3, 2), 4)])
def test_projection_rank(shape, zero_modes):
    """Dense matrix of G: eigenvalues in {0, 1}, rank 3 x (modes with xi != 0).

    On an even axis the Nyquist index has xi = 0, so the number of frequencies
    with xi = 0 is 2^(number of even axes).
    """
    N = int(np.prod(shape))
    M = np.zeros((9 * N, 9 * N))
    for c in range(9 * N):
        e = np.zeros(9 * N)
        e[c] = 1.0
        M[:, c] = spectral.project(e.reshape((9,) + shape)).reshape(-1)
    np.testing.assert_allclose(M, M.T, atol=1e-13)
    w = np.linalg.eigvalsh(M)
    assert np.all(np.minimum(np.abs(w), np.abs(w - 1)) < 1e-12)
    assert round(float(np.trace(M))) == 3 * (N - zero_modes)
