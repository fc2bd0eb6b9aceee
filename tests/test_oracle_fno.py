"""Pins of the oracle's factorized FNO (learned warm start).

* parameter layout: 352 lifting + 4 x 74784 layer + 14673 projection entries;
* one spectral layer on a single Fourier mode along x (constant along y, z)
  returns the closed form Re(W^x_m[o,c] e^{i theta}) + Re(W^y_0 + W^z_0)[o,c] cos theta,
  and a mode above the retained ones contributes only through y and z;
* the network commutes with periodic shifts of the input;
* with every spectral weight zero it is a per-voxel network, checked voxel by
  voxel against an explicit evaluation;
* gradients of the loss (autograd) against central finite differences of
  the loss for entries of every parameter block.
"""

import math

import numpy as np
import pytest
import torch

from oracle import fno

N = 24


def _theta(seed, spectral_scale=0.02):
    g = torch.Generator().manual_seed(seed)
    th = torch.empty(fno.n_params(), dtype=torch.float64)
    o = 0
    for name, shape in fno.layout():
        k = math.prod(shape)
        sc = spectral_scale if name.startswith("W") else 1.0 / math.sqrt(shape[-1])
        th[o:o + k] = (2 * torch.rand(k, generator=g, dtype=torch.float64) - 1) * sc
        o += k
    return th


def _inputs(seed, B=2, shape=(N, N, N)):
    rng = np.random.default_rng(seed)
    phi = torch.as_tensor((rng.uniform(size=(B,) + shape) < 0.3).astype(np.float64))
    dF = rng.uniform(-1, 1, size=(B, 9))
    dF *= 0.05 / np.linalg.norm(dF, axis=1, keepdims=True)
    Fbar = torch.as_tensor(np.eye(3).reshape(1, 9) + dF)
    return phi, Fbar


def test_parameter_layout():
    assert fno.n_params() == 352 + 4 * (3 * 12 * 2 * 32 * 32 + 32 * 32 + 32) + (128 * 32 + 128 + 81 * 128 + 81)
    p = fno.unpack(torch.arange(fno.n_params(), dtype=torch.float64))
    assert p["p2"][-1] == fno.n_params() - 1


@pytest.mark.parametrize("m", [3, 11, 12])
def test_spectral_layer_single_mode_closed_form(m):
    rng = np.random.default_rng(m)
    W = torch.as_tensor(rng.uniform(-1, 1, size=(3, fno.MODES, 2, 32, 32)))
    c = 5
    x = np.arange(N)
    theta = 2 * np.pi * m * x / N
    h = torch.zeros(1, 32, N, N, N, dtype=torch.float64)
    h[0, c] = torch.as_tensor(np.cos(theta))[:, None, None]
    S = sum(fno.spectral_axis(h, W[d], 2 + d) for d in range(3))[0]  # (32, N, N, N)
    Wn = W.numpy()
    yz = (Wn[1, 0, 0, :, c] + Wn[2, 0, 0, :, c])[:, None] * np.cos(theta)[None]
    if m < fno.MODES:
        xm = Wn[0, m, 0, :, c][:, None] * np.cos(theta)[None] - Wn[0, m, 1, :, c][:, None] * np.sin(theta)[None]
    else:
        xm = 0.0
    expect = xm + yz
    for j, k in [(0, 0), (7, 3), (N - 1, 11)]:
        np.testing.assert_allclose(S[:, :, j, k].numpy(), expect, rtol=0, atol=1e-12)


def test_shift_equivariance():
    th = _theta(1)
    phi, Fbar = _inputs(2, B=1, shape=(N, 32, N))
    q, _ = fno.forward(th, phi, Fbar)
    sh = (3, -5, 7)
    q2, _ = fno.forward(th, torch.roll(phi, sh, dims=(1, 2, 3)), Fbar)
    np.testing.assert_allclose(q2.numpy(), torch.roll(q, sh, dims=(2, 3, 4)).numpy(), rtol=0, atol=1e-12)


def test_zero_spectral_weights_is_a_voxel_network():
    th = _theta(3)
    p = fno.unpack(th)
    for l in range(fno.LAYERS):
        p[f"W{l}"].zero_()
    phi, Fbar = _inputs(4, B=1)
    q, s = fno.forward(th, phi, Fbar)
    P = {k: v.numpy() for k, v in p.items()}
    gelu = np.vectorize(lambda z: 0.5 * z * (1.0 + math.erf(z / math.sqrt(2.0))))
    dF = Fbar.numpy()[0] - np.eye(3).reshape(9)
    u = dF / np.linalg.norm(dF)
    for v in [(0, 0, 0), (5, 17, 2), (23, 23, 23)]:
        h = P["a"] * float(phi[0][v]) + P["B"] @ u + P["b0"]
        for l in range(fno.LAYERS):
            z = P[f"M{l}"] @ h + P[f"m{l}"]
            h = gelu(z) if l < fno.LAYERS - 1 else z
        R = (P["P2"] @ gelu(P["P1"] @ h + P["p1"]) + P["p2"]).reshape(9, 9)
        out = np.array([sum(R[i, j] * u[j] for j in range(9)) for i in range(9)])
        np.testing.assert_allclose(q[0][(slice(None),) + v].numpy(), out, rtol=1e-12, atol=1e-12)


def test_loss_gradient_matches_finite_differences():
    th = _theta(5)
    phi, Fbar = _inputs(6, B=2)
    rng = np.random.default_rng(7)
    target = torch.as_tensor(rng.normal(size=(2, 9, N, N, N)) * 0.3)
    L, g = fno.loss_and_grad(th, phi, Fbar, target)
    assert L > 0
    starts = {}
    o = 0
    for name, shape in fno.layout():
        starts[name] = (o, math.prod(shape))
        o += math.prod(shape)
    idx = []
    for name, (o, k) in starts.items():
        idx += list(o + rng.choice(k, size=min(2, k), replace=False))
    h = 1e-6
    for i in idx:
        tp = th.clone(); tp[i] += h
        tm = th.clone(); tm[i] -= h
        fd = (float(fno.loss(tp, phi, Fbar, target)) - float(fno.loss(tm, phi, Fbar, target))) / (2 * h)
        assert abs(fd - float(g[i])) <= 1e-8 * max(1.0, abs(fd)), (i, fd, float(g[i]))


def test_adam_first_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2: the step is lr g / (|g| + eps) (+ lr wd theta)."""
    rng = np.random.default_rng(8)
    th = rng.normal(size=50)
    g = rng.normal(size=50) * 1e-3
    z = np.zeros(50)
    lr, eps, wd = 1e-3, 1e-8, 0.01
    t1, m1, v1 = fno.adam_step(th, g, z, z, 1, lr, eps=eps, wd=wd)
    np.testing.assert_allclose(t1, th - lr * (g / (np.abs(g) + eps) + wd * th), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)
    # a constant gradient keeps the bias-corrected moments at g and g^2 at every step
    t2, m2, v2 = fno.adam_step(t1, g, m1, v1, 2, lr, eps=eps)
    np.testing.assert_allclose(t2, t1 - lr * g / (np.abs(g) + eps), rtol=1e-10, atol=1e-15)


def test_prediction_is_odd_in_the_load_direction_when_the_body_ignores_it():
    """With B = 0 the body sees only phi, and q = R(phi) u changes sign with u."""
    th = _theta(9)
    fno.unpack(th)["B"].zero_()
    phi, Fbar = _inputs(10, B=1)
    d = Fbar - torch.eye(3, dtype=torch.float64).reshape(1, 9)
    qp, _ = fno.forward(th, phi, torch.eye(3, dtype=torch.float64).reshape(1, 9) + d)
    qm, _ = fno.forward(th, phi, torch.eye(3, dtype=torch.float64).reshape(1, 9) - d)
    np.testing.assert_allclose(qp.numpy(), -qm.numpy(), rtol=0, atol=1e-12)
    assert float(qp.abs().max()) > 1e-3
