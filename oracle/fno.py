"""Factorized Fourier neural operator for the learned warm start (oracle).

TEST INFRASTRUCTURE (like the rest of ``oracle/``). A plain PyTorch CPU
float64 restatement of the network the GPU library trains and evaluates:
it maps a two-phase indicator field phi (1 = inclusion) and a macroscopic
tensor Fbar to a predicted fluctuation field F - Fbar, which the solver then
refines (Algorithm 1 started from the prediction instead of from Fbar).

Architecture (the reading of "4 layers, width 32, 12 retained modes per
axis" taken here: the spectral weights act per axis, one 32x32 complex matrix
per retained mode and axis, so each layer keeps 12 modes along x, along y and
along z; a full 12^3-mode kernel would have ~7M complex weights per layer):

    s = |Fbar - I|_F,  u = (Fbar - I) / s                (unit load direction)
    h0(x)  = a phi(x) + B u + b0                          (lifting, width 32)
    z_l    = sum_{d in x,y,z} S_{l,d}(h_l) + M_l h_l + m_l,  l = 0..3
    h_l+1  = gelu(z_l) for l < 3,  h_4 = z_3
    R(x)   = P2 gelu(P1 h_4 + p1) + p2                    (projection, 81 outputs R_ij)
    q_i(x) = sum_j R_ij(x) u_j                            (response to the load direction)
    F - Fbar ~ s q(x)

    S_{l,d}(h) = irfft_d( W_{l,d}[k] rfft_d(h)[k] for k < 12, zero above ),

with rfft/irfft along axis d alone (unnormalised forward, 1/n inverse, the
imaginary part of the k = 0 term dropped as irfft does) and
W_{l,d}[k] a complex 32x32 matrix acting on the channel vector. gelu is the
exact form z Phi(z). The head predicts a 9x9 response per voxel and applies
it to u, so the prediction is linear in the load direction for a given
microstructure, as the cell response is to first order in |Fbar - I|. The loss is the mean squared error against the solver's
normalised fluctuation (F - Fbar)/s over samples, components and voxels.

Parameters live in one flat vector (float64 here, the GPU stores float32
masters and bfloat16 copies); ``layout()`` gives the slices. Gradients come
from torch.autograd; the tests pin them against central finite differences,
the spectral layer against its closed form on single Fourier modes, the whole
map against translation equivariance and, with all spectral weights zero,
against a per-voxel evaluation.
"""

from __future__ import annotations

import math

import torch

WIDTH = 32
LAYERS = 4
MODES = 12
HIDDEN = 128
N_OUT = 9
N_HEAD = N_OUT * 9


def layout():
    """Ordered (name, shape) of the flat parameter vector."""
    items = [("a", (WIDTH,)), ("B", (WIDTH, 9)), ("b0", (WIDTH,))]
    for l in range(LAYERS):
        items += [(f"W{l}", (3, MODES, 2, WIDTH, WIDTH)), (f"M{l}", (WIDTH, WIDTH)), (f"m{l}", (WIDTH,))]
    items += [("P1", (HIDDEN, WIDTH)), ("p1", (HIDDEN,)), ("P2", (N_HEAD, HIDDEN)), ("p2", (N_HEAD,))]
    return items


def n_params() -> int:
    return sum(math.prod(s) for _, s in layout())


def unpack(theta: torch.Tensor) -> dict:
    out, o = {}, 0
    for name, shape in layout():
        k = math.prod(shape)
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def gelu(z):
    return 0.5 * z * (1.0 + torch.erf(z / math.sqrt(2.0)))


def spectral_axis(h: torch.Tensor, W: torch.Tensor, dim: int) -> torch.Tensor:
    """S_d(h) for h (B, C, nx, ny, nz) along spatial ``dim`` (2, 3 or 4); W (MODES, 2, C_out, C_in)."""
    n = h.shape[dim]
    if n < 2 * MODES:
        raise ValueError(f"axis length {n} < {2 * MODES}: the retained modes must lie below the Nyquist index")
    X = torch.fft.rfft(h, dim=dim).narrow(dim, 0, MODES)
    m = MODES
    Wc = torch.complex(W[:, 0], W[:, 1])  # (MODES, out, in)
    Xm = X.movedim(dim, -1)                  # (B, C, a, b, m)
    Y = torch.einsum("koc,bcxyk->boxyk", Wc, Xm)
    pad = n // 2 + 1 - m
    Y = torch.cat([Y, torch.zeros(Y.shape[:-1] + (pad,), dtype=Y.dtype)], dim=-1)
    return torch.fft.irfft(Y.movedim(-1, dim), n=n, dim=dim)


def forward(theta: torch.Tensor, phi: torch.Tensor, Fbar: torch.Tensor, return_all: bool = False):
    """Normalised prediction q (B, 9, nx, ny, nz) and the scale s (B,).

    phi: (B, nx, ny, nz) in {0, 1}; Fbar: (B, 9).
    """
    p = unpack(theta)
    eye = torch.eye(3, dtype=Fbar.dtype).reshape(9)
    dF = Fbar - eye
    s = torch.linalg.norm(dF, dim=1)
    u = dF / s[:, None]
    h = p["a"][None, :, None, None, None] * phi[:, None] + (u @ p["B"].T + p["b0"])[:, :, None, None, None]
    for l in range(LAYERS):
        W = p[f"W{l}"]
        z = sum(spectral_axis(h, W[d], 2 + d) for d in range(3))
        z = z + torch.einsum("oc,bcxyz->boxyz", p[f"M{l}"], h) + p[f"m{l}"][None, :, None, None, None]
        h = gelu(z) if l < LAYERS - 1 else z
    t = gelu(torch.einsum("oc,bcxyz->boxyz", p["P1"], h) + p["p1"][None, :, None, None, None])
    R = torch.einsum("oc,bcxyz->boxyz", p["P2"], t) + p["p2"][None, :, None, None, None]
    R = R.reshape((R.shape[0], N_OUT, 9) + R.shape[2:])
    q = torch.einsum("bijxyz,bj->bixyz", R, u)
    return q, s


def loss(theta, phi, Fbar, target):
    """Mean squared error of q against target (B, 9, nx, ny, nz) (normalised fluctuation)."""
    q, _ = forward(theta, phi, Fbar)
    return ((q - target) ** 2).mean()


def loss_and_grad(theta, phi, Fbar, target):
    th = theta.detach().clone().requires_grad_(True)
    L = loss(th, phi, Fbar, target)
    (g,) = torch.autograd.grad(L, th)
    return float(L.detach()), g


def predict(theta, phi, Fbar):
    """Predicted fluctuation F - Fbar (B, 9, nx, ny, nz)."""
    q, s = forward(theta, phi, Fbar)
    return q * s[:, None, None, None, None]


def adam_step(theta, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8,
              wd: float = 0.0):
    """One Adam step (Kingma and Ba, Algorithm 1) with decoupled weight decay.

    Returns the new (theta, m, v); arrays are float64 numpy arrays.
    """
    import numpy as np

    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    theta = theta - lr * (mhat / (np.sqrt(vhat) + eps) + wd * theta)
    return theta, m, v
