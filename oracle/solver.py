"""Newton-Krylov solve of the Fourier-Galerkin equilibrium equation (oracle).

Follows Appendix A, Algorithm 1 of the paper with the conjugate-gradient inner
solver it names (Section 3 and Section 4.1.1), applied to the linearised
form of Eq. 1:

    per load increment n (uniform additive steps of the macroscopic tensor):
        F <- F + dFbar                                   (load increment)
        repeat:
            P = P(F), K = K(F)                            (Eqs. 2-3)
            b = -G(P)                                     (right-hand side, Eq. 1)
            solve G(K : dF) = b by CG from dF = 0         (linearised Eq. 1)
            F <- F + dF                                   (update)
            e = ||dF||_2 / (||Fbar_n||_F sqrt(N))          (Alg. 1 convergence test)
            stop when e < tol
    Pbar = mean over voxels of P(F)                       (Eq. 4, midpoint rule)

Readings where the paper is silent or garbled:
* the test quantity "dF / ||Fbar||" is the field 2-norm of dF divided by
  ||Fbar_n||_F sqrt(N), i.e. RMS(dF)/||Fbar_n|| (grid-size independent); when
  ||Fbar_n|| = 0 the denominator is sqrt(N);
* the test is taken after the update, as in Algorithm 1, so a linear problem
  takes two Newton iterations;
* CG starts from zero, uses the Euclidean product over all 9N entries, tests
  ||r|| <= cg_tol ||b|| before each matrix-vector product, and counts products;
  cg_tol defaults to 1e-2 * newton_tol (the inner tolerance is tighter than the
  outer one in both of the paper's examples);
* a zero right-hand side gives dF = 0 without iterating;
* load increments are equal additive steps from the start tensor (I for a
  finite-strain law, 0 for small strain, or the mean of a given start field);
* for J2 plasticity (Section 4.1.2) the stress and tangent of every Newton
  iteration come from the history of the last converged increment, and the
  history advances once the increment has converged (the incremental scheme
  of Appendix B); the reported stress is the return-map stress at the final
  strain from the history before its last update.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import materials as mat
from . import plasticity
from .spectral import project


class NotConverged(RuntimeError):
    pass


@dataclass
class Result:
    F: np.ndarray
    P: np.ndarray
    Pbar: np.ndarray
    newton_residuals: list = field(default_factory=list)
    cg_iterations: list = field(default_factory=list)
    converged: bool = True
    history: np.ndarray | None = None  # J2: (10, ...) plastic strain and cumulative plastic strain


def cg(matvec, b: np.ndarray, tol: float, max_iter: int):
    """Plain conjugate gradients for a symmetric positive operator, x0 = 0.

    Returns (x, number of matrix-vector products, converged flag).
    """
    x = np.zeros_like(b)
    bnorm = math.sqrt(float(np.vdot(b, b)))
    if bnorm == 0.0:
        return x, 0, True
    r = b.copy()
    p = r.copy()
    rr = float(np.vdot(r, r))
    it = 0
    while True:
        if math.sqrt(rr) <= tol * bnorm:
            return x, it, True
        if it >= max_iter:
            return x, it, False
        y = matvec(p)
        it += 1
        py = float(np.vdot(p, y))
        if py <= 0.0:
            return x, it, False
        alpha = rr / py
        x += alpha * p
        r -= alpha * y
        rr_new = float(np.vdot(r, r))
        beta = rr_new / rr
        rr = rr_new
        p = r + beta * p


def voxel_lame(phase, params, scale=None):
    """Per-voxel (lambda, mu): the phase's row of params, times scale if given."""
    lam = params[phase, 0]
    mu = params[phase, 1]
    if scale is not None:
        lam = lam * scale
        mu = mu * scale
    return lam, mu


def reference_tensor(kind: int) -> np.ndarray:
    """Start tensor of a cold solve: I for finite strain, 0 for small strain."""
    return np.eye(3).reshape(9) if mat.FINITE_STRAIN[kind] else np.zeros(9)


def solve(phase: np.ndarray, params: np.ndarray, kind: int, Fbar, n_increments: int = 1,
          newton_tol: float = 1e-10, cg_tol: float | None = None, max_newton: int = 50,
          max_cg: int = 5000, F_init: np.ndarray | None = None, lengths=(1.0, 1.0, 1.0),
          raise_on_failure: bool = True, scale: np.ndarray | None = None,
          plastic: np.ndarray | None = None, history: np.ndarray | None = None) -> Result:
    """Solve the periodic cell under the macroscopic tensor ``Fbar`` (Alg. 1).

    phase: uint8 (nx, ny, nz); params: (n_phase, 2) Lame pairs (lambda, mu);
    Fbar: 9 entries (row-major); F_init: optional start field (9, nx, ny, nz);
    scale: optional per-voxel multiplier of both Lame parameters (a modulus
    field such as E = rho^3 at fixed Poisson ratio).
    J2 only: plastic (n_phase, 2) = (yield stress, hardening modulus) per
    phase; history (10, nx, ny, nz) start plastic strain and cumulative
    plastic strain (zero when None). The advanced history is returned in
    ``Result.history``; the input array is not modified.
    """
    shape = phase.shape
    nvox = phase.size
    lam, mu = voxel_lame(phase, params, scale)
    j2 = kind == mat.J2
    if j2:
        plastic = np.asarray(plastic, dtype=np.float64).reshape(-1, 2)
        sy, hh = plastic[phase, 0], plastic[phase, 1]
        hist = np.zeros((10,) + shape) if history is None else np.array(history, dtype=np.float64)

    def stress_of(F):
        if j2:
            return plasticity.stress(F, hist[:9], hist[9], lam, mu, sy, hh)
        return mat.stress(kind, F, lam, mu)

    def tangent_of(F):
        if j2:
            return plasticity.tangent(F, hist[:9], hist[9], lam, mu, sy, hh)
        return mat.tangent(kind, F, lam, mu)

    Fbar = np.asarray(Fbar, dtype=np.float64).reshape(9)
    if cg_tol is None:
        cg_tol = 1e-2 * newton_tol
    if F_init is None:
        start = reference_tensor(kind)
        F = np.broadcast_to(start.reshape(9, 1, 1, 1), (9,) + shape).copy()
    else:
        F = np.array(F_init, dtype=np.float64).reshape((9,) + shape)
        start = F.reshape(9, -1).mean(axis=1)
    dFbar = (Fbar - start) / n_increments
    res = Result(F=F, P=None, Pbar=None)
    for n in range(1, n_increments + 1):
        Fbar_n = start + n * dFbar
        denom = np.linalg.norm(Fbar_n) * math.sqrt(nvox)
        if denom == 0.0:
            denom = math.sqrt(nvox)
        F += dFbar.reshape(9, 1, 1, 1)
        for _ in range(max_newton):
            P = stress_of(F)
            K = tangent_of(F)
            b = -project(P, lengths)
            dF, ncg, ok = cg(lambda p: project(mat.apply_tangent(K, p), lengths), b, cg_tol, max_cg)
            F += dF
            e = float(np.linalg.norm(dF)) / denom
            res.newton_residuals.append(e)
            res.cg_iterations.append(ncg)
            if not ok:
                res.converged = False
                if raise_on_failure:
                    raise NotConverged("CG did not converge")
                break
            if e < newton_tol:
                break
        else:
            res.converged = False
            if raise_on_failure:
                raise NotConverged("Newton did not converge")
        if j2 and res.converged:
            res.P = stress_of(F)
            eps_p, pc = plasticity.update(F, hist[:9], hist[9], lam, mu, sy, hh)
            hist = np.concatenate([eps_p, pc[None]], axis=0)
    res.F = F
    if not j2 or res.P is None:
        res.P = stress_of(F)
    if j2:
        res.history = hist
    res.Pbar = res.P.reshape(9, -1).mean(axis=1)
    return res


def strain_field(kind: int, F: np.ndarray) -> np.ndarray:
    """The strain measure reported for a solution: sym(H) for small strain, else F."""
    if mat.FINITE_STRAIN[kind]:
        return F
    F3 = F.reshape((3, 3) + F.shape[1:])
    return (0.5 * (F3 + F3.swapaxes(0, 1))).reshape(F.shape)
