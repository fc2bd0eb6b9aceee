"""torch.autograd.Function wrappers over the C-ABI (Section 3.3, Section 4.4.2).

* Pbar(Fbar) of a neo-Hookean cell: the gradient of w . Pbar with respect to
  Fbar equals Cbar^T w with Cbar the oracle's homogenized tangent at its own
  converged state (1e-8 relative), and central finite differences of two
  solves (step 1e-6, relative 1e-5);
* Cbar_1212(rho) of a SIMP cell: the gradient with respect to the voxel
  density equals the oracle's sensitivity field (1e-8 max-relative);
* Pbar(rho) of a finite-strain SIMP cell under a fixed Fbar: the gradient of
  w . Pbar equals sum_ab w_ab of the oracle's stress sensitivity fields
  (1e-8 max-relative) and central differences of two solves at a voxel.
"""

import numpy as np
import pytest

from gpu_helpers import dev, field_maxrel, host, require_gpu
from oracle import homogenize, solver as osolver
from rve_inputs import random_spheres, shear_macro, simp_config, two_phase_table

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fh():
    require_gpu()
    import paper_2408_03804_gb300 as fh

    return fh


def test_stress_gradient_is_homogenized_tangent(fh):
    import torch

    from paper_2408_03804_gb300.autograd import homogenized_stress

    n = 16
    phase = random_spheres(n, seed=2, r_min=2.0, r_max=3.0)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar0 = shear_macro(0.03, finite=True)
    w = np.random.default_rng(0).uniform(-1, 1, 9)
    opts = fh.default_options(newton_tol=1e-12)
    topt = fh.default_options(cg_tol=1e-12)
    with fh.Context(n, n, n) as ctx:
        mat = fh.Material(1, phase, params)
        F = torch.zeros((9, n, n, n), dtype=torch.float64, device="cuda")
        Fbar = torch.tensor(Fbar0, dtype=torch.float64, requires_grad=True)
        P = homogenized_stress(Fbar, ctx, mat, F, 2, opts, topt)
        (P * torch.as_tensor(w)).sum().backward()
        g = Fbar.grad.numpy()
        # finite differences: two warm-started solves per direction
        h = 1e-6
        fd = np.zeros(9)
        Fc = F.clone()
        for c in range(9):
            vals = []
            for sgn in (1.0, -1.0):
                Fb = Fbar0.copy()
                Fb[c] += sgn * h
                Fw = Fc.clone()
                pb, _, _ = ctx.fft_homog_solve(mat, Fb, Fw, options=fh.default_options(
                    newton_tol=1e-13, init=fh.INIT_GIVEN), allow=(fh.FH_ERR_NOT_CONVERGED,))
                vals.append(pb @ w)
            fd[c] = (vals[0] - vals[1]) / (2 * h)
    ref = osolver.solve(phase, params, 1, Fbar0, n_increments=2, newton_tol=1e-12)
    C_ref = homogenize.tangent(phase, params, 1, ref.F, cg_tol=1e-12)
    np.testing.assert_allclose(g, C_ref.T @ w, rtol=0, atol=1e-8 * np.abs(C_ref.T @ w).max())
    np.testing.assert_allclose(g, fd, rtol=0, atol=1e-5 * np.abs(fd).max())


def test_modulus_gradient_is_sensitivity_field(fh):
    import torch

    from paper_2408_03804_gb300.autograd import homogenized_modulus

    n = 16
    phase, params, rho, scale, dscale = simp_config(n, seed=3)
    with fh.Context(n, n, n) as ctx:
        mat = fh.Material(0, phase, params, scale=scale)
        r = torch.tensor(rho, dtype=torch.float64, device="cuda", requires_grad=True)
        c = homogenized_modulus(r, ctx, mat, (0, 1, 0, 1), dev(dscale), fh.default_options(cg_tol=1e-13))
        c.backward()
        grad = host(r.grad)
    C_ref = homogenize.tangent(phase, params, 0, np.zeros((9,) + phase.shape), scale=scale, cg_tol=1e-13)
    np.testing.assert_allclose(float(c), C_ref[1, 1], rtol=1e-9)
    ref = homogenize.sensitivity(phase, params, scale, dscale, 1, 1, cg_tol=1e-13)
    assert field_maxrel(grad[None], ref[None]) < 1e-8


def test_stress_of_density_gradient_is_weighted_stress_sensitivity(fh):
    import torch

    from paper_2408_03804_gb300.autograd import homogenized_stress_of_density

    n = 12
    rho = 0.35 + 0.65 * simp_config(n, seed=4)[2]
    scale, dscale = rho ** 3, 3.0 * rho ** 2
    phase = np.zeros((n, n, n), np.uint8)
    params = np.array([[1.5, 1.0]])
    Fbar = shear_macro(0.05, finite=True)
    w = np.random.default_rng(2).uniform(-1, 1, 9)
    opts = fh.default_options(newton_tol=1e-12, cg_tol=1e-13)
    with fh.Context(n, n, n) as cell:
        mat = fh.Material(fh.NEO_HOOKEAN, phase, params, scale=dev(scale))
        F = torch.zeros((9, n, n, n), dtype=torch.float64, device="cuda")
        r = torch.tensor(rho, dtype=torch.float64, device="cuda", requires_grad=True)
        pbar = homogenized_stress_of_density(r, cell, mat, Fbar, F, dev(dscale), options=opts,
                                             adjoint_options=fh.default_options(cg_tol=1e-13))
        (pbar * torch.as_tensor(w, device="cuda")).sum().backward()
        grad = host(r.grad)
        ref = sum(w[ab] * homogenize.stress_sensitivity(phase, params, 1, host(F), scale, dscale, ab, cg_tol=1e-13)
                  for ab in range(9))
        assert field_maxrel(grad[None], ref[None]) < 1e-8

        def wpbar(rr):
            Fs = torch.zeros_like(F)
            p, _, _ = cell.fft_homog_solve(fh.Material(fh.NEO_HOOKEAN, phase, params, scale=dev(rr ** 3)), Fbar,
                                           Fs, options=opts)
            return float(w @ p)

        v = (3, 7, 1)
        h = 1e-4
        rp, rm = rho.copy(), rho.copy()
        rp[v] += h
        rm[v] -= h
        fd = (wpbar(rp) - wpbar(rm)) / (2 * h)
        assert abs(fd - grad[v]) <= 1e-5 * abs(grad[v]) + 1e-7 * np.abs(grad).max()
