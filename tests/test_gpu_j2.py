"""J2 elastoplasticity on the GPU against the oracle (Section 4.1.2, Appendix B).

* stress and packed tangent of fh_constitutive (AD of the return map) against
  the oracle's return map and closed-form consistent tangent, over voxels in
  the elastic and the plastic regime, with a stress-free voxel, at 1e-12;
* full solves with history: the 2D biaxial cell with hard disks (z-invariant,
  nz = 2) in ten increments and a 3D cell of random spheres under shear, in
  both tangent modes: homogenized stress at 1e-9, strain and plastic-strain
  fields at 1e-8 (max-relative), equal Newton counts;
* the history carries over between calls: loading then partial unloading in
  two solves matches the oracle's two solves;
* the entry points that J2 does not support refuse it with an error code.
"""

import numpy as np
import pytest

from gpu_helpers import dev, field_maxrel, host, pack_tangent, require_gpu
from oracle import materials as omat, plasticity as pl, solver as osolver
from rve_inputs import j2_config, random_spheres

pytestmark = pytest.mark.gpu

OP_TOL = 1e-12
FIELD_TOL = 1e-8
PBAR_TOL = 1e-9


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


@pytest.fixture(scope="module")
def fh(torch):
    import paper_2408_03804_gb300 as fh

    return fh


def _sym(A):
    A3 = A.reshape((3, 3) + A.shape[1:])
    return (0.5 * (A3 + A3.swapaxes(0, 1))).reshape(A.shape)


def test_j2_constitutive_matches_return_map(fh, torch):
    shape = (8, 6, 4)
    n = int(np.prod(shape))
    rng = np.random.default_rng(5)
    H = rng.uniform(-0.01, 0.01, size=(9, n))
    ep = _sym(rng.uniform(-0.002, 0.002, size=(9, n)))
    ep[0] -= (ep[0] + ep[4] + ep[8]) / 3  # plastic strain is deviatoric
    p = rng.uniform(0.0, 0.01, size=n)
    H[:, 0] = 0.0
    ep[:, 0] = 0.0
    p[0] = 0.0  # stress-free voxel: the q = 0 branch
    phase = rng.integers(0, 2, size=n).astype(np.uint8)
    params = np.array([[1.2, 0.8], [2.4, 1.6]])
    plastic = np.array([[0.02, 0.2], [0.04, 0.4]])
    lam, mu = params[phase, 0], params[phase, 1]
    sy, hh = plastic[phase, 0], plastic[phase, 1]
    P_ref = pl.stress(H, ep, p, lam, mu, sy, hh)
    K_ref = pl.tangent(H, ep, p, lam, mu, sy, hh)
    plastic_vox = (pl.update(H, ep, p, lam, mu, sy, hh)[1] > p)
    assert 0.2 < plastic_vox.mean() < 0.8, "the case should mix elastic and plastic voxels"
    hist = np.concatenate([ep, p[None]], axis=0).reshape((10,) + shape)
    with fh.Context(*shape) as ctx:
        mat = fh.Material(fh.J2, phase.reshape(shape), params, plastic=plastic, history=dev(hist))
        Hd = dev(H.reshape((9,) + shape))
        P = torch.empty_like(Hd)
        K = torch.empty((45,) + shape, dtype=torch.float64, device="cuda")
        ctx.fh_constitutive(mat, Hd, P, K)
    Pg = host(P).reshape(9, n)
    Kg = host(K).reshape(45, n)
    assert np.abs(Pg - P_ref).max() <= OP_TOL * np.abs(P_ref).max()
    Kp = pack_tangent(K_ref)
    assert np.abs(Kg - Kp).max() <= OP_TOL * np.abs(Kp).max()


def _j2_solve_both(fh, torch, phase, params, plastic, Ebar, n_inc, tol, tangent_mode=0):
    shape = phase.shape
    with fh.Context(*shape) as ctx:
        hist = torch.zeros((10,) + shape, dtype=torch.float64, device="cuda")
        mat = fh.Material(fh.J2, phase, params, plastic=plastic, history=hist)
        F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        opts = fh.default_options(newton_tol=tol, tangent_mode=tangent_mode, check_every=4)
        pbar, stats, _ = ctx.fft_homog_solve(mat, Ebar, F, n_increments=n_inc, options=opts)
        Fg, hg = host(F), host(hist)
    ref = osolver.solve(phase, params, omat.J2, Ebar, n_increments=n_inc, newton_tol=tol, plastic=plastic)
    return Fg, hg, pbar, stats, ref


def _check(Fg, hg, pbar, stats, ref):
    assert stats["n_newton"] == len(ref.newton_residuals)
    assert all(abs(a - b) <= 1 for a, b in zip(stats["cg_iterations"], ref.cg_iterations))
    np.testing.assert_allclose(pbar, ref.Pbar, rtol=PBAR_TOL, atol=PBAR_TOL * np.abs(ref.Pbar).max())
    assert field_maxrel(_sym(Fg), _sym(ref.F)) < FIELD_TOL
    assert field_maxrel(hg, ref.history) < FIELD_TOL


def test_j2_biaxial_disks_2d_matches_oracle(fh, torch):
    phase, params, plastic, Ebar = j2_config(48, 0, nz=2)
    Fg, hg, pbar, stats, ref = _j2_solve_both(fh, torch, phase, params, plastic, Ebar, 10, 1e-8)
    assert ref.history[9].max() > 0
    _check(Fg, hg, pbar, stats, ref)


@pytest.mark.parametrize("tangent_mode", [0, 1])
def test_j2_spheres_3d_matches_oracle(fh, torch, tangent_mode):
    phase = random_spheres(16, seed=3, r_min=2.0, r_max=4.0)
    params = np.array([[1.2, 0.8], [2.4, 1.6]])
    plastic = np.array([[0.004, 0.8], [0.008, 1.6]])
    Ebar = np.zeros(9)
    Ebar[1] = Ebar[3] = 0.01
    Ebar[0] = 0.004
    Fg, hg, pbar, stats, ref = _j2_solve_both(fh, torch, phase, params, plastic, Ebar, 4, 1e-9, tangent_mode)
    assert ref.history[9].max() > 0
    _check(Fg, hg, pbar, stats, ref)


def test_j2_history_carries_over_between_solves(fh, torch):
    phase, params, plastic, Ebar = j2_config(32, 1, nz=2)
    shape = phase.shape
    Eun = 0.6 * Ebar
    Eun[1] = Eun[3] = 0.002
    with fh.Context(*shape) as ctx:
        hist = torch.zeros((10,) + shape, dtype=torch.float64, device="cuda")
        mat = fh.Material(fh.J2, phase, params, plastic=plastic, history=hist)
        F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        ctx.fft_homog_solve(mat, Ebar, F, n_increments=5, options=fh.default_options(newton_tol=1e-9))
        pbar, _, _ = ctx.fft_homog_solve(mat, Eun, F, n_increments=3,
                                         options=fh.default_options(newton_tol=1e-9, init=fh.INIT_GIVEN))
        Fg, hg = host(F), host(hist)
    r1 = osolver.solve(phase, params, omat.J2, Ebar, n_increments=5, newton_tol=1e-9, plastic=plastic)
    r2 = osolver.solve(phase, params, omat.J2, Eun, n_increments=3, newton_tol=1e-9, F_init=r1.F,
                       plastic=plastic, history=r1.history)
    np.testing.assert_allclose(pbar, r2.Pbar, rtol=PBAR_TOL, atol=PBAR_TOL * np.abs(r2.Pbar).max())
    assert field_maxrel(_sym(Fg), _sym(r2.F)) < FIELD_TOL
    assert field_maxrel(hg, r2.history) < FIELD_TOL


def test_j2_refused_where_unsupported(fh, torch):
    phase, params, plastic, Ebar = j2_config(16, 0, nz=2)
    shape = phase.shape
    with fh.Context(*shape) as ctx:
        hist = torch.zeros((10,) + shape, dtype=torch.float64, device="cuda")
        F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        with pytest.raises(fh.FhError) as e:
            ctx.fft_homog_solve(fh.Material(fh.J2, phase, params), Ebar, F)  # no plastic table / history
        assert e.value.code == fh.FH_ERR_ARG
        mat = fh.Material(fh.J2, phase, params, plastic=plastic, history=hist)
        with pytest.raises(fh.FhError) as e:
            ctx.fft_homog_tangent(mat, F)
        assert e.value.code == fh.FH_ERR_UNSUPPORTED
    b = fh.Batch([(phase, None)])
    try:
        with pytest.raises(fh.FhError) as e:
            b.fft_homog_solve_batched(fh.J2, params, Ebar)
        assert e.value.code == fh.FH_ERR_UNSUPPORTED
    finally:
        b.close()
