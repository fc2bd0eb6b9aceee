"""GPU path against the CPU oracle, element by element, through the C-ABI.

Tolerances: homogenized stress relative 1e-9, voxel fields 1e-8 in the
max-relative measure (max|a - b| / max|b| per component field); single
operators (stress, tangent, projection, matrix-vector product) are compared
at 1e-12, since both sides evaluate the same expression and differ only by
rounding order (FFT sums of a few hundred terms, AD vs closed form).
"""

import numpy as np
import pytest

from gpu_helpers import dev, field_maxrel, host, pack_tangent, require_gpu
from oracle import materials as omat
from oracle import solver as osolver
from oracle import spectral
from rve_inputs import (centered_sphere, laminate, random_deformation, random_spheres, shear_macro,
                        small_strain_config, two_phase_table)

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


def _phase(shape, seed, n_phase=2):
    rng = np.random.default_rng(seed)
    return rng.integers(0, n_phase, size=shape).astype(np.uint8)


# ---------------------------------------------------------------------------
# a2: stress and tangent by AD
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("shape", [(4, 8, 16), (2, 2, 2), (8, 1, 6 + 2)])
def test_constitutive_matches_closed_form(fh, torch, kind, shape):
    n = int(np.prod(shape))
    F = random_deformation(n, seed=kind + 3, scale=0.2, identity=omat.FINITE_STRAIN[kind]).reshape((9,) + shape)
    phase = _phase(shape, 1, 3)
    params = np.array([[1.5, 1.0], [15.0, 10.0], [0.3, 0.7]])
    lam, mu = params[phase, 0], params[phase, 1]
    with fh.Context(*shape) as ctx:
        mat = fh.Material(kind, phase, params)
        Fd = dev(F)
        P = torch.empty_like(Fd)
        K = torch.empty((45,) + shape, dtype=torch.float64, device="cuda")
        pbar = ctx.fh_constitutive(mat, Fd, P, K)
    P_ref = omat.stress(kind, F, lam, mu)
    K_ref = pack_tangent(omat.tangent(kind, F, lam, mu))
    assert field_maxrel(host(P), P_ref) < OP_TOL
    assert np.abs(host(K) - K_ref).max() < OP_TOL * np.abs(K_ref).max()
    np.testing.assert_allclose(pbar, P_ref.reshape(9, -1).mean(axis=1), rtol=1e-12, atol=1e-14)


def test_constitutive_reports_nonphysical_voxels(fh, torch):
    shape = (4, 4, 4)
    F = random_deformation(64, seed=1, scale=0.05).reshape((9,) + shape)
    F[0, 1, 2, 3] = -1.0  # det F < 0 in one voxel
    with fh.Context(*shape) as ctx:
        mat = fh.Material(fh.NEO_HOOKEAN, np.zeros(shape, np.uint8), [[1.5, 1.0]])
        _, rc = ctx.fh_constitutive(mat, dev(F), allow_nonphysical=True)
    assert rc == fh.FH_ERR_NONPHYSICAL


def test_out_of_range_phase_is_reported(fh, torch):
    shape = (4, 4, 4)
    F = random_deformation(64, seed=2, scale=0.05).reshape((9,) + shape)
    phase = np.zeros(shape, np.uint8)
    phase[0, 0, 0] = 5
    with fh.Context(*shape) as ctx:
        mat = fh.Material(fh.NEO_HOOKEAN, phase, [[1.5, 1.0], [3.0, 2.0]])
        _, rc = ctx.fh_constitutive(mat, dev(F), allow_nonphysical=True)
    assert rc == fh.FH_ERR_NONPHYSICAL


# ---------------------------------------------------------------------------
# a3/a4: projection and matrix-vector product
# ---------------------------------------------------------------------------
PROJ_SHAPES = [(8, 8, 8), (4, 8, 16), (16, 4, 2), (2, 2, 2), (1, 4, 8), (32, 16, 8), (8, 1, 32),
               (256, 2, 2), (2, 256, 2), (2, 2, 256), (64, 32, 128),
               # radix-3 lengths (3 * 2^a), odd axes and odd half lengths
               (48, 12, 6), (3, 6, 24), (96, 8, 4), (6, 3, 96), (24, 48, 12), (192, 2, 2), (2, 2, 192),
               (12, 12, 12),
               # x/y lengths without a compile-time plan (run-time plans: radix 5, 7 and direct prime stages,
               # even lengths with odd factors, extents above 256)
               (5, 7, 4), (13, 11, 2), (15, 21, 8), (9, 25, 6), (10, 14, 4), (199, 3, 2), (3, 199, 2),
               (169, 2, 2), (127, 4, 2), (121, 6, 2), (299, 2, 2), (512, 2, 2), (2, 512, 2), (384, 3, 2),
               (40, 20, 16),
               # primes from 37 on by Rader's algorithm (inner lengths 36, 508 = 4 x 127 with a direct stage)
               (37, 5, 2), (2, 37, 4), (509, 2, 2),
               # cells one voxel thick (nz = 1: plane problems, the z transform is the identity)
               (8, 8, 1), (199, 5, 1), (12, 37, 1), (1, 6, 1), (1, 1, 1)]


@pytest.mark.parametrize("shape", PROJ_SHAPES)
def test_projection_matches_oracle(fh, torch, shape):
    rng = np.random.default_rng(sum(shape))
    A = rng.standard_normal((9,) + shape)
    lengths = (1.0, 2.0, 0.5) if shape[0] == 4 else (1.0, 1.0, 1.0)
    with fh.Context(*shape) as ctx:
        Ad = dev(A)
        out = torch.empty_like(Ad)
        ctx.fh_project(Ad, out, scale=-1.5, lengths=lengths)
        inplace = Ad.clone()
        ctx.fh_project(inplace, inplace, scale=1.0, lengths=lengths)
    ref = spectral.project(A, lengths)
    assert np.abs(host(out) + 1.5 * ref).max() < OP_TOL * 1.5 * np.abs(A).max()
    assert np.abs(host(inplace) - ref).max() < OP_TOL * np.abs(A).max()


@pytest.mark.parametrize("kind", [1, 2, 0])
@pytest.mark.parametrize("shape", [(8, 8, 8), (4, 16, 32), (15, 7, 8), (15, 7, 1)])
def test_matvec_matches_oracle_stored_and_jvp(fh, torch, kind, shape):
    n = int(np.prod(shape))
    F = random_deformation(n, seed=5, scale=0.1, identity=omat.FINITE_STRAIN[kind]).reshape((9,) + shape)
    p = np.random.default_rng(6).standard_normal((9,) + shape)
    phase = _phase(shape, 7)
    params = two_phase_table(1.5, 1.0, 10.0)
    lam, mu = params[phase, 0], params[phase, 1]
    Kref = omat.tangent(kind, F, lam, mu)
    ref = spectral.project(omat.apply_tangent(Kref, p))
    with fh.Context(*shape) as ctx:
        mat = fh.Material(kind, phase, params)
        Fd, pd = dev(F), dev(p)
        K = torch.empty((45,) + shape, dtype=torch.float64, device="cuda")
        ctx.fh_constitutive(mat, Fd, None, K)
        y1 = torch.empty_like(pd)
        y2 = torch.empty_like(pd)
        ctx.fh_matvec(pd, y1, K=K)
        ctx.fh_matvec(pd, y2, mat=mat, F=Fd)
        # the double-float option in both forms (stored K converted by the library, jvp)
        y3 = torch.empty_like(pd)
        y4 = torch.empty_like(pd)
        ctx.fh_matvec(pd, y3, K=K, arith=fh.ARITH_DF64)
        ctx.fh_matvec(pd, y4, mat=mat, F=Fd, arith=fh.ARITH_DF64)
    scale = np.abs(ref).max()
    assert np.abs(host(y1) - ref).max() < OP_TOL * 10 * scale
    assert np.abs(host(y2) - ref).max() < OP_TOL * 10 * scale
    assert np.abs(host(y3) - ref).max() < 1e-12 * scale
    assert np.abs(host(y4) - ref).max() < 1e-12 * scale


# ---------------------------------------------------------------------------
# a1-a7: the whole Newton-Krylov solve
# ---------------------------------------------------------------------------
def _solve_both(fh, torch, phase, params, kind, Fbar, n_inc, tol, cg_tol=None, tangent_mode=0,
                lengths=(1.0, 1.0, 1.0), max_newton=50, max_cg=5000, allow=()):
    shape = phase.shape
    with fh.Context(*shape) as ctx:
        mat = fh.Material(kind, phase, params)
        F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        opts = fh.default_options(newton_tol=tol, cg_tol=cg_tol or 0.0, tangent_mode=tangent_mode,
                                  lengths=lengths, max_newton=max_newton, max_cg=max_cg, check_every=4)
        pbar, stats, rc = ctx.fft_homog_solve(mat, Fbar, F, n_increments=n_inc, options=opts, allow=allow)
        Fg = host(F)
    ref = osolver.solve(phase, params, kind, Fbar, n_increments=n_inc, newton_tol=tol, cg_tol=cg_tol,
                        lengths=lengths, max_newton=max_newton, max_cg=max_cg, raise_on_failure=not allow)
    return Fg, pbar, stats, rc, ref


def test_small_strain_sphere_16_matches_oracle(fh, torch):
    """Linear elastic 16^3 cube, centred sphere r = 0.25 L, eps_xy = 0.01, tol 1e-10."""
    phase, params, Ebar = small_strain_config(16)
    Fg, pbar, stats, _, ref = _solve_both(fh, torch, phase, params, 0, Ebar, 1, 1e-10)
    assert stats["n_newton"] == len(ref.newton_residuals) == 2
    assert all(abs(a - b) <= 1 for a, b in zip(stats["cg_iterations"], ref.cg_iterations))
    np.testing.assert_allclose(pbar, ref.Pbar, rtol=PBAR_TOL, atol=PBAR_TOL * np.abs(ref.Pbar).max())
    eps_g = osolver.strain_field(0, Fg)
    eps_r = osolver.strain_field(0, ref.F)
    assert field_maxrel(eps_g, eps_r) < FIELD_TOL


def test_neo_hookean_random_spheres_matches_oracle(fh, torch):
    n = 32
    phase = random_spheres(n, seed=0, r_min=2.0, r_max=4.0)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.05, finite=True)
    Fg, pbar, stats, _, ref = _solve_both(fh, torch, phase, params, 1, Fbar, 5, 1e-8)
    assert stats["n_newton"] == len(ref.newton_residuals)
    np.testing.assert_allclose(pbar, ref.Pbar, rtol=PBAR_TOL, atol=PBAR_TOL * np.abs(ref.Pbar).max())
    assert field_maxrel(Fg - np.eye(3).reshape(9, 1, 1, 1), ref.F - np.eye(3).reshape(9, 1, 1, 1)) < FIELD_TOL


@pytest.mark.parametrize("kind", [1, 2])
def test_anisotropic_box_and_ragged_grid(fh, torch, kind):
    shape = (8, 16, 4)
    phase = _phase(shape, 11)
    params = two_phase_table(1.5, 1.0, 5.0)
    rng = np.random.default_rng(3)
    Fbar = np.eye(3).reshape(9) + rng.uniform(-0.03, 0.03, 9)
    Fg, pbar, stats, _, ref = _solve_both(fh, torch, phase, params, kind, Fbar, 2, 1e-10,
                                          lengths=(1.0, 2.0, 0.5))
    np.testing.assert_allclose(pbar, ref.Pbar, rtol=PBAR_TOL, atol=PBAR_TOL * np.abs(ref.Pbar).max())
    assert np.abs(Fg - ref.F).max() < FIELD_TOL * np.abs(ref.F - Fbar.reshape(9, 1, 1, 1)).max()


def test_radix3_grid_solve_matches_oracle(fh, torch):
    shape = (12, 24, 12)
    phase = random_spheres(shape, seed=4, r_min=1.5, r_max=3.0)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.05, finite=True)
    Fg, pbar, stats, _, ref = _solve_both(fh, torch, phase, params, 1, Fbar, 2, 1e-10)
    assert stats["n_newton"] == len(ref.newton_residuals)
    np.testing.assert_allclose(pbar, ref.Pbar, rtol=PBAR_TOL, atol=PBAR_TOL * np.abs(ref.Pbar).max())
    assert np.abs(Fg - ref.F).max() < FIELD_TOL * np.abs(ref.F - Fbar.reshape(9, 1, 1, 1)).max()


@pytest.mark.parametrize("shape", [(15, 21, 8), (27, 25, 2), (27, 25, 1)])
def test_odd_grid_solve_matches_oracle(fh, torch, shape):
    """Odd x/y extents (the paper's grids are odd, Section 4.1.1): run-time FFT plans, no Nyquist index."""
    if shape[2] > 2:
        phase = random_spheres(shape, seed=6, r_min=1.5, r_max=3.0)
    else:  # z-invariant (plane strain) cell
        phase = np.ascontiguousarray(np.repeat(_phase(shape[:2] + (1,), 9), shape[2], axis=2))
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.05, finite=True)
    Fg, pbar, stats, _, ref = _solve_both(fh, torch, phase, params, 1, Fbar, 2, 1e-10)
    assert stats["n_newton"] == len(ref.newton_residuals)
    assert all(abs(a - b) <= 1 for a, b in zip(stats["cg_iterations"], ref.cg_iterations))
    np.testing.assert_allclose(pbar, ref.Pbar, rtol=PBAR_TOL, atol=PBAR_TOL * np.abs(ref.Pbar).max())
    assert np.abs(Fg - ref.F).max() < FIELD_TOL * np.abs(ref.F - Fbar.reshape(9, 1, 1, 1)).max()


def test_jvp_mode_equals_stored_mode(fh, torch):
    shape = (16, 8, 8)
    phase = _phase(shape, 12)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.03, finite=True)
    out = []
    for mode in (0, 1):
        with fh.Context(*shape) as ctx:
            mat = fh.Material(1, phase, params)
            F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
            opts = fh.default_options(newton_tol=1e-10, tangent_mode=mode)
            pbar, stats, _ = ctx.fft_homog_solve(mat, Fbar, F, n_increments=2, options=opts)
            out.append((host(F), pbar, stats))
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-12
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-12)


def test_svk_laminate_matches_exact_solution(fh, torch):
    from oracle import laminate as olam

    shape = (8, 4, 4)
    phase = laminate(shape, 2, axis=0)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = np.eye(3).reshape(9) + np.array([0.02, 0.03, -0.01, 0.01, -0.02, 0.0, 0.015, 0.0, 0.01])
    with fh.Context(*shape) as ctx:
        mat = fh.Material(2, phase, params)
        F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        ctx.fft_homog_solve(mat, Fbar, F, n_increments=1, options=fh.default_options(newton_tol=1e-12))
        Fg = host(F).reshape(9, -1)
    FA, FB = olam.laminate_states(2, params, 0.25, Fbar)
    ph = phase.reshape(-1)
    assert np.abs(Fg[:, ph == 1] - FA[:, None]).max() < 1e-11
    assert np.abs(Fg[:, ph == 0] - FB[:, None]).max() < 1e-11


def test_homogeneous_and_degenerate_grids(fh, torch):
    # homogeneous material: no fluctuation at all
    shape = (8, 8, 8)
    with fh.Context(*shape) as ctx:
        mat = fh.Material(1, np.zeros(shape, np.uint8), [[1.5, 1.0]])
        F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        Fbar = shear_macro(0.05, finite=True)
        pbar, _, _ = ctx.fft_homog_solve(mat, Fbar, F, options=fh.default_options(newton_tol=1e-12))
        assert np.abs(host(F) - Fbar.reshape(9, 1, 1, 1)).max() < 1e-14
        np.testing.assert_allclose(pbar, omat.stress(1, Fbar.reshape(9, 1), 1.5, 1.0)[:, 0], rtol=1e-14, atol=1e-15)
    # a 1 x 1 x 2 grid has no compatible fluctuation: F = Fbar in both voxels
    with fh.Context(1, 1, 2) as ctx:
        mat = fh.Material(1, np.array([[[0, 1]]], np.uint8), two_phase_table(1.5, 1.0, 10.0))
        F = torch.zeros((9, 1, 1, 2), dtype=torch.float64, device="cuda")
        ctx.fft_homog_solve(mat, Fbar, F)
        assert np.abs(host(F) - Fbar.reshape(9, 1, 1, 1)).max() < 1e-15


def test_iteration_caps_and_warm_start(fh, torch):
    shape = (16, 16, 16)
    phase = centered_sphere(shape, 0.25)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.05, finite=True)
    with fh.Context(*shape) as ctx:
        mat = fh.Material(1, phase, params)
        F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        _, stats, rc = ctx.fft_homog_solve(mat, Fbar, F, options=fh.default_options(max_cg=3),
                                           allow=(fh.FH_ERR_NOT_CONVERGED,))
        assert rc == fh.FH_ERR_NOT_CONVERGED and stats["cg_iterations"] == [3]
        assert torch.isfinite(F).all()
        _, _, rc = ctx.fft_homog_solve(mat, Fbar, F, options=fh.default_options(max_newton=1),
                                       allow=(fh.FH_ERR_NOT_CONVERGED,))
        assert rc == fh.FH_ERR_NOT_CONVERGED
        # cold solve to gamma = 0.02, then warm start to 0.05 equals a cold solve to 0.05
        F1 = torch.zeros_like(F)
        ctx.fft_homog_solve(mat, shear_macro(0.02, True), F1, options=fh.default_options(newton_tol=1e-11))
        ctx.fft_homog_solve(mat, Fbar, F1, n_increments=3,
                            options=fh.default_options(newton_tol=1e-11, init=fh.INIT_GIVEN))
        F2 = torch.zeros_like(F)
        ctx.fft_homog_solve(mat, Fbar, F2, n_increments=1, options=fh.default_options(newton_tol=1e-11))
        assert (F1 - F2).abs().max().item() < 1e-10


def test_solve_is_deterministic(fh, torch):
    shape = (16, 16, 16)
    phase = _phase(shape, 4)
    params = two_phase_table(1.5, 1.0, 10.0)
    res = []
    for _ in range(2):
        with fh.Context(*shape) as ctx:
            F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
            pbar, stats, _ = ctx.fft_homog_solve(fh.Material(1, phase, params), shear_macro(0.05, True), F,
                                                 n_increments=2)
            res.append((host(F), pbar, stats["cg_iterations"]))
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert res[0][2] == res[1][2]


@pytest.mark.parametrize("nz", [2, 1])
def test_svk_square_inclusion_2d_matches_oracle(fh, torch, nz):
    """Section 4.1.1's St. Venant-Kirchhoff cell in the 2D mode (48 x 48 x nz, z-invariant): stiff square
    of side L/3 at a corner, simple shear 0.1, one increment, Newton tolerance 1e-5 and CG tolerance 1e-8
    as in the paper. The residual of every Newton iteration and the CG counts agree with the oracle."""
    from rve_inputs import svk_square_config

    phase, params, Fbar = svk_square_config(48, nz=nz)
    Fg, pbar, stats, _, ref = _solve_both(fh, torch, phase, params, 2, Fbar, 1, 1e-5, cg_tol=1e-8)
    assert stats["n_newton"] == len(ref.newton_residuals) >= 2
    np.testing.assert_allclose(stats["newton_residuals"], ref.newton_residuals, rtol=1e-6)
    assert all(abs(a - b) <= 1 for a, b in zip(stats["cg_iterations"], ref.cg_iterations))
    np.testing.assert_allclose(pbar, ref.Pbar, rtol=1e-8, atol=1e-8 * np.abs(ref.Pbar).max())


# ---------------------------------------------------------------------------
# launch accounting: per-kernel counts cover launches that did work only
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("check_every", [1, 16])
def test_launch_accounting_books_idle_launches_apart(fh, torch, check_every):
    """Each Newton iteration runs one right-hand-side projection and one product per CG iteration, so the
    forward z pass must be counted n_newton + n_cg times whatever check_every is; the launches queued after
    CG had converged are counted as idle (none with check_every = 1, when the host reads the flag after
    every iteration)."""
    shape = (16, 16, 16)
    phase = centered_sphere(shape, 0.25)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.05, finite=True)
    with fh.Context(*shape) as ctx:
        F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        ctx.fh_profile_enable(True)
        _, st, _ = ctx.fft_homog_solve(fh.Material(fh.NEO_HOOKEAN, phase, params), Fbar, F, n_increments=2,
                                       options=fh.default_options(newton_tol=1e-10, check_every=check_every))
        prof = ctx.fh_profile_read()
    n_real = st["n_newton"] + st["n_cg"]
    for cls in ("fwd_z", "fwd_y", "x_ghat", "inv_y", "inv_z"):
        assert prof[cls][0] == n_real
        assert prof[cls][1] > 0.0
    assert prof["cg_update"][0] == st["n_cg"] + st["n_newton"]  # one update per product, one finalize per solve
    if check_every == 1:
        assert prof["idle"][0] == 0
    else:
        # each CG loop queues whole chunks of check_every iterations of 8 launches
        idle = prof["idle"][0]
        assert idle > 0 and idle % 8 == 0
        assert (idle // 8 + st["n_cg"]) % check_every == 0


@pytest.mark.parametrize("kind", [2, 0])
def test_plane_cell_one_voxel_thick_equals_two_layer_cell(fh, torch, kind):
    """A z-invariant cell solved with nz = 1 and with nz = 2 (two identical layers): the second layer
    only adds a zero Nyquist plane, so both give the same in-plane field, the same Pbar and the same
    Newton iteration count (CG counts within one: the norms sum the layers in another order)."""
    from rve_inputs import svk_square_config

    res = []
    for nz in (2, 1):
        phase, params, Fbar = svk_square_config(45, nz=nz)
        if kind == 0:
            Fbar = np.zeros(9)
            Fbar[1] = Fbar[3] = 0.01
        with fh.Context(*phase.shape) as ctx:
            F = torch.zeros((9,) + phase.shape, dtype=torch.float64, device="cuda")
            pbar, st, _ = ctx.fft_homog_solve(fh.Material(kind, phase, params), Fbar, F, n_increments=1,
                                              options=fh.default_options(newton_tol=1e-10))
            res.append((host(F)[..., 0], pbar, st["n_newton"], st["cg_iterations"]))
    (F2, p2, n2, c2), (F1, p1, n1, c1) = res
    assert n1 == n2 and all(abs(a - b) <= 1 for a, b in zip(c1, c2))
    assert np.abs(F1 - F2).max() < 1e-12
    np.testing.assert_allclose(p1, p2, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("shape,kind,check_every", [((16, 16, 16), 0, 16), ((12, 10, 8), 1, 5), ((27, 25, 1), 2, 16)])
def test_graph_replayed_cg_equals_plain_launches(fh, torch, shape, kind, check_every):
    """Without per-launch timing each chunk of check_every CG iterations is the replay of a captured CUDA
    graph; with timing on (fh_profile_enable), or with launch_mode FH_LAUNCH_PLAIN, the same kernels are
    launched one by one. All give the same field bit for bit, the same iteration counts and the same
    per-class launch counts."""
    phase = centered_sphere(shape, 0.25) if shape[2] > 1 else _phase(shape, 4)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.02, finite=kind != 0)
    res = []
    stream = torch.cuda.Stream()  # graphs are not captured on the legacy default stream
    with torch.cuda.stream(stream), fh.Context(*shape, stream=stream.cuda_stream) as ctx:
        mat = fh.Material(kind, phase, params)
        F = torch.empty((9,) + shape, dtype=torch.float64, device="cuda")
        for timed, mode in ((False, fh.LAUNCH_GRAPH), (True, fh.LAUNCH_GRAPH), (False, fh.LAUNCH_PLAIN),
                            (False, fh.LAUNCH_GRAPH)):
            ctx.fh_profile_enable(timed)
            F.zero_()
            pbar, st, _ = ctx.fft_homog_solve(mat, Fbar, F, n_increments=2,
                                              options=fh.default_options(newton_tol=1e-10, check_every=check_every,
                                                                         launch_mode=mode))
            counts = {k: v[0] for k, v in ctx.fh_profile_read().items()}
            res.append((host(F), pbar, st["cg_iterations"], counts))
            replayed = not timed and mode == fh.LAUNCH_GRAPH
            assert (st["cg_graph_replays"] > 0) == replayed
            if replayed:
                # one replay per chunk of check_every iterations of every CG loop
                assert st["cg_graph_replays"] == sum(max(1, -(-c // check_every)) for c in st["cg_iterations"])
        # the second graph solve replays the graphs the first one captured
        assert st["cg_graph_captures"] == 0
    for F, pbar, cg, counts in res[1:]:
        assert np.array_equal(F, res[0][0]) and np.array_equal(pbar, res[0][1])
        assert cg == res[0][2] and counts == res[0][3]
