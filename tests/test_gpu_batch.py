"""Batched solves of cells with uneven grids (fft_homog_solve_batched).

Every cell of a batch runs Algorithm 1 with its own Newton and CG state;
passes are launched per group of equal grids and the CG iterations run as a
captured CUDA graph. The tests compare each cell with the oracle's solve of
that cell, and with the single-cell GPU solve (fft_homog_solve): the same
pass bodies in the same order, but the single-cell contexts tile small grids
finer, so their dot products sum the same terms in another order; the two
fields agree to a few units of rounding (5e-14 of the field's maximum).
"""

import numpy as np
import pytest

from gpu_helpers import require_gpu
from oracle import solver as osolver
from rve_inputs import batch_config, random_spheres, shear_macro, two_phase_table

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fh():
    require_gpu()
    import paper_2408_03804_gb300 as fh

    return fh


def test_batch_of_uneven_linear_cells_matches_oracle_and_single_solves(fh):
    import torch

    cells, params, Ebar = batch_config(7, seed=3, sizes=(8, 12, 16, 24))
    opts = fh.default_options(newton_tol=1e-10, check_every=4)
    with fh.Batch(cells) as b:
        pbar, status, newton, cg, rc = b.fft_homog_solve_batched(fh.LINEAR_ELASTIC, params, Ebar, options=opts)
        F_batch = [F.cpu().numpy() for F in b.F]
    assert rc == fh.FH_OK and np.all(status == 0)
    for i, (phase, scale) in enumerate(cells):
        ref = osolver.solve(phase, params, 0, Ebar, newton_tol=1e-10, scale=scale)
        np.testing.assert_allclose(pbar[i], ref.Pbar, rtol=1e-9, atol=1e-9 * np.abs(ref.Pbar).max())
        assert np.abs(F_batch[i] - ref.F).max() < 1e-8 * np.abs(ref.F).max()
        assert newton[i] == len(ref.newton_residuals)
        with fh.Context(*phase.shape) as ctx:
            F1 = torch.zeros((9,) + phase.shape, dtype=torch.float64, device="cuda")
            p1, st1, _ = ctx.fft_homog_solve(fh.Material(0, phase, params, scale=scale), Ebar, F1, options=opts)
        np.testing.assert_allclose(pbar[i], p1, rtol=1e-14, atol=1e-18)
        assert np.abs(F_batch[i] - F1.cpu().numpy()).max() <= 5e-14 * np.abs(F_batch[i]).max()
        assert cg[i] == st1["n_cg"]


def test_batch_neo_hookean_cells_converge_independently(fh):
    """Cells needing different Newton/CG counts are masked out as they finish."""
    shapes = [(16, 16, 16), (12, 12, 24), (16, 16, 16), (8, 8, 8)]
    cells = []
    Fbar = shear_macro(0.05, finite=True)
    for k, shape in enumerate(shapes):
        phase = random_spheres(shape, seed=10 + k, r_min=1.5, r_max=3.0)
        cells.append((phase, None))
    params = two_phase_table(1.5, 1.0, 10.0)
    with fh.Batch(cells) as b:
        pbar, status, newton, cg, rc = b.fft_homog_solve_batched(fh.NEO_HOOKEAN, params, Fbar, n_increments=2,
                                                                 options=fh.default_options(newton_tol=1e-10))
        F_batch = [F.cpu().numpy() for F in b.F]
    assert rc == fh.FH_OK
    for i, (phase, _) in enumerate(cells):
        ref = osolver.solve(phase, params, 1, Fbar, n_increments=2, newton_tol=1e-10)
        np.testing.assert_allclose(pbar[i], ref.Pbar, rtol=1e-9, atol=1e-9 * np.abs(ref.Pbar).max())
        assert np.abs(F_batch[i] - ref.F).max() < 1e-8 * np.abs(ref.F - Fbar.reshape(9, 1, 1, 1)).max()
        assert newton[i] == len(ref.newton_residuals)
        assert abs(cg[i] - sum(ref.cg_iterations)) <= len(ref.cg_iterations)
    assert len(set(cg.tolist())) > 1  # the cells really needed different iteration counts


def test_batch_reports_per_cell_failures(fh):
    cells, params, Ebar = batch_config(3, seed=5, sizes=(8, 16))
    opts = fh.default_options(newton_tol=1e-10, max_cg=2)
    with fh.Batch(cells) as b:
        pbar, status, newton, cg, rc = b.fft_homog_solve_batched(fh.LINEAR_ELASTIC, params, Ebar, options=opts,
                                                                 allow=(fh.FH_ERR_NOT_CONVERGED,))
    assert rc == fh.FH_ERR_NOT_CONVERGED
    assert np.all(status == fh.FH_ERR_NOT_CONVERGED) and np.all(cg == 2)
    assert np.all(np.isfinite(pbar))


def test_autotuned_tiles_give_the_same_solution(fh):
    """fh_autotune only changes how the passes are tiled, not what they compute."""
    import torch

    shape = (32, 32, 64)
    phase = random_spheres(shape, seed=2, r_min=2.0, r_max=4.0)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.03, finite=True)
    out = []
    for tune in (False, True):
        with fh.Context(*shape) as ctx:
            if tune:
                ms, chosen = ctx.fh_autotune(reps=2)
                assert ms > 0 and all(c >= 1 for c in chosen)
            F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
            pbar, st, _ = ctx.fft_homog_solve(fh.Material(1, phase, params), Fbar, F,
                                              options=fh.default_options(newton_tol=1e-10))
            out.append((F.cpu().numpy(), pbar))
    assert np.abs(out[0][0] - out[1][0]).max() < 1e-10 * np.abs(out[0][0] - Fbar.reshape(9, 1, 1, 1)).max()
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-10, atol=1e-14)
