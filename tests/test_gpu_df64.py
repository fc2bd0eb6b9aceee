"""The double-float option of the CG matrix-vector product (FH_ARITH_DF64).

The five projection passes of every CG product transform in double-float
arithmetic (pairs of FP32 values, about 48 significant bits) and K : p is
formed in double-float; the CG updates and dot products, the Newton
right-hand side and residuals stay FP64.
The method's results must not move beyond the parity bars: against the CPU
oracle, 1e-9 relative on the homogenized stress and tangent and 1e-8
max-relative on the voxel fields, with the same Newton iteration counts.
"""

import numpy as np
import pytest

from gpu_helpers import dev, field_maxrel, host, require_gpu
from oracle import homogenize, materials as omat, solver as osolver, spectral
from rve_inputs import random_deformation, random_spheres, shear_macro, small_strain_config, two_phase_table

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-8
PBAR_TOL = 1e-9


@pytest.fixture(scope="module")
def fh():
    require_gpu()
    import paper_2408_03804_gb300 as fh

    return fh


@pytest.fixture(scope="module")
def torch():
    import torch

    return torch


def _solve(fh, torch, phase, params, kind, Fbar, n_inc, tol, arith, tangent_mode=0, check_every=4):
    shape = phase.shape
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), fh.Context(*shape, stream=stream.cuda_stream) as ctx:
        F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        opts = fh.default_options(newton_tol=tol, matvec_arith=arith, tangent_mode=tangent_mode,
                                  check_every=check_every)
        pbar, stats, _ = ctx.fft_homog_solve(fh.Material(kind, phase, params), Fbar, F, n_increments=n_inc,
                                            options=opts)
        torch.cuda.synchronize()
        return host(F), pbar, stats


@pytest.mark.parametrize("kind,shape,tangent_mode", [(1, (16, 16, 16), 0), (2, (12, 16, 8), 0), (1, (8, 12, 24), 1),
                                                     (0, (16, 8, 6), 0)])
def test_df64_solve_matches_oracle(fh, torch, kind, shape, tangent_mode):
    phase = random_spheres(shape, seed=sum(shape), r_min=1.5, r_max=3.0)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.05, finite=kind != 0)
    Fg, pbar, st = _solve(fh, torch, phase, params, kind, Fbar, 2, 1e-10, fh.ARITH_DF64, tangent_mode)
    ref = osolver.solve(phase, params, kind, Fbar, n_increments=2, newton_tol=1e-10)
    assert st["n_newton"] == len(ref.newton_residuals)
    assert all(abs(a - b) <= 2 for a, b in zip(st["cg_iterations"], ref.cg_iterations))
    np.testing.assert_allclose(pbar, ref.Pbar, rtol=PBAR_TOL, atol=PBAR_TOL * np.abs(ref.Pbar).max())
    assert np.abs(Fg - ref.F).max() < FIELD_TOL * np.abs(ref.F - Fbar.reshape(9, 1, 1, 1)).max()


def test_df64_projection_error_is_at_double_float_level(fh, torch):
    """One product y = G(K : p) through fh_matvec (jvp form) with each arithmetic against the oracle's:
    the double-float product is off by about the double-float unit 2^-48 times log2 N relative to |y|,
    far below the CG tolerances, and more than the FP64 product (the option really is another
    arithmetic)."""
    shape = (32, 32, 32)
    n = int(np.prod(shape))
    F = random_deformation(n, seed=3, scale=0.1, identity=True).reshape((9,) + shape)
    phase = (np.random.default_rng(4).random(shape) < 0.3).astype(np.uint8)
    params = two_phase_table(1.5, 1.0, 10.0)
    lam, mu = params[phase, 0], params[phase, 1]
    K = omat.tangent(1, F, lam, mu)
    p = np.random.default_rng(5).standard_normal((9,) + shape)
    ref = spectral.project(omat.apply_tangent(K, p))
    out = {}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), fh.Context(*shape, stream=stream.cuda_stream) as ctx:
        for arith in (fh.ARITH_FP64, fh.ARITH_DF64):
            y = torch.empty((9,) + shape, dtype=torch.float64, device="cuda")
            ctx.fh_matvec(dev(p), y, mat=fh.Material(1, phase, params), F=dev(F), arith=arith)
            out[arith] = host(y)
    scale = np.abs(ref).max()
    err64 = np.abs(out[fh.ARITH_FP64] - ref).max() / scale
    errdf = np.abs(out[fh.ARITH_DF64] - ref).max() / scale
    assert err64 < 1e-13
    assert errdf < 1e-12
    assert errdf > err64


def test_df64_graph_replay_and_plain_launches_agree(fh, torch):
    shape = (16, 16, 16)
    phase = random_spheres(shape, seed=2, r_min=1.5, r_max=3.0)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.05, finite=True)
    res = []
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), fh.Context(*shape, stream=stream.cuda_stream) as ctx:
        mat = fh.Material(1, phase, params)
        F = torch.empty((9,) + shape, dtype=torch.float64, device="cuda")
        for mode in (fh.LAUNCH_GRAPH, fh.LAUNCH_PLAIN):
            F.zero_()
            opts = fh.default_options(newton_tol=1e-10, matvec_arith=fh.ARITH_DF64, launch_mode=mode)
            pbar, st, _ = ctx.fft_homog_solve(mat, Fbar, F, n_increments=1, options=opts)
            res.append((host(F), pbar, st["cg_iterations"], st["cg_graph_replays"]))
    assert np.array_equal(res[0][0], res[1][0]) and res[0][2] == res[1][2]
    assert res[0][3] > 0 and res[1][3] == 0


def test_df64_tangent_matches_oracle(fh, torch):
    phase, params, _ = small_strain_config(16)
    zero = np.zeros((9, 16, 16, 16))
    C_ref = homogenize.tangent(phase, params, 0, zero, cg_tol=1e-13)
    with fh.Context(16, 16, 16) as ctx:
        C = ctx.fft_homog_tangent(fh.Material(0, phase, params), dev(zero),
                                  options=fh.default_options(cg_tol=1e-13, matvec_arith=fh.ARITH_DF64))
    assert np.abs(C - C_ref).max() < PBAR_TOL * np.abs(C_ref).max()


@pytest.mark.parametrize("shape,kind", [((27, 25, 1), 2), ((15, 21, 8), 1), ((37, 12, 4), 1), ((45, 45, 1), 0),
                                        ((199, 6, 2), 2)])
def test_df64_on_run_time_plans_and_plane_cells_matches_oracle(fh, torch, shape, kind):
    """The double-float transforms on every kind of axis: odd lengths (direct odd-radix stages), primes
    from 37 on (Rader's algorithm) and plane cells (nz = 1), against the oracle."""
    if shape[2] > 2:
        phase = random_spheres(shape, seed=sum(shape), r_min=1.5, r_max=3.0)
    else:  # z-invariant cell
        phase = np.ascontiguousarray(np.repeat(
            (np.random.default_rng(sum(shape)).random(shape[:2] + (1,)) < 0.3).astype(np.uint8), shape[2], axis=2))
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.05, finite=kind != 0)
    Fg, pbar, st = _solve(fh, torch, phase, params, kind, Fbar, 2, 1e-10, fh.ARITH_DF64)
    ref = osolver.solve(phase, params, kind, Fbar, n_increments=2, newton_tol=1e-10)
    assert st["n_newton"] == len(ref.newton_residuals)
    assert all(abs(a - b) <= 2 for a, b in zip(st["cg_iterations"], ref.cg_iterations))
    np.testing.assert_allclose(pbar, ref.Pbar, rtol=PBAR_TOL, atol=PBAR_TOL * np.abs(ref.Pbar).max())
    assert np.abs(Fg - ref.F).max() < FIELD_TOL * np.abs(ref.F - Fbar.reshape(9, 1, 1, 1)).max()


def test_df64_full_size_bench_cell_matches_fp64_solve(fh, torch):
    """The 128^3 neo-Hookean benchmark cell (5 increments, tolerance 1e-8) with each arithmetic: the same
    Newton count, CG counts within 2 per Newton iteration, Pbar within 1e-9 and the fields within 1e-8
    max-relative of each other (the FP64 solve matches the oracle's stored 128^3 solve to 1e-16 in Pbar)."""
    from rve_inputs import neo_hookean_config

    shape = (128, 128, 128)
    phase, params, Fbar = neo_hookean_config(shape, seed=0)
    out = {}
    for arith in (fh.ARITH_FP64, fh.ARITH_DF64):
        Fg, pbar, st = _solve(fh, torch, phase, params, 1, Fbar, 5, 1e-8, arith, check_every=16)
        out[arith] = (Fg, pbar, st)
    (F64, p64, s64), (Fdf, pdf, sdf) = out[fh.ARITH_FP64], out[fh.ARITH_DF64]
    assert sdf["n_newton"] == s64["n_newton"]
    assert all(abs(a - b) <= 2 for a, b in zip(sdf["cg_iterations"], s64["cg_iterations"]))
    np.testing.assert_allclose(pdf, p64, rtol=PBAR_TOL, atol=PBAR_TOL * np.abs(p64).max())
    assert field_maxrel(Fdf - Fbar.reshape(9, 1, 1, 1), F64 - Fbar.reshape(9, 1, 1, 1)) < FIELD_TOL


def test_df64_batched_cells_match_oracle_and_single_cell_df64_solves(fh, torch):
    """A batch of uneven neo-Hookean cells with double-float CG products: each cell against the oracle
    (the parity bars, same Newton counts) and against the single-cell double-float solve (1e-12)."""
    shapes = [(16, 16, 16), (12, 12, 24), (8, 8, 8), (16, 16, 16)]
    cells = [(random_spheres(shape, seed=20 + k, r_min=1.5, r_max=3.0), None) for k, shape in enumerate(shapes)]
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.05, finite=True)
    opts = fh.default_options(newton_tol=1e-10, check_every=4, matvec_arith=fh.ARITH_DF64)
    with fh.Batch(cells) as b:
        pbar, status, newton, cg, rc = b.fft_homog_solve_batched(fh.NEO_HOOKEAN, params, Fbar, options=opts)
        F_batch = [F.cpu().numpy() for F in b.F]
    assert rc == fh.FH_OK and np.all(status == 0)
    for i, (phase, _) in enumerate(cells):
        ref = osolver.solve(phase, params, 1, Fbar, newton_tol=1e-10)
        assert newton[i] == len(ref.newton_residuals)
        np.testing.assert_allclose(pbar[i], ref.Pbar, rtol=PBAR_TOL, atol=PBAR_TOL * np.abs(ref.Pbar).max())
        assert np.abs(F_batch[i] - ref.F).max() < FIELD_TOL * np.abs(ref.F - Fbar.reshape(9, 1, 1, 1)).max()
        F1, p1, st1 = _solve(fh, torch, phase, params, 1, Fbar, 1, 1e-10, fh.ARITH_DF64)
        np.testing.assert_allclose(pbar[i], p1, rtol=1e-12, atol=1e-14)
        assert np.abs(F_batch[i] - F1).max() <= 1e-12 * np.abs(F1 - Fbar.reshape(9, 1, 1, 1)).max()
        assert abs(cg[i] - st1["n_cg"]) <= 2 * newton[i]


def test_df64_split_and_join_of_field_values(fh, torch):
    """The conversions the double-float kernels apply to FP64 field values: hi is x with its significand
    cut after 23 bits (exact), lo the rest truncated to 24 significant bits, |x - hi - lo| < 2^-47 |x|
    (or below 2^-125 where lo would fall below the smallest normal float),
    hi + lo joined back with one FP64 addition; values below the smallest normal float give 0 and values
    beyond the float range give an infinite hi."""
    rng = np.random.default_rng(7)
    x = np.concatenate([
        np.array([0.0, -0.0, 1.0, -1.0, np.pi, -np.e, 2.0 ** -126, 2.0 ** -125 * 3, 1e-30, -3e-38, 1e300, -1e39]),
        rng.standard_normal(4000) * 10.0 ** rng.uniform(-30, 30, 4000),
    ])
    hi, lo, out = fh.fh_df64_roundtrip(dev(x))
    hi, lo, out = (host(t) for t in (hi, lo, out))
    # expected hi: the double's bit pattern with the low 29 significand bits cleared, as a float32
    bits = x.view(np.uint64) & ~np.uint64((1 << 29) - 1)
    hi_ref = bits.view(np.float64).astype(np.float32)
    normal = (np.abs(x) >= 2.0 ** -126) & (np.abs(x) < 2.0 ** 128)
    assert np.array_equal(hi[normal], hi_ref[normal])
    # relative 2^-47, or (a lo below the smallest normal float is dropped) absolute 2^-125
    err = np.abs(x[normal] - (hi[normal].astype(np.float64) + lo[normal]))
    assert np.all(err <= np.maximum(2.0 ** -47 * np.abs(x[normal]), 2.0 ** -125))
    assert np.all(lo[normal] * np.sign(x[normal]) >= 0)  # truncation: lo has the sign of x (or is 0)
    np.testing.assert_array_equal(out, hi.astype(np.float64) + lo.astype(np.float64))
    tiny = np.abs(x) < 2.0 ** -126
    assert np.all(hi[tiny] == 0) and np.all(lo[tiny] == 0)
    huge = np.abs(x) >= 2.0 ** 128
    assert np.all(np.isinf(hi[huge])) and np.all(np.sign(hi[huge]) == np.sign(x[huge]))


@pytest.mark.parametrize("shape", [(16, 8, 12), (15, 7, 1)])
def test_df64_anisotropic_box_matches_oracle(fh, torch, shape):
    """Box side lengths (1, 2, 0.5): the double-float wave vectors k / L_a against the oracle."""
    lengths = (1.0, 2.0, 0.5)
    phase = (np.random.default_rng(11).random(shape) < 0.3).astype(np.uint8)
    if shape[2] == 1:
        lengths = (1.0, 2.0, 1.0)
    params = two_phase_table(1.5, 1.0, 10.0)
    Fbar = shear_macro(0.05, finite=True)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), fh.Context(*shape, stream=stream.cuda_stream) as ctx:
        F = torch.zeros((9,) + shape, dtype=torch.float64, device="cuda")
        opts = fh.default_options(newton_tol=1e-10, matvec_arith=fh.ARITH_DF64, lengths=lengths)
        pbar, st, _ = ctx.fft_homog_solve(fh.Material(1, phase, params), Fbar, F, n_increments=2, options=opts)
        Fg = host(F)
    ref = osolver.solve(phase, params, 1, Fbar, n_increments=2, newton_tol=1e-10, lengths=lengths)
    assert st["n_newton"] == len(ref.newton_residuals)
    np.testing.assert_allclose(pbar, ref.Pbar, rtol=PBAR_TOL, atol=PBAR_TOL * np.abs(ref.Pbar).max())
    assert np.abs(Fg - ref.F).max() < FIELD_TOL * np.abs(ref.F - Fbar.reshape(9, 1, 1, 1)).max()
