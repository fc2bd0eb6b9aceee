"""The full 128^3 neo-Hookean workload on the GPU, against the oracle's own full solve.

The reference values come from ``tests/golden/make_neo_hookean_128.py``, which
runs only the CPU oracle (about 15 minutes on 8 cores): the homogenized
stress, the Newton/CG history, F at 64 sampled voxels and every voxel of two
full x-planes (2 x 128 x 128 voxels, 9 components), compared element by
element in the max-relative measure of the fluctuation. The GPU solve uses
the same launch configuration as ``bench.py``. Besides the stored values, the
test checks properties that hold at any size with the oracle's own operators:
mean(F) = Fbar, and equilibrium of the GPU state, ||G(P(F))|| small, with P
from the oracle's closed-form stress and G from the oracle's FFT projection.
"""

import json
import os

import numpy as np
import pytest

from gpu_helpers import require_gpu
from oracle import materials as omat
from oracle import spectral
from rve_inputs import neo_hookean_config

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "neo_hookean_128_seed0.json")
PLANES = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "neo_hookean_128_seed0_planes.npy")
FIELD_TOL = 1e-8


def test_neo_hookean_128_matches_oracle_full_solve():
    torch = require_gpu()
    import paper_2408_03804_gb300 as fh

    with open(GOLDEN) as f:
        ref = json.load(f)
    phase, params, Fbar = neo_hookean_config(128, 0)
    assert abs(phase.mean() - ref["phase_fraction"]) < 1e-12
    with fh.Context(128, 128, 128) as ctx:
        F = torch.zeros((9, 128, 128, 128), dtype=torch.float64, device="cuda")
        pbar, stats, _ = ctx.fft_homog_solve(fh.Material(fh.NEO_HOOKEAN, phase, params), Fbar, F, n_increments=5,
                                             options=fh.default_options(newton_tol=1e-8))
        Fg = F.cpu().numpy()
    assert stats["n_newton"] == ref["n_newton"]
    assert all(abs(a - b) <= 1 for a, b in zip(stats["cg_iterations"], ref["cg_iterations"]))
    Pref = np.asarray(ref["Pbar"])
    np.testing.assert_allclose(pbar, Pref, rtol=1e-9, atol=1e-9 * np.abs(Pref).max())
    fluct = np.abs(Fg - Fbar.reshape(9, 1, 1, 1)).reshape(9, -1).max(axis=1)
    np.testing.assert_allclose(fluct, ref["fluct_max"], rtol=1e-7)
    for s in ref["samples"]:
        i, j, k = s["voxel"]
        assert np.all(np.abs(Fg[:, i, j, k] - np.asarray(s["F"])) <= FIELD_TOL * fluct)
    # every voxel of the stored x-planes, per component: max|a - b| / max|F - Fbar| (over the whole field)
    planes = np.load(PLANES)
    err = np.abs(Fg[:, ref["planes_x"]] - planes).reshape(9, -1).max(axis=1) / np.asarray(ref["fluct_max"])
    assert err.max() < FIELD_TOL, err
    np.testing.assert_allclose(Fg.reshape(9, -1).mean(axis=1), Fbar, atol=1e-13)
    lam, mu = params[phase, 0], params[phase, 1]
    P = omat.stress(omat.NEO_HOOKEAN, Fg, lam, mu)
    GP = spectral.project(P)
    assert np.linalg.norm(GP) < 1e-9 * np.linalg.norm(P - P.reshape(9, -1).mean(axis=1).reshape(9, 1, 1, 1))
