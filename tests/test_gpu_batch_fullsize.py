"""The 256-cell batch of the benchmark (config 3), at full size and in the benchmark's launch
configuration: every cell converges, and one sampled cell of each grid size (32^3, 48^3, 64^3, 96^3)
matches the oracle's solve of that cell (homogenized stress 1e-9, field 1e-8 max-relative) and the
single-cell GPU solve (bit-identical up to 1e-14)."""

import numpy as np
import pytest

from gpu_helpers import require_gpu
from oracle import solver as osolver
from rve_inputs import batch_config

pytestmark = pytest.mark.gpu


def test_full_batch_converges_and_sampled_cells_match_the_oracle():
    torch = require_gpu()
    import paper_2408_03804_gb300 as fh

    cells, params, Ebar = batch_config(256, seed=0)
    opts = fh.default_options(newton_tol=1e-8, check_every=8)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b = fh.Batch(cells, stream=stream.cuda_stream)
        try:
            pbar, status, newton, cg, rc = b.fft_homog_solve_batched(fh.LINEAR_ELASTIC, params, Ebar, options=opts)
            torch.cuda.synchronize()
            assert rc == fh.FH_OK and np.all(status == 0)
            c1111 = pbar[:, 0] / Ebar[0]
            assert np.all(np.isfinite(c1111)) and np.all(c1111 > 0)
            picked = {}
            for i, (ph, _) in enumerate(cells):
                picked.setdefault(ph.shape[0], i)
            for n, i in sorted(picked.items()):
                phase, scale = cells[i]
                F_batch = b.F[i].cpu().numpy()
                ref = osolver.solve(phase, params, 0, Ebar, newton_tol=1e-8, scale=scale)
                np.testing.assert_allclose(pbar[i], ref.Pbar, rtol=1e-9, atol=1e-9 * np.abs(ref.Pbar).max())
                assert np.abs(F_batch - ref.F).max() < 1e-8 * np.abs(ref.F).max(), n
                assert newton[i] == len(ref.newton_residuals), n
                with fh.Context(*phase.shape, stream=stream.cuda_stream) as ctx:
                    F1 = torch.zeros((9,) + phase.shape, dtype=torch.float64, device="cuda")
                    p1, st1, _ = ctx.fft_homog_solve(fh.Material(0, phase, params, scale=scale), Ebar, F1,
                                                     options=opts)
                np.testing.assert_allclose(pbar[i], p1, rtol=1e-14, atol=1e-18)
                assert cg[i] == st1["n_cg"], n
        finally:
            b.close()
