"""The trained warm-start network against the zero initial guess.

Twelve held-out 64^3 cells of the training distribution (seeds disjoint from
the training, validation and benchmark cells; six with an inclusion fraction
at or below 0.3 and six between 0.32 and 0.4) are solved to Newton tolerance
1e-8 from Fbar and from the committed network's prediction. The warm start
must converge in every cell, reach the same field (within the Newton
tolerance), need no more Newton iterations and at least 5 % fewer CG
iterations on average, over all twelve cells and over the six above 0.3.
(The 256-cell evaluation of the committed network saves 16 % of the CG
iterations; Newton counts are integers of about 3, too coarse to threshold
on a handful of cells.)
"""

import os

import numpy as np
import pytest

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2408_03804_gb300", "weights", "fno_neo_hookean_64.npy")


def test_trained_network_saves_newton_iterations():
    torch = require_gpu()
    import paper_2408_03804_gb300 as fh
    from paper_2408_03804_gb300 import warm_start as ws

    theta = np.load(WEIGHTS)
    assert theta.size == fh.load().fh_fno_param_count()
    n = 64
    low = [k for k in range(3_000_000, 3_000_200) if ws.cell_fraction(k) <= 0.3][:6]
    high = [k for k in range(3_000_000, 3_000_200) if ws.cell_fraction(k) > 0.32][:6]
    rows = ws.evaluate(n, theta, low + high, workers=1)
    s = ws.summarize(rows)
    assert s["converged_both"] == 12, rows
    assert s["max_field_diff"] < 1e-7, s
    for part in (s, s["fraction_gt_0.3"]):
        assert part["newton_warm"] <= part["newton_zero"], s
        assert part["cg_warm"] <= 0.95 * part["cg_zero"], s
    assert s["fraction_gt_0.3"]["converged_both"] == 6, s
