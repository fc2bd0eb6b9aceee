"""The trained warm-start network against the zero initial guess.

Eight held-out 64^3 cells of the training distribution (seeds disjoint from
the training, validation and benchmark cells) are solved to Newton tolerance
1e-8 from Fbar and from the committed network's prediction. The warm start
must converge in every cell, reach the same field (within the Newton
tolerance) and save Newton iterations on average.
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
    rows = ws.evaluate(n, theta, range(3_000_000, 3_000_008), workers=1)
    s = ws.summarize(rows)
    assert s["converged_both"] == 8, rows
    assert s["max_field_diff"] < 1e-7, s
    assert s["newton_warm"] <= s["newton_zero"] - 0.25, s
