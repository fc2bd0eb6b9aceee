"""Host-side logic of the learned warm start (no GPU): the training-cell recipe and the
parameter vector the driver initialises, against the network's layout in the oracle."""

import numpy as np
import pytest

from oracle import fno as ofno


def test_cells_follow_the_recipe_and_are_seeded():
    pytest.importorskip("torch")
    from paper_2408_03804_gb300 import warm_start as ws

    for seed in (0, 7, 1_000_000):
        ph, Fb = ws.make_cell(32, seed)
        ph2, Fb2 = ws.make_cell(32, seed)
        assert np.array_equal(ph, ph2) and np.array_equal(Fb, Fb2)
        assert ph.shape == (32, 32, 32) and ph.dtype == np.uint8
        assert 0.1 <= ph.mean() <= 0.41
        m = np.linalg.norm(Fb - np.eye(3).reshape(9))
        assert 0.005 <= m <= 0.05 + 1e-12
    assert not np.array_equal(ws.make_cell(32, 1)[0], ws.make_cell(32, 2)[0])


def test_initial_parameters_match_the_network_layout():
    pytest.importorskip("torch")
    from paper_2408_03804_gb300 import warm_start as ws
    from paper_2408_03804_gb300 import build

    build.build()
    th = ws.init_params(0)
    assert th.dtype == np.float32 and th.size == ofno.n_params()
    blocks = {}
    o = 0
    for name, shape in ofno.layout():
        k = int(np.prod(shape))
        blocks[name] = th[o:o + k]
        o += k
    # biases start at zero, spectral weights in [0, 1/C^2)
    for name in ("b0", "m0", "m3", "p1", "p2"):
        assert np.all(blocks[name] == 0), name
    assert 0 <= blocks["W0"].min() and blocks["W0"].max() < 1.0 / 32 ** 2
