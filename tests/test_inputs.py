"""The seeded input generators: determinism, geometry and the stated statistics."""

import numpy as np

from rve_inputs import centered_sphere, neo_hookean_config, random_spheres, small_strain_config


def test_random_spheres_fraction_and_determinism():
    a = random_spheres(32, seed=0, r_min=2.0, r_max=4.0)
    b = random_spheres(32, seed=0, r_min=2.0, r_max=4.0)
    c = random_spheres(32, seed=1, r_min=2.0, r_max=4.0)
    assert a.dtype == np.uint8 and a.shape == (32, 32, 32)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    f = a.mean()
    assert 0.30 <= f < 0.32


def test_centered_sphere_is_symmetric_and_has_expected_volume():
    ph = centered_sphere((16, 16, 16), 0.25)
    assert np.array_equal(ph, ph[::-1]) and np.array_equal(ph, ph.transpose(1, 0, 2))
    # voxel count close to the continuum volume 4/3 pi 4^3 = 268
    assert abs(int(ph.sum()) - 4 / 3 * np.pi * 64) < 30


def test_configs_shapes():
    phase, params, E = small_strain_config(16)
    assert phase.shape == (16, 16, 16) and params.shape == (2, 2)
    assert E[1] == E[3] == 0.01 and np.count_nonzero(E) == 2
    phase, params, F = neo_hookean_config(48, seed=2)
    assert abs(phase.mean() - 0.30) < 0.03
    np.testing.assert_array_equal(params, [[1.5, 1.0], [15.0, 10.0]])
