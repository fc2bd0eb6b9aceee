"""The seeded input generators: determinism, geometry and the stated statistics."""

import numpy as np

from rve_inputs import (centered_sphere, neo_hookean_config, random_spheres, random_spheres_dense,
                        small_strain_config)


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


def test_two_dimensional_cells():
    from rve_inputs import centered_disk, corner_square, j2_config, random_disks, svk_square_config

    ph, f = centered_disk(199, 0.007, nz=1)
    assert ph.shape == (199, 199, 1) and abs(f - 0.007) < 5e-4
    assert np.array_equal(ph[:, :, 0], ph[::-1, :, 0]) and np.array_equal(ph[:, :, 0], ph[:, :, 0].T)
    sq = corner_square(48, nz=2)
    assert sq.shape == (48, 48, 2) and sq[:16, :16].all() and sq.sum() == 16 * 16 * 2
    ph, params, Fbar = svk_square_config(48, nz=2)
    assert params[1, 0] == 10 * params[0, 0] and Fbar[1] == 0.1 and Fbar[0] == Fbar[4] == Fbar[8] == 1.0
    d = random_disks(96, seed=3, nz=2)
    assert np.array_equal(d, random_disks(96, seed=3, nz=2))
    assert np.array_equal(d[:, :, 0], d[:, :, 1]) and 0.25 <= d.mean() < 0.35
    ph, params, plastic, Ebar = j2_config(48, 0, nz=2)
    assert ph.shape == (48, 48, 2) and np.allclose(plastic[1], 2 * plastic[0])
    assert Ebar[0] == Ebar[4] == 0.01 and Ebar[8] == 0.0


def test_dense_packing_passes_the_rsa_jamming_limit_without_overlap():
    ph, c, r = random_spheres_dense(48, seed=3, r_min=1.5, r_max=3.75, target_fraction=0.4, return_spheres=True)
    assert 0.40 <= ph.mean() < 0.42
    assert r.min() >= 0.75 - 1e-12 and r.max() <= 3.75
    box = np.array(ph.shape, dtype=float)
    d = c[:, None, :] - c[None, :, :]
    d -= box * np.round(d / box)
    dist = np.sqrt((d * d).sum(-1))
    gap = dist - (r[:, None] + r[None, :])
    np.fill_diagonal(gap, 1.0)
    assert gap.min() >= 0.0
    # every stamped voxel lies in some sphere and every voxel centre inside a sphere is stamped
    idx = np.stack(np.meshgrid(*[np.arange(n) + 0.5 for n in ph.shape], indexing="ij"), -1).reshape(-1, 3)
    inside = np.zeros(idx.shape[0], bool)
    for ci, ri in zip(c, r):
        e = idx - ci
        e -= box * np.round(e / box)
        inside |= (e * e).sum(1) <= ri * ri
    assert np.array_equal(inside.reshape(ph.shape), ph.astype(bool))
    assert np.array_equal(ph, random_spheres_dense(48, seed=3, r_min=1.5, r_max=3.75, target_fraction=0.4))


def test_dense_packing_equals_plain_rsa_below_the_first_stall():
    a = random_spheres(40, seed=5, r_min=2.0, r_max=4.0, target_fraction=0.15)
    b = random_spheres_dense(40, seed=5, r_min=2.0, r_max=4.0, target_fraction=0.15)
    assert np.array_equal(a, b)
