"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds geometry and random numbers only: phase maps (spheres,
random sequential addition of spheres, laminates), material parameter tables
and random deformation fields. It contains none of the homogenization
method's arithmetic (no projection, no constitutive law, no solver), so both
the CPU oracle and the CUDA path may take their inputs from here without
sharing any computational code.

Conventions
-----------
* A grid is ``(nx, ny, nz)``; voxel ``(i, j, k)`` has its centre at
  ``((i + 1/2) h_x, (j + 1/2) h_y, (k + 1/2) h_z)`` in a periodic box of side
  lengths ``L = (1, 1, 1)`` unless stated otherwise.
* A phase map is a C-contiguous ``uint8`` array of shape ``(nx, ny, nz)``
  (z fastest), value ``p`` selecting row ``p`` of a parameter table.
* A parameter table is a float64 array of shape ``(n_phase, 2)`` holding the
  Lame pair ``(lambda, mu)`` of each phase.
* Tensor fields are float64 arrays of shape ``(9, nx, ny, nz)`` with component
  index ``3*i + j`` for the entry ``F_ij`` (row-major 3x3).
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "lame_from_bulk_shear",
    "centered_sphere",
    "random_spheres",
    "laminate",
    "two_phase_table",
    "random_deformation",
    "shear_macro",
    "small_strain_config",
    "neo_hookean_config",
    "simp_density",
    "simp_config",
    "lognormal_modulus",
    "batch_config",
    "random_disks",
    "j2_config",
    "corner_square",
    "svk_square_config",
    "centered_disk",
]


def lame_from_bulk_shear(bulk: float, shear: float) -> tuple[float, float]:
    """Lame pair (lambda, mu) of an isotropic solid from bulk and shear moduli."""
    return bulk - 2.0 * shear / 3.0, shear


def _periodic_sq_dist(n: int, c: float) -> np.ndarray:
    """Squared periodic minimum-image distance (in voxels) of voxel centres to c."""
    x = np.arange(n) + 0.5 - c
    x = x - n * np.round(x / n)
    return x * x


def centered_sphere(n: tuple[int, int, int], radius_frac: float = 0.25,
                    center_frac: tuple[float, float, float] = (0.5, 0.5, 0.5)) -> np.ndarray:
    """Phase map of one sphere (phase 1) in a matrix (phase 0).

    The sphere has radius ``radius_frac * nx`` voxels and its centre at
    ``center_frac * n`` (in voxel units). A voxel is inside iff the periodic
    minimum-image distance of its centre to the sphere centre is <= r.
    """
    nx, ny, nz = n
    r = radius_frac * nx
    d2 = (_periodic_sq_dist(nx, center_frac[0] * nx)[:, None, None]
          + _periodic_sq_dist(ny, center_frac[1] * ny)[None, :, None]
          + _periodic_sq_dist(nz, center_frac[2] * nz)[None, None, :])
    return (d2 <= r * r).astype(np.uint8)


def _stamp_sphere(phase: np.ndarray, c: np.ndarray, r: float) -> int:
    """Mark the voxels whose centres lie within r of c (periodic); returns how many were newly filled."""
    shape = phase.shape
    lo = np.floor(c - r - 1).astype(int)
    hi = np.ceil(c + r + 1).astype(int)
    ix = np.arange(lo[0], hi[0] + 1)
    iy = np.arange(lo[1], hi[1] + 1)
    iz = np.arange(lo[2], hi[2] + 1)
    dx = ix + 0.5 - c[0]
    dy = iy + 0.5 - c[1]
    dz = iz + 0.5 - c[2]
    inside = (dx[:, None, None] ** 2 + dy[None, :, None] ** 2 + dz[None, None, :] ** 2) <= r * r
    sel = np.ix_(ix % shape[0], iy % shape[1], iz % shape[2])
    sub = phase[sel]
    # a sphere wider than a short axis may wrap onto itself: count each voxel once
    keys = (ix % shape[0])[:, None, None] * (shape[1] * shape[2]) + \
           (iy % shape[1])[None, :, None] * shape[2] + (iz % shape[2])[None, None, :]
    new_vox = np.unique(keys[inside & (sub == 0)])
    sub[inside] = 1
    phase[sel] = np.maximum(phase[sel], sub)
    return int(new_vox.size)


def random_spheres(n, seed: int, r_min: float = 4.0, r_max: float = 10.0,
                   target_fraction: float = 0.30, max_attempts: int = 200000) -> np.ndarray:
    """Random sequential addition of non-overlapping spheres on a periodic grid.

    ``n`` is an int (an n^3 cube) or a shape (nx, ny, nz), in voxels of unit
    size. Radii are drawn uniformly in [r_min, r_max] voxels and centres
    uniformly in the periodic box; a candidate is rejected when its periodic
    centre distance to any accepted sphere is below the sum of the radii.
    Spheres are added until the voxelised inclusion fraction first reaches
    ``target_fraction``. Returns a uint8 phase map (1 = inclusion).
    """
    shape = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
    box = np.asarray(shape, dtype=np.float64)
    rng = np.random.default_rng(seed)
    phase = np.zeros(shape, dtype=np.uint8)
    centres: list[np.ndarray] = []
    radii: list[float] = []
    filled = 0
    target = target_fraction * phase.size
    for _ in range(max_attempts):
        if filled >= target:
            break
        r = rng.uniform(r_min, r_max)
        c = rng.uniform(0.0, 1.0, size=3) * box
        if centres:
            d = np.asarray(centres) - c
            d -= box * np.round(d / box)
            if np.any(np.sqrt((d * d).sum(axis=1)) < np.asarray(radii) + r):
                continue
        centres.append(c)
        radii.append(r)
        filled += _stamp_sphere(phase, c, r)
    else:
        raise RuntimeError("random_spheres: target fraction not reached")
    return phase


def random_spheres_dense(n, seed: int, r_min: float, r_max: float, target_fraction: float,
                         r_floor: float | None = None, patience: int = 500, shrink: float = 0.85,
                         max_attempts: int = 3_000_000, return_spheres: bool = False):
    """Random sequential addition that keeps going past the jamming limit of plain RSA (about 0.38).

    As ``random_spheres`` (radius uniform in [lo, hi], centre uniform, rejected on periodic overlap),
    starting from [lo, hi] = [r_min, r_max]; after ``patience`` consecutive rejections the range
    shrinks: hi by the factor ``shrink`` (not below lo), and once hi = lo both shrink, down to
    ``r_floor`` (default r_min / 2). Until the first stall the draws are those of plain RSA. Spheres
    never overlap. Returns a uint8 phase map (1 = inclusion) at the first fraction >= target, and with
    ``return_spheres`` also the centres (k, 3) and radii (k,) in voxel units.
    """
    shape = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
    box = np.asarray(shape, dtype=np.float64)
    floor_r = r_min / 2.0 if r_floor is None else r_floor
    rng = np.random.default_rng(seed)
    phase = np.zeros(shape, dtype=np.uint8)
    centres = np.zeros((0, 3))
    radii = np.zeros(0)
    filled, fails = 0, 0
    lo, hi = r_min, r_max
    target = target_fraction * phase.size
    for _ in range(max_attempts):
        if filled >= target:
            break
        r = rng.uniform(lo, hi)
        c = rng.uniform(0.0, 1.0, size=3) * box
        if radii.size:
            d = centres - c
            d -= box * np.round(d / box)
            if np.any(np.sqrt((d * d).sum(axis=1)) < radii + r):
                fails += 1
                if fails >= patience:
                    fails = 0
                    if hi > lo:
                        hi = max(lo, hi * shrink)
                    else:
                        lo = hi = max(floor_r, lo * shrink)
                continue
        fails = 0
        centres = np.vstack([centres, c])
        radii = np.append(radii, r)
        filled += _stamp_sphere(phase, c, r)
    else:
        raise RuntimeError("random_spheres_dense: target fraction not reached")
    return (phase, centres, radii) if return_spheres else phase


def laminate(n: tuple[int, int, int], thickness: int, axis: int = 0) -> np.ndarray:
    """Two-phase laminate: phase 1 on the first ``thickness`` layers along ``axis``."""
    phase = np.zeros(n, dtype=np.uint8)
    idx = [slice(None)] * 3
    idx[axis] = slice(0, thickness)
    phase[tuple(idx)] = 1
    return phase


def two_phase_table(lam: float, mu: float, contrast: float) -> np.ndarray:
    """Parameter table: phase 0 = (lam, mu), phase 1 = contrast * (lam, mu)."""
    return np.array([[lam, mu], [contrast * lam, contrast * mu]], dtype=np.float64)


def random_deformation(n_vox: int, seed: int, scale: float = 0.1,
                       identity: bool = True) -> np.ndarray:
    """Random 3x3 tensors as a (9, n_vox) float64 array: I + scale * U(-1, 1)."""
    rng = np.random.default_rng(seed)
    F = rng.uniform(-scale, scale, size=(9, n_vox))
    if identity:
        F[[0, 4, 8]] += 1.0
    return F


def shear_macro(gamma: float, finite: bool) -> np.ndarray:
    """Macroscopic tensor with a simple shear gamma e_x (x) e_y (entry 01).

    With ``finite`` it is the deformation gradient I + gamma e_x (x) e_y; else
    the small-strain tensor with eps_xy = eps_yx = gamma.
    """
    F = np.zeros(9)
    if finite:
        F[[0, 4, 8]] = 1.0
        F[1] = gamma
    else:
        F[1] = F[3] = gamma
    return F


def small_strain_config(n: int = 16):
    """Two-phase linear elastic cube: centred sphere of radius 0.25 L.

    Matrix bulk 0.833 and shear 0.386; the inclusion is 10x stiffer. The
    macroscopic strain has only eps_xy = eps_yx = 0.01.
    Returns (phase, params, Ebar).
    """
    lam, mu = lame_from_bulk_shear(0.833, 0.386)
    phase = centered_sphere((n, n, n), 0.25)
    params = np.array([[lam, mu], list(lame_from_bulk_shear(8.33, 3.86))], dtype=np.float64)
    return phase, params, shear_macro(0.01, finite=False)


def neo_hookean_config(n=128, seed: int = 0):
    """Random-sphere neo-Hookean cell: matrix mu=1, lambda=1.5, inclusions 10x.

    ``n`` is the cube edge in voxels or a shape (nx, ny, nz).

    Spheres of radius U[4, 10] voxels fill a volume fraction of 0.3. The
    macroscopic deformation gradient is I + 0.05 e_x (x) e_y.
    Returns (phase, params, Fbar).
    """
    phase = random_spheres(n, seed)
    params = two_phase_table(1.5, 1.0, 10.0)
    return phase, params, shear_macro(0.05, finite=True)


def simp_density(n, seed: int, sigma: float = 2.0, rho_min: float = 0.01) -> np.ndarray:
    """Smoothed seeded noise rescaled to [rho_min, 1] (a SIMP density field).

    Uniform noise on an n^3 (or (nx, ny, nz)) grid is smoothed by a periodic
    Gaussian filter of standard deviation ``sigma`` voxels and min-max
    rescaled to [rho_min, 1].
    """
    from scipy.ndimage import gaussian_filter

    shape = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
    rng = np.random.default_rng(seed)
    t = gaussian_filter(rng.uniform(size=shape), sigma=sigma, mode="wrap")
    t = (t - t.min()) / (t.max() - t.min())
    return rho_min + (1.0 - rho_min) * t


def simp_config(n: int = 64, seed: int = 0, penalty: float = 3.0, nu: float = 0.3):
    """SIMP cell: one phase with E = 1, nu = 0.3, scaled per voxel by rho^penalty.

    Returns (phase, params, rho, scale, dscale) with scale = rho^p and
    dscale = p rho^(p-1) (the derivative of the modulus scale).
    """
    rho = simp_density(n, seed)
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    phase = np.zeros(rho.shape, dtype=np.uint8)
    params = np.array([[lam, mu]], dtype=np.float64)
    return phase, params, rho, rho ** penalty, penalty * rho ** (penalty - 1)


def lognormal_modulus(n, seed: int, corr: float = 0.1, sigma_log: float = 0.3) -> np.ndarray:
    """Log-normal modulus field E = exp(sigma_log * g) about a median of 1.

    g is a unit-variance Gaussian random field on the periodic grid with the
    covariance exp(-r^2 / (2 l^2)), l = corr * (box edge): white noise filtered
    in Fourier space by the square root of the covariance's spectrum, then
    scaled to unit sample variance.
    """
    shape = (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape)
    d2 = np.zeros(shape)
    for a, m in enumerate(shape):
        x = np.arange(m, dtype=np.float64)
        x = np.minimum(x, m - x) / m  # periodic distance in box units
        sh = [1, 1, 1]
        sh[a] = m
        d2 = d2 + (x ** 2).reshape(sh)
    cov = np.exp(-d2 / (2.0 * corr ** 2))
    spec = np.maximum(np.fft.rfftn(cov).real, 0.0)
    g = np.fft.irfftn(np.fft.rfftn(w) * np.sqrt(spec), s=shape, axes=(0, 1, 2))
    g = (g - g.mean()) / g.std()
    return np.exp(sigma_log * g)


def batch_config(n_cells: int = 256, seed: int = 0, sizes=(32, 48, 64, 96), nu: float = 0.3):
    """Cells of uneven cubic grids with log-normal Young's modulus fields.

    Sizes are drawn uniformly from ``sizes`` (seeded); cell i has the modulus
    field lognormal_modulus(n_i, seed + 1 + i). All cells are linear elastic
    with E = 1 (median), nu = 0.3, and share the macroscopic strain
    eps_xx = 0.01. Returns (list of (phase, scale) per cell, params, Ebar).
    """
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=n_cells)
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    params = np.array([[lam, mu]], dtype=np.float64)
    cells = []
    for i, n in enumerate(ns):
        E = lognormal_modulus(int(n), seed + 1 + i)
        cells.append((np.zeros(E.shape, dtype=np.uint8), E))
    Ebar = np.zeros(9)
    Ebar[0] = 0.01
    return cells, params, Ebar


def random_disks(n: int, seed: int, nz: int = 1, r_min: float = 6.0, r_max: float = 14.0,
                 target_fraction: float = 0.25, max_attempts: int = 200000) -> np.ndarray:
    """Random sequential addition of non-overlapping disks on an n x n periodic grid.

    The same rule as ``random_spheres`` in the (x, y) plane; the map is
    repeated ``nz`` times along z, so the cell is invariant along z (a 2D
    cell; nz = 1 for the oracle, nz = 2 for the GPU's even-z layout).
    Returns a uint8 phase map (n, n, nz), 1 = inclusion.
    """
    rng = np.random.default_rng(seed)
    phase = np.zeros((n, n), dtype=np.uint8)
    centres: list[np.ndarray] = []
    radii: list[float] = []
    x = np.arange(n) + 0.5
    target = target_fraction * phase.size
    for _ in range(max_attempts):
        if int(phase.sum()) >= target:
            break
        r = rng.uniform(r_min, r_max)
        c = rng.uniform(0.0, n, size=2)
        if centres:
            d = np.asarray(centres) - c
            d -= n * np.round(d / n)
            if np.any(np.sqrt((d * d).sum(axis=1)) < np.asarray(radii) + r):
                continue
        centres.append(c)
        radii.append(r)
        dx = x - c[0]
        dx -= n * np.round(dx / n)
        dy = x - c[1]
        dy -= n * np.round(dy / n)
        phase[(dx[:, None] ** 2 + dy[None, :] ** 2) <= r * r] = 1
    else:
        raise RuntimeError("random_disks: target fraction not reached")
    return np.repeat(phase[:, :, None], nz, axis=2).copy()


def j2_config(n: int = 192, seed: int = 0, nz: int = 1, nu: float = 0.3):
    """Two-phase J2 elastoplastic cell with hard circular inclusions.

    Disks of radius U[6, 14] * n / 192 voxels fill an area fraction of 0.25
    in an elastic matrix of the same stiffness (E = 1, nu = 0.3 in both
    phases). Matrix yield stress 2e-3 and hardening modulus 0.05; the
    inclusions have twice both (a yield and hardening contrast of 2). The
    load is the biaxial small strain eps_xx = eps_yy = 0.01 (plane strain,
    eps_zz = 0). Returns (phase, params, plastic, Ebar).
    """
    k = n / 192.0
    phase = random_disks(n, seed, nz=nz, r_min=6.0 * k, r_max=14.0 * k)
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    params = np.array([[lam, mu], [lam, mu]], dtype=np.float64)
    plastic = np.array([[2e-3, 0.05], [4e-3, 0.10]], dtype=np.float64)
    Ebar = np.zeros(9)
    Ebar[0] = Ebar[4] = 0.01
    return phase, params, plastic, Ebar


def corner_square(n: int, frac: float = 1.0 / 3.0, nz: int = 1) -> np.ndarray:
    """Square inclusion (phase 1) of side round(frac * n) voxels at the corner x, y < side.

    Repeated nz times along z (a z-invariant 2D cell). Returns uint8 (n, n, nz).
    """
    side = int(round(frac * n))
    phase = np.zeros((n, n, nz), dtype=np.uint8)
    phase[:side, :side, :] = 1
    return phase


def svk_square_config(n: int = 256, nz: int = 1):
    """St. Venant-Kirchhoff cell with a stiff square of side L/3 at a corner, under simple shear.

    Matrix (lambda, mu) = (2, 1), inclusion 10x; Fbar = I + 0.1 e_x (x) e_y.
    Returns (phase, params, Fbar).
    """
    phase = corner_square(n, 1.0 / 3.0, nz)
    params = np.array([[2.0, 1.0], [20.0, 10.0]], dtype=np.float64)
    Fbar = np.eye(3).reshape(9).copy()
    Fbar[1] = 0.1
    return phase, params, Fbar


def centered_disk(n: int, fraction: float = 0.007, nz: int = 1):
    """Disk (phase 1) of area fraction ``fraction`` centred in an n x n cell, repeated nz times.

    A voxel belongs to the disk when its centre lies within r = sqrt(fraction / pi) n of the cell
    centre. Returns (uint8 phase map (n, n, nz), the voxelised area fraction).
    """
    r = np.sqrt(fraction / np.pi) * n
    x = np.arange(n) + 0.5 - n / 2
    ph2 = ((x[:, None] ** 2 + x[None, :] ** 2) <= r * r).astype(np.uint8)
    return np.repeat(ph2[:, :, None], nz, axis=2), float(ph2.mean())
