"""Write the oracle's full-size result for the 128^3 random-sphere neo-Hookean cell.

Workload: 128^3 voxels, random sequential addition of spheres (radius
U[4, 10] voxels, seed 0) to a volume fraction of 0.3, matrix (lambda, mu) =
(1.5, 1), inclusions 10x stiffer, Fbar = I + 0.05 e_x (x) e_y reached in 5
equal increments, Newton tolerance 1e-8, CG tolerance 1e-10.

Only the CPU oracle (``oracle/``) and the seeded input generator
(``rve_inputs``) are used. Outputs: ``neo_hookean_128_seed0.json`` with the
homogenized stress, the Newton residual and CG-count history, the oracle's
wall time and core count, and the deformation gradient at 64 sampled voxels;
``neo_hookean_128_seed0_planes.npy``, every voxel of the x-planes listed in
the JSON (``planes_x``) as float64 [9][len(planes_x)][128][128], and the
per-component maximum of |F - Fbar| over the whole field (``fluct_max``).

Run from the repository root:  python tests/golden/make_neo_hookean_128.py
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import solver  # noqa: E402
from rve_inputs import neo_hookean_config  # noqa: E402


def main():
    n, seed = 128, 0
    phase, params, Fbar = neo_hookean_config(n, seed)
    t0 = time.time()
    r = solver.solve(phase, params, 1, Fbar, n_increments=5, newton_tol=1e-8)
    wall = time.time() - t0
    rng = np.random.default_rng(12345)
    idx = rng.integers(0, n, size=(64, 3))
    samples = [{"voxel": [int(i), int(j), int(k)], "F": r.F[:, i, j, k].tolist()} for i, j, k in idx]
    planes_x = [0, 77]
    here = os.path.dirname(os.path.abspath(__file__))
    np.save(os.path.join(here, "neo_hookean_128_seed0_planes.npy"), np.ascontiguousarray(r.F[:, planes_x]))
    fluct_max = np.abs(r.F - Fbar.reshape(9, 1, 1, 1)).reshape(9, -1).max(axis=1)
    out = {
        "workload": "neo-Hookean 128^3, RSA spheres r~U[4,10] seed 0, f=0.3, contrast 10, "
                    "Fbar = I + 0.05 e_x(x)e_y in 5 increments, newton_tol 1e-8, cg_tol 1e-10",
        "phase_fraction": float(phase.mean()),
        "Pbar": r.Pbar.tolist(),
        "newton_residuals": r.newton_residuals,
        "cg_iterations": r.cg_iterations,
        "n_newton": len(r.newton_residuals),
        "n_cg": int(sum(r.cg_iterations)),
        "oracle_wall_s": wall,
        "oracle_cores": os.cpu_count(),
        "samples": samples,
        "planes_x": planes_x,
        "fluct_max": fluct_max.tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "neo_hookean_128_seed0.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, wall)


if __name__ == "__main__":
    main()
