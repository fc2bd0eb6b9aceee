"""Learned warm start: data generation, training and evaluation on the GPU.

Every numerical step runs in the CUDA library (fft_homog_solve for the
training data, fh_fno_forward / fh_fno_loss_grad / fh_fno_adam for training,
fh_fno_warm_start + fft_homog_solve for evaluation); this module only
arranges cells into batches and records counts and times.

Workload (neo-Hookean cells like the 128^3 benchmark): matrix (lambda, mu) =
(1.5, 1), inclusions 10x, random non-overlapping spheres of radius
U[4, 10]/128 of the box filling a volume fraction U[0.1, 0.4] (random
sequential addition whose radius range shrinks when additions stall, since
plain RSA jams near 0.38; rve_inputs.random_spheres_dense), and a
macroscopic tensor Fbar = I + m d with d uniform on the unit sphere of the
nine entries and m ~ U[0.005, 0.05] (so |Fbar - I| <= 0.05). Each training
target is the solver's converged fluctuation (F - Fbar)/|Fbar - I| at Newton
tolerance 1e-8.

Command line (writes JSON lines to stdout):
  python -m paper_2408_03804_gb300.warm_start train --n 64 --n-train 4096 --epochs 30 --out fno.npy
  python -m paper_2408_03804_gb300.warm_start evaluate --weights fno.npy --n 64 --cases 256
"""

from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import sys
import time

import numpy as np

from . import _binding as B

MATRIX = (1.5, 1.0)
CONTRAST = 10.0
NEWTON_TOL = 1e-8


def params_table() -> np.ndarray:
    lam, mu = MATRIX
    return np.array([[lam, mu], [CONTRAST * lam, CONTRAST * mu]], dtype=np.float64)


def cell_fraction(seed: int) -> float:
    """Target inclusion fraction of the seeded cell ``seed`` (the first draw of its recipe)."""
    return float(np.random.default_rng([seed, 20240807]).uniform(0.1, 0.4))


def make_cell(n: int, seed: int):
    """Phase map (uint8 n^3) and Fbar (9) of the seeded cell ``seed``."""
    from rve_inputs import random_spheres_dense

    rng = np.random.default_rng([seed, 20240807])
    frac = rng.uniform(0.1, 0.4)
    phase = random_spheres_dense(n, seed, r_min=4.0 * n / 128, r_max=10.0 * n / 128, target_fraction=frac)
    d = rng.normal(size=9)
    d /= np.linalg.norm(d)
    Fbar = np.eye(3).reshape(9) + rng.uniform(0.005, 0.05) * d
    return phase, Fbar


def _cell_job(args):
    return make_cell(*args)


def cells(n: int, seeds, workers: int):
    """Yield (seed, phase, Fbar) for every seed, generated on ``workers`` processes."""
    if workers <= 1:
        for s in seeds:
            yield (s,) + make_cell(n, s)
        return
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        for s, (ph, fb) in zip(seeds, pool.imap(_cell_job, [(n, s) for s in seeds], chunksize=4)):
            yield s, ph, fb


def init_params(seed: int) -> np.ndarray:
    """Seeded initial parameters in the order of include/fh_fno.h."""
    rng = np.random.default_rng(seed)
    C, L, K, H = 32, 4, 12, 128
    parts = [rng.uniform(-1, 1, C), rng.uniform(-1, 1, C * 9) / 3.0, np.zeros(C)]
    for _ in range(L):
        parts += [rng.uniform(0, 1, 3 * K * 2 * C * C) / (C * C), rng.uniform(-1, 1, C * C) / math.sqrt(C),
                  np.zeros(C)]
    parts += [rng.uniform(-1, 1, H * C) / math.sqrt(C), np.zeros(H), rng.uniform(-1, 1, 81 * H) / math.sqrt(H),
              np.zeros(81)]
    th = np.concatenate(parts).astype(np.float32)
    assert th.size == B.load().fh_fno_param_count()
    return th


def solve_cell(ctx, phase_dev, Fbar, F, n_increments: int = 1, init_given: bool = False):
    """Newton-Krylov solve of one neo-Hookean cell; returns (stats, return code)."""
    mat = B.Material(B.NEO_HOOKEAN, phase_dev, params_table())
    opts = B.default_options(newton_tol=NEWTON_TOL, init=B.INIT_GIVEN if init_given else B.INIT_REFERENCE)
    _, stats, rc = ctx.fft_homog_solve(mat, Fbar, F, n_increments=n_increments, options=opts,
                                       allow=(B.FH_ERR_NOT_CONVERGED, B.FH_ERR_NONPHYSICAL))
    return stats, rc


def generate(n: int, seeds, workers: int, log=None):
    """Solve every cell and keep phases and normalised targets on the device."""
    import torch

    seeds = list(seeds)
    phases = torch.empty((len(seeds), n, n, n), dtype=torch.uint8, device="cuda")
    targets = torch.empty((len(seeds), 9, n, n, n), dtype=torch.float32, device="cuda")
    Fbars = np.zeros((len(seeds), 9))
    t0 = time.time()
    solve_s = 0.0
    newton = cg = 0
    with B.Context(n, n, n) as ctx, B.Fno(n, n, n, max_batch=1) as net:
        F = torch.empty((9, n, n, n), dtype=torch.float64, device="cuda")
        for i, (s, ph, fb) in enumerate(cells(n, seeds, workers)):
            phases[i].copy_(torch.as_tensor(ph))
            Fbars[i] = fb
            t = time.time()
            F.zero_()
            st, rc = solve_cell(ctx, phases[i], fb, F)
            if rc != B.FH_OK:  # fall back to load increments
                F.zero_()
                st, rc = solve_cell(ctx, phases[i], fb, F, n_increments=5)
            if rc != B.FH_OK:
                raise RuntimeError(f"cell {s} did not converge")
            solve_s += time.time() - t
            newton += st["n_newton"]
            cg += st["n_cg"]
            net.make_target(F, fb, targets[i])
            if log and (i + 1) % 256 == 0:
                log({"generated": i + 1, "wall_s": time.time() - t0, "solve_s": solve_s})
    return phases, targets, Fbars, {"cells": len(seeds), "wall_s": time.time() - t0, "solve_s": solve_s,
                                    "newton": newton, "cg": cg}


def train(n: int, phases, targets, Fbars, epochs: int, batch: int = 8, lr: float = 1e-3, wd: float = 1e-4,
          seed: int = 0, val=None, log=None, time_budget_s: float | None = None):
    """Adam on the mean squared error; cosine learning-rate decay. Returns (theta, history)."""
    import torch

    th = torch.as_tensor(init_params(seed)).cuda()
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    g = torch.empty_like(th)
    n_train = phases.shape[0]
    steps_per_epoch = n_train // batch
    total = epochs * steps_per_epoch
    rng = np.random.default_rng(seed + 1)
    hist = []
    t0 = time.time()
    step = 0
    with B.Fno(n, n, n, max_batch=batch, train=True) as net:
        for ep in range(epochs):
            perm = rng.permutation(n_train)
            run = 0.0
            for k in range(steps_per_epoch):
                idx = perm[k * batch:(k + 1) * batch]
                ph = [phases[i] for i in idx]
                tg = [targets[i] for i in idx]
                net.set_params(th)
                net.forward(ph, Fbars[idx])
                run += net.loss_grad(tg, g)
                step += 1
                rate = lr * 0.5 * (1.0 + math.cos(math.pi * step / total))
                net.adam(th, g, m, v, step, rate, wd=wd)
            rec = {"epoch": ep + 1, "train_loss": run / steps_per_epoch, "wall_s": time.time() - t0}
            if val is not None:
                if ep == 0:  # loss of the zero prediction: the mean square of the targets
                    zero_loss = evaluate_loss(net, torch.zeros_like(th), *val, batch=batch)
                rec["val_loss"] = evaluate_loss(net, th, *val, batch=batch)
                rec["val_rel_err"] = math.sqrt(rec["val_loss"] / zero_loss)
            hist.append(rec)
            if log:
                log(rec)
            if time_budget_s is not None and time.time() - t0 > time_budget_s:
                break
    return th, hist


def evaluate_loss(net, th, phases, targets, Fbars, batch: int = 8) -> float:
    net.set_params(th)
    tot, cnt = 0.0, 0
    for k in range(0, phases.shape[0] - batch + 1, batch):
        ph = [phases[i] for i in range(k, k + batch)]
        net.forward(ph, Fbars[k:k + batch])
        tot += net.loss_grad([targets[i] for i in range(k, k + batch)])
        cnt += 1
    return tot / max(cnt, 1)


def evaluate(n: int, theta, seeds, workers: int, n_increments: int = 1, log=None):
    """Zero-guess solve vs warm-started solve of every cell: counts and device-synchronised times."""
    import torch

    rows = []
    with B.Context(n, n, n) as ctx, B.Fno(n, n, n, max_batch=1) as net:
        net.set_params(torch.as_tensor(np.asarray(theta, dtype=np.float32)).cuda())
        F = torch.empty((9, n, n, n), dtype=torch.float64, device="cuda")
        for s, ph, fb in cells(n, seeds, workers):
            phd = torch.as_tensor(ph).cuda()
            torch.cuda.synchronize()
            t = time.perf_counter()
            F.zero_()
            st0, rc0 = solve_cell(ctx, phd, fb, F, n_increments=n_increments)
            torch.cuda.synchronize()
            t_zero = time.perf_counter() - t
            P0 = F.clone()
            t = time.perf_counter()
            net.warm_start(ctx, phd, fb, F)
            torch.cuda.synchronize()
            t_inf = time.perf_counter() - t
            st1, rc1 = solve_cell(ctx, phd, fb, F, init_given=True)
            torch.cuda.synchronize()
            t_warm = time.perf_counter() - t
            diff = float((F - P0).abs().max())
            rows.append({"seed": int(s), "fraction": float(ph.mean()), "rc": [rc0, rc1],
                         "newton": [st0["n_newton"], st1["n_newton"]],
                         "cg": [st0["n_cg"], st1["n_cg"]], "s": [t_zero, t_warm], "inference_s": t_inf,
                         "max_field_diff": diff})
            if log:
                log(rows[-1])
    return rows


def summarize(rows, split: float | None = 0.3):
    """Means over the cells that converged from both starts; with ``split``, also for the cells at or below
    and above that inclusion fraction."""
    out = _summary(rows)
    if split is not None:
        out["fraction_le_%g" % split] = _summary([r for r in rows if r.get("fraction", 0.0) <= split])
        out["fraction_gt_%g" % split] = _summary([r for r in rows if r.get("fraction", 0.0) > split])
    return out


def _summary(rows):
    ok = [r for r in rows if r["rc"] == [0, 0]]
    f = lambda key, i: float(np.mean([r[key][i] for r in ok])) if ok else float("nan")  # noqa: E731
    return {"cases": len(rows), "converged_both": len(ok),
            "newton_zero": f("newton", 0), "newton_warm": f("newton", 1),
            "cg_zero": f("cg", 0), "cg_warm": f("cg", 1),
            "s_zero": f("s", 0), "s_warm": f("s", 1),
            "inference_s": float(np.mean([r["inference_s"] for r in ok])) if ok else float("nan"),
            "time_saved_frac": 1.0 - f("s", 1) / f("s", 0) if ok else float("nan"),
            "max_field_diff": float(max(r["max_field_diff"] for r in ok)) if ok else float("nan")}



def _log(rec):
    print(json.dumps(rec), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train")
    tr.add_argument("--n", type=int, default=64)
    tr.add_argument("--n-train", type=int, default=4096)
    tr.add_argument("--n-val", type=int, default=64)
    tr.add_argument("--epochs", type=int, default=30)
    tr.add_argument("--batch", type=int, default=8)
    tr.add_argument("--lr", type=float, default=1e-3)
    tr.add_argument("--time-budget", type=float, default=None, help="stop training after this many seconds")
    tr.add_argument("--workers", type=int, default=max(1, min(16, (mp.cpu_count() or 2) - 1)))
    tr.add_argument("--out", required=True)
    tr.add_argument("--eval-cases", type=int, default=0)
    ev = sub.add_parser("evaluate")
    ev.add_argument("--weights", required=True)
    ev.add_argument("--n", type=int, default=64)
    ev.add_argument("--cases", type=int, default=256)
    ev.add_argument("--first-seed", type=int, default=1_000_000)
    ev.add_argument("--workers", type=int, default=max(1, min(16, (mp.cpu_count() or 2) - 1)))
    a = ap.parse_args(argv)
    B.load()
    if a.cmd == "train":
        import torch

        # seeds: training 0.., validation 500000.., evaluation 1000000.. (disjoint)
        ph, tg, fb, info = generate(a.n, range(a.n_train), a.workers, log=_log)
        _log({"generation": info})
        vph, vtg, vfb, _ = generate(a.n, range(500_000, 500_000 + a.n_val), a.workers)
        th, hist = train(a.n, ph, tg, fb, a.epochs, batch=a.batch, lr=a.lr, val=(vph, vtg, vfb), log=_log,
                         time_budget_s=a.time_budget)
        np.save(a.out, th.cpu().numpy())
        del ph, tg
        torch.cuda.empty_cache()
        if a.eval_cases:
            rows = evaluate(a.n, th.cpu().numpy(), range(1_000_000, 1_000_000 + a.eval_cases), a.workers)
            _log({"evaluation": summarize(rows), "n": a.n})
    else:
        th = np.load(a.weights)
        rows = evaluate(a.n, th, range(a.first_seed, a.first_seed + a.cases), a.workers)
        _log({"evaluation": summarize(rows), "n": a.n})
    return 0


if __name__ == "__main__":
    sys.exit(main())
