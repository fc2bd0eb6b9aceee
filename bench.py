"""Benchmark: time-to-solve of the 128^3 neo-Hookean cell on the GB300 library.

One step = one complete Newton-Krylov solve (Appendix A, Algorithm 1) of the
128^3 random-sphere neo-Hookean cell: Fbar = I + 0.05 e_x (x) e_y reached in
5 increments, Newton tolerance 1e-8 on ||dF||/(||Fbar|| sqrt(N)), CG
tolerance 1e-10, every kernel of the path (AD constitutive evaluation, the
five FFT/projection passes, CG and Newton updates) in the CUDA library.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle
instead (the reference arm). Under torchrun every rank solves its own
replica (seed = rank); nothing is exchanged between ranks but the barrier and
the max of the timings.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 128
N_INC = 5
NEWTON_TOL = 1e-8
WARM_WEIGHTS = os.path.join(ROOT, "paper_2408_03804_gb300", "weights", "fno_neo_hookean_64.npy")
GAMMA = 0.05
METRIC = "time-to-solve @1e-8 residual (128³ neo-Hookean); CG matvec GB/s vs HBM peak"
WORKLOAD = ("neo-Hookean 128^3, RSA spheres r~U[4,10] vox, f=0.30, contrast 10 (mu=1, lambda=1.5), "
            "Fbar=I+0.05 e_x(x)e_y in 5 increments, Newton tol 1e-8, CG tol 1e-10, FP64")
def l2_note(shape) -> str:
    """The working set of one CG iteration (fields, packed tangent, spectrum: about 0.8 KB per voxel)."""
    gb = 810.0 * shape[0] * shape[1] * shape[2] / 1e9
    return f"working set ~{gb:.1f} GB per solve (inputs larger than L2), no explicit flush"
HBM_PEAK_FALLBACK = 6694.5
# FP64 issue rate from unit counts and clock (152 SMs x 2 FP64 FMA lanes per
# clock x 2.07 GHz), used only when the live DFMA probe cannot run
FP64_LANE_PEAK_DERIVED = 152 * 2 * 2.07e9


# ---------------------------------------------------------------------------
# algorithmic work per launch of each kernel class (bytes moved at minimum,
# FP64 flops with the conventional 5 L log2 L count per complex length-L FFT)
# ---------------------------------------------------------------------------
def algorithmic_work(cls: str, nx: int, ny: int, nz: int):
    n = nx * ny * nz
    h = nx * ny * (nz // 2 + 1)
    c16 = 16  # bytes of a complex double
    lg = math.log2
    if cls == "fwd_z":        # read r, p, x, K(45); write p, x; write 9 half spectra
        return (72 + 72 + 72 + 360 + 72 + 72) * n + 9 * c16 * h, (162 + 36) * n + 9 * 2.5 * n * lg(nz) + 3 * 2 * h
    if cls == "fwd_y":        # read 9, write 6 spectral components
        return (9 + 6) * c16 * h, 9 * 5 * h * lg(ny) + 3 * 4 * h
    if cls == "x_ghat":       # read 6, write 6; 12 transforms + Ghat
        return (6 + 6) * c16 * h, 12 * 5 * h * lg(nx) + 40 * h
    if cls == "inv_y":        # read 6, write 9
        return (6 + 9) * c16 * h, 9 * 5 * h * lg(ny) + 24 * h
    if cls == "inv_z":        # read 9 spectra and p; write y
        return 9 * c16 * h + (72 + 72) * n, 9 * 2.5 * n * lg(nz) + 18 * n
    if cls == "cg_update":    # read r, y; write r (x += alpha p is done by the next forward z pass)
        return 3 * 72 * n, 4 * 9 * n
    return None, None


# FP64 lane operations (DADD, DMUL, DFMA each one) per launch, counted from the
# kernels' code: complex length-L transform per point = FP64_FFT_OPS[L], from the
# compile-time plans of the library (radix of each stage) and the FP64 operations per point of
# an R-point butterfly: BUTTERFLY_OPS for the first stage (no twiddles), TWIDDLED_OPS for the
# later ones (radix 2^P: P layers of 6-FMA butterflies with the twiddles in the tangent form,
# 3 P per point; radix 3: two tangent-form products of 4 operations and the radix-3 butterfly)
FFT_PLANS = {1: (), 2: (2,), 3: (3,), 4: (4,), 6: (2, 3), 8: (8,), 12: (4, 3), 16: (16,), 24: (8, 3),
             32: (8, 4), 48: (16, 3), 64: (8, 8), 96: (8, 4, 3), 128: (16, 8), 192: (16, 4, 3), 256: (16, 4, 4)}
BUTTERFLY_OPS = {2: 2.0, 3: 4.0, 4: 4.0, 8: 6.5, 16: 9.0}
TWIDDLED_OPS = {2: 3.0, 3: 4.0 + 8.0 / 3.0, 4: 6.0, 8: 9.0, 16: 12.0}
FP64_FFT_OPS = {L: sum((TWIDDLED_OPS if k else BUTTERFLY_OPS)[r] for k, r in enumerate(plan))
                for L, plan in FFT_PLANS.items()}


def fp64_ops(cls: str, nx: int, ny: int, nz: int):
    n = nx * ny * nz
    h = nx * ny * (nz // 2 + 1)
    m = nz // 2
    r2c = 9 * (FP64_FFT_OPS[m] * m + 10 * (m // 2 + 1)) * nx * ny  # half-length FFT + unpack (tangent-form pairs)
    if cls == "fwd_z":
        return 99 * n + r2c + 3 * 4 * (m // 2 + 1) * nx * ny
    if cls == "fwd_y":
        return (9 * FP64_FFT_OPS[ny] + 12) * h
    if cls == "x_ghat":
        return (12 * FP64_FFT_OPS[nx] + 30) * h
    if cls == "inv_y":
        return (9 * FP64_FFT_OPS[ny] + 12) * h
    if cls == "inv_z":
        return 9 * n + r2c
    if cls == "cg_update":
        return 18 * n
    return None


def fp64_pipe_frac(cls, shape, avg_s, lane_peak):
    ops = fp64_ops(cls, *shape)
    return ops / avg_s / lane_peak if ops else None


def probe_fp64(fh, local):
    """Measured FP64 FMA lane operations per second (the library's DFMA probe), with the SM clock during it."""
    try:
        shapes = [(2, 8), (4, 8), (8, 8), (2, 16), (4, 16), (4, 4)]
        with ClockSampler(local) as clk:
            runs = {f"{c}cta_{ch}ch": fh.fh_probe_fp64(ctas_per_sm=c, chains=ch, iters=(1 << 20) // (c * ch))
                    for c, ch in shapes}
        rates = {k: ops / (ms / 1e3) for k, (ms, ops) in runs.items()}
        best = max(rates.values())
        return {"lane_ops_per_s": best, "tflops": 2.0 * best / 1e12, "rates": rates,
                "clocks": clk.summary(), "source": "measured in this run: fh_probe_fp64 (independent DFMA chains, "
                                                  "best over CTAs/SM x chains per thread)"}
    except Exception as exc:  # noqa: BLE001 -- report, fall back to the unit-count figure
        return {"lane_ops_per_s": FP64_LANE_PEAK_DERIVED, "tflops": 2.0 * FP64_LANE_PEAK_DERIVED / 1e12,
                "source": f"derived (probe failed: {exc}): 152 SM x 2 FP64 FMA/clk x 2.07 GHz"}


def cg_iteration_bytes(nx, ny, nz):
    return sum(algorithmic_work(c, nx, ny, nz)[0] for c in ("fwd_z", "fwd_y", "x_ghat", "inv_y", "inv_z",
                                                           "cg_update"))


# sources of the projection and CG kernels whose DRAM traffic profiles/ncu_traffic.json records
TRAFFIC_SOURCES = ("kernels_fft.cu", "passes.cuh", "fft_core.cuh", "fh_common.cuh", "fh_kernels.h")


def _code_only(text: str) -> str:
    """C++ source without comments and with whitespace collapsed: what the compiler sees."""
    import re

    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash() -> str:
    """Hash of the code (comments and layout excluded) of the passes whose traffic was captured."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2408_03804_gb300", "csrc")
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh_:
            h.update(_code_only(fh_.read()).encode())
    return h.hexdigest()[:16]


def committed_traffic(kernel_class: str):
    """DRAM bytes per launch from the committed ncu summary, if it matches this source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("source_hash") != kernel_source_hash():
        return None
    ent = d.get("kernels", {}).get(kernel_class)
    if not ent or ent.get("grid") != [N_GRID] * 3:
        return None
    return ent.get("dram_bytes_per_launch")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, src = HBM_PEAK_FALLBACK, "fallback"
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        if "hbm_gbs" in d:
            hbm, src = float(d["hbm_gbs"]), "measured"
    return hbm, src


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed plumbing (barrier and max only)
# ---------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)


def barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist

        if device is not None:
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def max_over_ranks(world, value, device):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle timing on a bounded sample of the workload
# ---------------------------------------------------------------------------
def oracle_sample(phase, params, Fbar, n_cg_iters=6):
    """Seconds per CG iteration and per Newton-step overhead of the oracle at full size.

    The sample is one Newton iteration of the first increment with the CG
    loop capped at n_cg_iters products, timed in two parts.
    """
    from oracle import materials as omat
    from oracle import solver as osolver
    from oracle import spectral

    lam, mu = params[phase, 0], params[phase, 1]
    F = np.broadcast_to(np.eye(3).reshape(9, 1, 1, 1), (9,) + phase.shape).copy()
    F += ((Fbar - np.eye(3).reshape(9)) / N_INC).reshape(9, 1, 1, 1)
    t0 = time.perf_counter()
    P = omat.stress(1, F, lam, mu)
    K = omat.tangent(1, F, lam, mu)
    b = -spectral.project(P)
    t1 = time.perf_counter()
    x, it, _ = osolver.cg(lambda p: spectral.project(omat.apply_tangent(K, p)), b, 1e-30, n_cg_iters)
    F += x
    _ = float(np.linalg.norm(x))
    t2 = time.perf_counter()
    return (t2 - t1) / max(it, 1), t1 - t0, it


def reference_counts():
    path = os.path.join(ROOT, "tests", "golden", "neo_hookean_128_seed0.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    return d["n_newton"], d["n_cg"]


def oracle_full_solve_record():
    """The oracle's one recorded full solve of this workload (stored with its golden values)."""
    path = os.path.join(ROOT, "tests", "golden", "neo_hookean_128_seed0.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    return {"wall_s": d.get("oracle_wall_s"), "cores": d.get("oracle_cores"), "n_newton": d.get("n_newton"),
            "n_cg": d.get("n_cg"), "source": "tests/golden/neo_hookean_128_seed0.json (make_neo_hookean_128.py)"}


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle as it stands, on this host's cores."""
    if rank != 0:
        return
    from rve_inputs import neo_hookean_config

    counts = reference_counts()
    if counts is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle Newton/CG counts for the 128^3 workload "
                                                               "not generated (tests/golden)"}))
        return
    n_newton, n_cg = counts
    phase, params, Fbar = neo_hookean_config(N_GRID, 0)
    vals = []
    for step in range(args.warmup + args.steps):
        t_cg, t_newton, it = oracle_sample(phase, params, Fbar, n_cg_iters=3)
        est = n_newton * t_newton + n_cg * t_cg
        if step >= args.warmup:
            vals.append(est)
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [N_GRID] * 3, "l2": l2_note([N_GRID] * 3)},
        "extrapolated": True,
        "cpu_baseline": {"value": v, "unit": "s", "cores": os.cpu_count(), "kind": "oracle", "extrapolated": True,
                         "sample": f"extrapolated from a sample: per step one Newton iteration at 128^3 with 3 CG "
                                   f"products, times the oracle's own counts ({n_newton} Newton, {n_cg} CG) of this "
                                   f"workload",
                         "full_solve_recorded": oracle_full_solve_record()},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def _events_ms(torch, fn, reps, stream):
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def cufft_projection_fns(torch, shape, device):
    """The projection G(tau) and the bare FFT pair with cuFFT (torch.fft) and torch elementwise Ghat, for comparison.

    Ghat is applied as v_i = (sum_j A_ij xi_j) / |xi|^2, out_ij = v_i xi_j, with the Nyquist wave number
    of every even axis set to 0 as in the library. Nothing is gathered or expanded inside the timed calls.
    """
    nx, ny, nz = shape

    def freq(n):
        k = torch.fft.fftfreq(n, d=1.0 / n, device=device, dtype=torch.float64)
        if n % 2 == 0:
            k[n // 2] = 0.0
        return k

    kz = torch.fft.rfftfreq(nz, d=1.0 / nz, device=device, dtype=torch.float64)
    if nz % 2 == 0:
        kz[-1] = 0.0
    xi = torch.meshgrid(freq(nx), freq(ny), kz, indexing="ij")
    xi2 = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
    inv = torch.where(xi2 > 0, 1.0 / torch.where(xi2 > 0, xi2, torch.ones_like(xi2)), torch.zeros_like(xi2))

    def project(tau):
        A = torch.fft.rfftn(tau, dim=(1, 2, 3)).reshape(3, 3, *xi2.shape)
        v = (A[:, 0] * xi[0] + A[:, 1] * xi[1] + A[:, 2] * xi[2]) * inv
        out = torch.stack([v * xi[j] for j in range(3)], dim=1).reshape(9, *xi2.shape)
        return torch.fft.irfftn(out, s=shape, dim=(1, 2, 3))

    def fft_pair(tau):
        return torch.fft.irfftn(torch.fft.rfftn(tau, dim=(1, 2, 3)), s=shape, dim=(1, 2, 3))

    return project, fft_pair


def run_matvec_comparison(ctx, fh, torch, mat, F, shape, dev, stream, reps=5):
    """Our five-pass projection and fused matrix-vector product against cuFFT (torch.fft) doing the same.

    Both sides get the same resident inputs. The cuFFT matrix-vector product applies K : p from a dense
    9x9 tangent per voxel expanded once outside the timed calls (torch.einsum), then the cuFFT projection.
    """
    K = torch.empty((45,) + shape, dtype=torch.float64, device=dev)
    ctx.fh_constitutive(mat, F, None, K, want_pbar=False)
    p = torch.randn((9,) + shape, dtype=torch.float64, device=dev)
    y = torch.empty_like(p)
    out = {}
    out["matvec_ms_ours"] = _events_ms(torch, lambda: ctx.fh_matvec(p, y, K=K), reps, stream)
    out["projection_ms_ours"] = _events_ms(torch, lambda: ctx.fh_project(p, y), reps, stream)
    project, fft_pair = cufft_projection_fns(torch, shape, dev)
    out["projection_ms_cufft_torch"] = _events_ms(torch, lambda: project(p), reps, stream)
    out["fft_pair_ms_cufft"] = _events_ms(torch, lambda: fft_pair(p), reps, stream)
    idx = torch.tensor([[min(a, b) * 9 - min(a, b) * (min(a, b) - 1) // 2 + abs(a - b) for b in range(9)]
                        for a in range(9)], device=dev)
    Kd = K[idx.reshape(-1)].reshape(9, 9, -1)
    del K
    pf = p.reshape(9, -1)
    out["matvec_ms_cufft_torch"] = _events_ms(
        torch, lambda: project(torch.einsum("abn,bn->an", Kd, pf).reshape((9,) + shape)), reps, stream)
    out["note"] = ("same inputs on both sides; cuFFT side: cufft R2C/C2R via torch.fft, Ghat as torch elementwise "
                   "ops, K:p as einsum over a dense 9x9 tangent expanded outside the timed calls")
    del Kd, p, y, pf
    torch.cuda.empty_cache()
    return out


def run_small_strain_16(fh, torch, stream, reps=20):
    """The 16^3 linear-elastic sphere cell (tol 1e-10): GPU time-to-solve beside the oracle's full solve."""
    from oracle import solver as osolver
    from rve_inputs import small_strain_config

    phase, params, Ebar = small_strain_config(16)
    with fh.Context(16, 16, 16, stream=stream.cuda_stream) as c16:
        mat = fh.Material(fh.LINEAR_ELASTIC, phase, params)
        F = torch.zeros((9, 16, 16, 16), dtype=torch.float64, device="cuda")
        opts = fh.default_options(newton_tol=1e-10)
        res = {}

        def solve():
            res["r"] = c16.fft_homog_solve(mat, Ebar, F, n_increments=1, options=opts)

        gpu_ms = _events_ms(torch, solve, reps, stream)
        pbar, st, _ = res["r"]
    t0 = time.perf_counter()
    ref = osolver.solve(phase, params, 0, Ebar, n_increments=1, newton_tol=1e-10)
    cpu_s = time.perf_counter() - t0
    return {"workload": "linear elastic 16^3, centred sphere r=0.25L, contrast 10, eps_xy=0.01, Newton tol 1e-10",
            "gpu_ms": gpu_ms, "newton": st["n_newton"], "cg": st["n_cg"], "oracle_s": cpu_s,
            "oracle_newton": len(ref.newton_residuals), "oracle_cg": int(sum(ref.cg_iterations)),
            "sigma_xy_gpu_vs_oracle": [float(pbar[1]), float(ref.Pbar[1])]}


def run_e2e(args, world, ctx, fh, torch, phase, params, Fbar, F, opts, dev, stream):
    """The same solve through the public API with host buffers: the phase map
    goes host -> device and the converged field device -> host every step."""
    shape = phase.shape
    phase_host = torch.from_numpy(phase.copy()).pin_memory()
    F_host = torch.empty((9,) + shape, dtype=torch.float64).pin_memory()
    phase_dev = torch.empty(shape, dtype=torch.uint8, device=dev)
    barrier(world, dev.index)
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        phase_dev.copy_(phase_host, non_blocking=True)
        mat_e = fh.Material(fh.NEO_HOOKEAN, phase_dev, params)
        ctx.fft_homog_solve(mat_e, Fbar, F, n_increments=N_INC, options=opts)
        F_host.copy_(F, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    return max_over_ranks(world, e2.elapsed_time(e3) / 1e3, dev) / args.steps


def run_batch(args, world, rank, local):
    """Batched solve of uneven linear-elastic cells with log-normal moduli.

    N cells with grids drawn from {32, 48, 64, 96}^3, eps_xx = 0.01, Newton
    tolerance 1e-8: the batched solve (one launch per pass and grid group, CG
    chunks as CUDA graphs) against solving the same cells one after another
    with the single-cell solver. Reports the mean and variance of Cbar_1111 =
    Pbar_xx / eps_xx over the cells.
    """
    import torch

    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    import paper_2408_03804_gb300 as fh
    from paper_2408_03804_gb300 import build as fhbuild
    from rve_inputs import batch_config

    fhbuild.build()
    fh.load()
    t_in = time.perf_counter()
    cells, params, Ebar = batch_config(args.batch, seed=rank)
    t_in = time.perf_counter() - t_in
    nvox = sum(int(c[0].size) for c in cells)
    stream = torch.cuda.Stream()
    opts = fh.default_options(newton_tol=NEWTON_TOL, check_every=8)
    with torch.cuda.stream(stream):
        b = fh.Batch(cells, stream=stream.cuda_stream)
        for _ in range(max(args.warmup, 1)):
            b.fft_homog_solve_batched(fh.LINEAR_ELASTIC, params, Ebar, options=opts)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            pbar, status, newton, cg, rc = b.fft_homog_solve_batched(fh.LINEAR_ELASTIC, params, Ebar, options=opts)
        e1.record(stream)
        torch.cuda.synchronize()
        t_batch = max_over_ranks(world, e0.elapsed_time(e1) / 1e3 / args.steps, torch.device("cuda", local))
        df = None
        if args.df64:
            # the same batch with double-float CG products (an option; the line's value stays FP64)
            opts_df = fh.default_options(newton_tol=NEWTON_TOL, check_every=8, matvec_arith=fh.ARITH_DF64)
            for _ in range(max(args.warmup, 1)):
                b.fft_homog_solve_batched(fh.LINEAR_ELASTIC, params, Ebar, options=opts_df)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                pb_df, st_df, nw_df, cg_df, rc_df = b.fft_homog_solve_batched(fh.LINEAR_ELASTIC, params, Ebar,
                                                                             options=opts_df)
            e1.record(stream)
            torch.cuda.synchronize()
            t_df = max_over_ranks(world, e0.elapsed_time(e1) / 1e3 / args.steps, torch.device("cuda", local))
            df = {"batched_df64_s": t_df, "speedup_vs_fp64_batched": t_batch / t_df, "rc": int(rc_df),
                  "newton_iterations": int(nw_df.sum()), "cg_iterations": int(cg_df.sum()),
                  "max_rel_diff_pbar_vs_fp64": float(np.abs(pb_df - pbar).max() / np.abs(pbar).max())}
        b.close()
        # the same cells one after another with the single-cell solver (one context per grid)
        ctxs = {}
        for ph, _ in cells:
            if ph.shape not in ctxs:
                ctxs[ph.shape] = fh.Context(*ph.shape, stream=stream.cuda_stream)
        mats = [fh.Material(fh.LINEAR_ELASTIC, ph, params, scale=sc) for ph, sc in cells]
        Fs = {shape: torch.zeros((9,) + shape, dtype=torch.float64, device="cuda") for shape in ctxs}
        torch.cuda.synchronize()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        seq_pbar = []
        for (ph, _), m in zip(cells, mats):
            pb, _, _ = ctxs[ph.shape].fft_homog_solve(m, Ebar, Fs[ph.shape], options=opts)
            seq_pbar.append(pb)
        e3.record(stream)
        torch.cuda.synchronize()
        t_seq = max_over_ranks(world, e2.elapsed_time(e3) / 1e3, torch.device("cuda", local))
        for c in ctxs.values():
            c.close()
    if rank != 0:
        return
    c1111 = pbar[:, 0] / Ebar[0]
    diff = float(np.abs(pbar - np.asarray(seq_pbar)).max() / np.abs(pbar).max())
    it_bytes = sum(cg_iteration_bytes(*c[0].shape) * int(k) for c, k in zip(cells, cg))
    # FP64 floor of the batch: counted FP64 lane operations of every cell's CG iterations and
    # right-hand-side projections at the measured DFMA issue rate
    fp64 = probe_fp64(fh, local)
    cg_cls = ("fwd_z", "fwd_y", "x_ghat", "inv_y", "inv_z", "cg_update")
    rhs_cls = ("fwd_z", "fwd_y", "x_ghat", "inv_y", "inv_z")
    ops = 0.0
    for (ph, _), k, nw in zip(cells, cg, newton):
        shp = ph.shape
        ops += int(k) * sum(fp64_ops(c, *shp) for c in cg_cls) + int(nw) * sum(fp64_ops(c, *shp) for c in rhs_cls)
    floor_s = ops / fp64["lane_ops_per_s"]
    line = {
        "metric": f"batched time-to-solve of {args.batch} uneven RVEs @1e-8 (linear elastic, log-normal E)",
        "value": t_batch, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 1),
        "higher_is_better": False, "scaling": "weak", "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.batch} cells, grids U{{32,48,64,96}}^3, log E = 0.3 g (GRF, corr 0.1 L), "
                               "nu 0.3, eps_xx 0.01, Newton tol 1e-8", "voxels": nvox,
                   "newton_iterations": int(newton.sum()), "cg_iterations": int(cg.sum()),
                   "input_generation_s": t_in},
        "sequential_single_cell_s": t_seq, "speedup_vs_sequential": t_seq / t_batch,
        "cbar1111_mean": float(c1111.mean()), "cbar1111_var": float(c1111.var(ddof=1)),
        "max_rel_diff_batched_vs_single": diff,
        "cg_bytes_gbs": it_bytes / t_batch / 1e9,
        "fp64_floor_s": floor_s, "fp64_floor_frac_batched": floor_s / t_batch,
        "fp64_floor_frac_sequential": floor_s / t_seq, "max_speedup_at_fp64_floor": t_seq / floor_s,
        "fp64_lane_ops": ops, "fp64_probe_lane_ops_per_s": fp64["lane_ops_per_s"],
    }
    if df is not None:
        line["df64_option"] = df
    print(json.dumps(line), flush=True)


def run_warm_start(args, world, rank, local):
    """Learned warm start against the zero initial guess on held-out cells.

    Each step is one held-out neo-Hookean cell (the training distribution of
    the network: random spheres of radius U[4, 10]/128 of the box at a volume
    fraction U[0.1, 0.4], matrix (lambda, mu) = (1.5, 1), inclusions 10x,
    |Fbar - I| <= 0.05, one load increment, Newton tolerance 1e-8) solved from
    Fbar and from the network's prediction; both times are CUDA-event times on
    the solver's stream, the warm-started one including the network's forward
    pass and the projection. Also times one training step (batch 8 at 64^3:
    forward, loss gradient, Adam) of the network's own kernels.
    """
    import torch

    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    import paper_2408_03804_gb300 as fh
    from paper_2408_03804_gb300 import build as fhbuild
    from paper_2408_03804_gb300 import warm_start as ws

    fhbuild.build()
    fh.load()
    n = args.shape[0]
    shape = (n, n, n)
    theta = np.load(WARM_WEIGHTS).astype(np.float32)
    n_cells = args.warmup + args.steps
    seeds = [2_000_000 + 1000 * rank + i for i in range(n_cells)]
    t_in = time.perf_counter()
    cells = [(ph, fb) for _, ph, fb in ws.cells(n, seeds, max(1, min(16, (os.cpu_count() or 2) - 1)))]
    t_in = time.perf_counter() - t_in
    stream = torch.cuda.Stream()
    rows = []
    with torch.cuda.stream(stream), fh.Context(*shape, stream=stream.cuda_stream) as ctx, \
            fh.Fno(*shape, max_batch=1, stream=stream.cuda_stream) as net:
        net.set_params(torch.as_tensor(theta).cuda())
        F = torch.empty((9,) + shape, dtype=torch.float64, device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with ClockSampler(local) as clk:
            for i, (ph, fb) in enumerate(cells):
                phd = torch.as_tensor(ph).cuda()
                torch.cuda.synchronize()
                ev[0].record(stream)
                F.zero_()
                st0, rc0 = ws.solve_cell(ctx, phd, fb, F)
                ev[1].record(stream)
                ref = F.clone()
                ev[2].record(stream)
                net.warm_start(ctx, phd, fb, F)
                st1, rc1 = ws.solve_cell(ctx, phd, fb, F, init_given=True)
                ev[3].record(stream)
                torch.cuda.synchronize()
                if i >= args.warmup:
                    rows.append({"t0": ev[0].elapsed_time(ev[1]) / 1e3, "t1": ev[2].elapsed_time(ev[3]) / 1e3,
                                 "n0": st0["n_newton"], "n1": st1["n_newton"], "c0": st0["n_cg"], "c1": st1["n_cg"],
                                 "rc": (rc0, rc1), "diff": float((F - ref).abs().max())})
        # one training step of the network's kernels (batch 8 at 64^3, synthetic cells and targets)
        m = 64
        with fh.Fno(m, m, m, max_batch=8, train=True, stream=stream.cuda_stream) as tnet:
            th = torch.as_tensor(theta).cuda()
            mom = torch.zeros_like(th)
            var = torch.zeros_like(th)
            g = torch.empty_like(th)
            gen = torch.Generator(device="cuda").manual_seed(rank)
            ph8 = [(torch.rand((m, m, m), generator=gen, device="cuda") < 0.25).to(torch.uint8) for _ in range(8)]
            tg8 = [0.1 * torch.randn((9, m, m, m), generator=gen, device="cuda") for _ in range(8)]
            fb8 = np.tile(np.eye(3).reshape(1, 9), (8, 1)) + 0.03 * np.random.default_rng(rank).normal(size=(8, 9))
            times = []
            for t in range(1, 6):
                torch.cuda.synchronize()
                ev[0].record(stream)
                tnet.set_params(th)
                tnet.forward(ph8, fb8)
                tnet.loss_grad(tg8, g)
                tnet.adam(th, g, mom, var, t, 1e-4)
                ev[1].record(stream)
                torch.cuda.synchronize()
                times.append(ev[0].elapsed_time(ev[1]))
            train_ms = statistics.median(times[2:])
    t0 = max_over_ranks(world, float(np.mean([r["t0"] for r in rows])), torch.device("cuda", local))
    t1 = max_over_ranks(world, float(np.mean([r["t1"] for r in rows])), torch.device("cuda", local))
    if rank != 0:
        return
    line = {
        "metric": f"time-to-solve @1e-8 of held-out {n}^3 neo-Hookean cells, learned warm start vs zero guess",
        "value": t1, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": False, "scaling": "weak", "dtype": "f64 solve, bf16/f32 network", "data": "synthetic",
        "config": {"workload": f"{n}^3 random spheres r U[4,10]/128 L, f U[0.1,0.4], inclusions 10x, "
                               "|Fbar - I| <= 0.05, 1 increment, Newton tol 1e-8; network trained at 64^3",
                   "weights": os.path.relpath(WARM_WEIGHTS, ROOT), "input_generation_s": t_in},
        "zero_guess_s": t0, "time_saved_frac": 1.0 - t1 / t0,
        "newton": [float(np.mean([r["n0"] for r in rows])), float(np.mean([r["n1"] for r in rows]))],
        "cg": [float(np.mean([r["c0"] for r in rows])), float(np.mean([r["c1"] for r in rows]))],
        "all_converged": all(r["rc"] == (0, 0) for r in rows),
        "max_field_diff_vs_zero_guess": max(r["diff"] for r in rows),
        "train_step_ms_batch8_64": train_ms,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_examples(args, world, rank, local):
    """The paper's 2D examples on this library, as cells one voxel thick (nz = 1: exact plane strain).

    svk_square   Section 4.1.1: St. Venant-Kirchhoff, stiff square L/3 at a corner, Fbar = I + 0.1 e_x e_y,
                 one increment, Newton tolerance 1e-5, CG tolerance 1e-8; 299 x 299 as in the paper.
    svk_scaling  the same cell on the paper's scaling grids 63^2, 127^2, 255^2, 511^2 (Section 4.1.3).
    j2_biaxial   Section 4.1.2: J2 plasticity, hard disks, biaxial strain 0.01, 10 increments, Newton
                 tolerance 1e-8; 199 x 199 as in the paper.
    eshelby      Section 4.2.1: homogenized tangent of the 0.7 % disk, (lambda, mu) = (2, 1) / (10, 5);
                 199 x 199 as in the paper.
    Each is timed with CUDA events over K repetitions after W warm-up runs; the paper's times (one
    4-core CPU, JAX) are quoted as context only.
    """
    import torch

    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    import paper_2408_03804_gb300 as fh
    from paper_2408_03804_gb300 import build as fhbuild
    from rve_inputs import centered_disk, j2_config, svk_square_config

    fhbuild.build()
    fh.load()
    stream = torch.cuda.Stream()
    out = {}

    def timed(fn):
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = None
        for _ in range(args.steps):
            res = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / args.steps, res

    arith = fh.ARITH_DF64 if args.df64 else fh.ARITH_FP64

    def svk_solve(n):
        phase, params, Fbar = svk_square_config(n, nz=1)
        with fh.Context(*phase.shape, stream=stream.cuda_stream) as ctx:
            mat = fh.Material(fh.SVK, phase, params)
            F = torch.empty((9,) + phase.shape, dtype=torch.float64, device="cuda")
            opts = fh.default_options(newton_tol=1e-5, cg_tol=1e-8, matvec_arith=arith)

            def svk():
                F.zero_()
                return ctx.fft_homog_solve(mat, Fbar, F, options=opts, allow=(fh.FH_ERR_NOT_CONVERGED,))

            t, (pb, st, rc) = timed(svk)
        return {"grid": [n, n, 1], "s": t, "rc": rc, "newton": st["n_newton"], "cg": st["n_cg"],
                "residuals": st["newton_residuals"], "Pbar_xy": float(pb[1])}

    def j2_solve():
        phase, params, plastic, Ebar = j2_config(199, 0, nz=1)
        with fh.Context(*phase.shape, stream=stream.cuda_stream) as ctx:
            hist = torch.zeros((10,) + phase.shape, dtype=torch.float64, device="cuda")
            mat = fh.Material(fh.J2, phase, params, plastic=plastic, history=hist)
            F = torch.empty((9,) + phase.shape, dtype=torch.float64, device="cuda")
            opts = fh.default_options(newton_tol=1e-8, matvec_arith=arith)

            def j2():
                F.zero_()
                hist.zero_()
                return ctx.fft_homog_solve(mat, Ebar, F, n_increments=10, options=opts,
                                           allow=(fh.FH_ERR_NOT_CONVERGED,))

            t, (pb, st, rc) = timed(j2)
        return {"grid": [199, 199, 1], "s": t, "rc": rc, "newton": st["n_newton"], "cg": st["n_cg"],
                "sigma_xx_yy": [float(pb[0]), float(pb[4])], "paper_s": 0.25, "paper_grid": "199^2"}

    def eshelby_tangent():
        phase, f = centered_disk(199, 0.007, nz=1)
        params = np.array([[2.0, 1.0], [10.0, 5.0]])
        with fh.Context(*phase.shape, stream=stream.cuda_stream) as ctx:
            mat = fh.Material(fh.LINEAR_ELASTIC, phase, params)
            zero = torch.zeros((9,) + phase.shape, dtype=torch.float64, device="cuda")
            t, C = timed(lambda: ctx.fft_homog_tangent(mat, zero, fh.default_options(matvec_arith=arith)))
        return {"grid": [199, 199, 1], "s": t, "fraction": f,
                "Cxxxx_Cyyyy_Cxyxy": [float(C[0, 0]), float(C[4, 4]), float(C[1, 1])],
                "paper_s": 4.0, "paper_grid": "199^2", "paper_table1": [4.035, 4.035, 1.010]}

    def wanted(name):
        return args.only is None or name in args.only

    with torch.cuda.stream(stream), ClockSampler(local) as clk:
        if wanted("svk_square"):
            out["svk_square"] = dict(svk_solve(299), paper_s=19.5, paper_grid="299^2")
        if wanted("svk_scaling"):
            out["svk_scaling"] = [svk_solve(n) for n in (63, 127, 255, 511)]
        if wanted("j2_biaxial"):
            out["j2_biaxial"] = j2_solve()
        if wanted("eshelby"):
            out["eshelby"] = eshelby_tangent()
    if rank != 0:
        return
    line = {"metric": "time of the paper's 2D examples (Sections 4.1.1, 4.1.2, 4.2.1) on one GPU",
            "matvec_arith": "df64 (an option; the method as stated is fp64)" if args.df64 else "fp64",
            "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 1),
            "higher_is_better": False, "dtype": "f64", "data": "synthetic", "examples": out,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_df64(args, world, rank, local):
    """The double-float option of the CG matrix-vector product (FH_ARITH_DF64) on the 128^3 bench cell:
    time-to-solve with each arithmetic (CUDA events, W warm-up and K timed solves each, alternating), the
    per-kernel split of one profiled solve each, and how far the two solutions are apart (Pbar relative,
    fluctuation field max-relative). Not the bench line: the method as stated is FP64 throughout."""
    import torch

    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    import paper_2408_03804_gb300 as fh
    from paper_2408_03804_gb300 import build as fhbuild
    from rve_inputs import neo_hookean_config

    fhbuild.build()
    fh.load()
    dev = torch.device("cuda", local)
    shape = tuple(args.shape)
    phase, params, Fbar = neo_hookean_config(shape, seed=rank)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    if args.probe_newton:
        # one Newton iteration with 16 double-float CG products (for ncu captures of those kernels)
        with fh.Context(*shape, stream=stream.cuda_stream) as ctx:
            F = torch.empty((9,) + shape, dtype=torch.float64, device=dev)
            probe = fh.default_options(newton_tol=NEWTON_TOL, max_newton=1, max_cg=16, matvec_arith=fh.ARITH_DF64)
            for _ in range(2):
                ctx.fft_homog_solve(fh.Material(fh.NEO_HOOKEAN, phase, params), Fbar, F, n_increments=N_INC,
                                    options=probe, allow=(fh.FH_ERR_NOT_CONVERGED,))
            torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"probe_newton_df64": "ok", "shape": list(shape)}), flush=True)
        return
    with fh.Context(*shape, stream=stream.cuda_stream) as ctx, ClockSampler(local) as clk:
        mat = fh.Material(fh.NEO_HOOKEAN, phase, params)
        F = {a: torch.empty((9,) + shape, dtype=torch.float64, device=dev) for a in (fh.ARITH_FP64, fh.ARITH_DF64)}
        opts = {a: fh.default_options(newton_tol=NEWTON_TOL, matvec_arith=a) for a in F}
        for _ in range(max(args.warmup, 1)):
            for a in F:
                ctx.fft_homog_solve(mat, Fbar, F[a], n_increments=N_INC, options=opts[a])
        times = {a: [] for a in F}
        stats = {}
        for _ in range(args.steps):
            for a in F:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pbar, st, _ = ctx.fft_homog_solve(mat, Fbar, F[a], n_increments=N_INC, options=opts[a])
                e1.record(stream)
                torch.cuda.synchronize()
                times[a].append(e0.elapsed_time(e1) / 1e3)
                stats[a] = (pbar, st)
        prof = {}
        for a in F:
            ctx.fh_profile_enable(True)
            ctx.fft_homog_solve(mat, Fbar, F[a], n_increments=N_INC, options=opts[a])
            prof[a] = ctx.fh_profile_read()
            ctx.fh_profile_enable(False)
        fl = {a: F[a].cpu().numpy() - Fbar.reshape(9, 1, 1, 1) for a in F}
    if rank != 0:
        return
    p64, pdf = stats[fh.ARITH_FP64][0], stats[fh.ARITH_DF64][0]
    d = np.abs(fl[fh.ARITH_DF64] - fl[fh.ARITH_FP64]).max(axis=(1, 2, 3)) / np.maximum(
        np.abs(fl[fh.ARITH_FP64]).max(axis=(1, 2, 3)), 1e-300)
    names = {fh.ARITH_FP64: "fp64", fh.ARITH_DF64: "df64"}
    out = {}
    for a in F:
        cls = {c: v for c, v in prof[a].items() if v[0] and c != "idle"}
        cg_its = cls["fwd_z"][0] - stats[a][1]["n_newton"]
        it_ms = sum(cls[c][1] / cls[c][0] for c in ("fwd_z", "fwd_y", "x_ghat", "inv_y", "inv_z", "cg_update"))
        out[names[a]] = {"s": statistics.median(times[a]), "runs_s": times[a], "newton": stats[a][1]["n_newton"],
                         "cg": stats[a][1]["n_cg"], "ms_per_cg_iteration": it_ms,
                         "kernels_ms_per_launch": {c: v[1] / v[0] for c, v in cls.items()},
                         "profiled_cg_products": cg_its}
    line = {"metric": "128^3 neo-Hookean time-to-solve with the CG transforms in double-float (FH_ARITH_DF64) "
                      "beside FP64", "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 1), "higher_is_better": False, "data": "synthetic",
            "config": {"workload": f"{shape[0]}x{shape[1]}x{shape[2]} neo-Hookean RSA spheres (seed 0), 5 "
                                   "increments to shear 0.05, Newton tol 1e-8"},
            "arith": out, "speedup": out["fp64"]["s"] / out["df64"]["s"],
            "pbar_rel_diff": float(np.abs(pdf - p64).max() / np.abs(p64).max()),
            "fluctuation_maxrel_diff": float(d.max()), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_differentiation(args, world, rank, local):
    """Config 4: the 64^3 SIMP cell (rho in [0.01, 1], E = rho^3, nu = 0.3). Each step computes the
    homogenized tangent (9 unit-response CG solves, fft_homog_tangent) and the sensitivity field
    dCbar_1212/drho of every voxel (one more unit response and the voxel contraction,
    fft_homog_sensitivity), CG tolerance 1e-10. CUDA-event times on the library's stream around steps
    without per-launch events; the CG iterations come from the library's launch counts, the per-kernel
    times from one more step with events around every launch. --df64 runs the CG products in
    double-float."""
    import torch

    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    import paper_2408_03804_gb300 as fh
    from paper_2408_03804_gb300 import build as fhbuild
    from rve_inputs import simp_config

    fhbuild.build()
    fh.load()
    n = 64
    phase, params, rho, scale, dscale = simp_config(n, seed=rank)
    stream = torch.cuda.Stream()
    opts = fh.default_options(cg_tol=1e-10, matvec_arith=fh.ARITH_DF64 if args.df64 else fh.ARITH_FP64)
    with torch.cuda.stream(stream), fh.Context(n, n, n, stream=stream.cuda_stream) as ctx, \
            ClockSampler(local) as clk:
        mat = fh.Material(fh.LINEAR_ELASTIC, phase, params, scale=scale)
        zero = torch.zeros((9, n, n, n), dtype=torch.float64, device="cuda")
        ds = torch.as_tensor(dscale).cuda()
        sens = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

        def step():
            ev[0].record(stream)
            C = ctx.fft_homog_tangent(mat, zero, options=opts)
            ev[1].record(stream)
            ctx.fft_homog_sensitivity(mat, (0, 1, 0, 1), ds, sens, options=opts)
            ev[2].record(stream)
            torch.cuda.synchronize()
            return C, ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3

        for _ in range(max(args.warmup, 1)):
            step()
        # timed steps without per-launch events (CG chunks as graph replays); launches still counted
        ctx.fh_profile_enable(False)
        tt, ts = [], []
        for _ in range(args.steps):
            C, a, b = step()
            tt.append(a)
            ts.append(b)
        counts = ctx.fh_profile_read()
        # one more step with events around every launch: the per-kernel split
        ctx.fh_profile_enable(True)
        step()
        prof = ctx.fh_profile_read()
        ctx.fh_profile_enable(False)
        s = sens.detach().cpu().numpy()
    t_tan = max_over_ranks(world, float(np.mean(tt)), torch.device("cuda", local))
    t_sen = max_over_ranks(world, float(np.mean(ts)), torch.device("cuda", local))
    if rank != 0:
        return
    voigt = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    Cv = [[float(C[3 * i + j, 3 * k + l]) for (k, l) in voigt] for (i, j) in voigt]
    cg_its = counts["fwd_z"][0] / args.steps
    line = {
        "metric": "homogenized 6x6 tangent and per-voxel dCbar_1212/drho of the 64^3 SIMP cell (config 4)",
        "matvec_arith": "df64 (an option; the method as stated is fp64)" if args.df64 else "fp64",
        "value": t_tan + t_sen, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 1),
        "higher_is_better": False, "scaling": "weak", "dtype": "f64", "data": "synthetic",
        "config": {"workload": "64^3 SIMP rho in [0.01,1] (Gaussian-smoothed noise, sigma 2 vox), E = rho^3, "
                               "nu 0.3, CG tol 1e-10"},
        "tangent_s": t_tan, "sensitivity_s": t_sen, "cg_iterations_per_step": cg_its,
        "ms_per_cg_iteration": 1e3 * (t_tan + t_sen) / max(cg_its, 1),
        "cbar_voigt_diag": [Cv[i][i] for i in range(6)],
        "euler_check_sum_rho_s_over_3_vs_C1212": [float((s * rho / 3.0).sum()), float(C[1, 1])],
        "kernels_one_profiled_step": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items() if v[0]},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch

    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    import paper_2408_03804_gb300 as fh
    from paper_2408_03804_gb300 import build as fhbuild
    from rve_inputs import neo_hookean_config

    if rank == 0:
        fhbuild.build()
    barrier(world, local)
    fhbuild.build()
    fh.load()
    dev = torch.device("cuda", local)
    shape = tuple(args.shape)
    phase, params, Fbar = neo_hookean_config(shape, seed=rank)
    n = phase.size
    # a stream of our own, current for every torch op below: the library replays
    # its CG chunks as CUDA graphs, which the legacy default stream cannot capture
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    ctx = fh.Context(*shape, stream=stream.cuda_stream)
    mat = fh.Material(fh.NEO_HOOKEAN, phase, params)
    F = torch.empty((9,) + shape, dtype=torch.float64, device=dev)
    opts = fh.default_options(newton_tol=NEWTON_TOL)

    def step():
        return ctx.fft_homog_solve(mat, Fbar, F, n_increments=N_INC, options=opts)

    if args.probe_newton:
        # one Newton iteration of the first increment with 16 CG products: every
        # kernel of the solve in its bench launch configuration, few launches
        probe = fh.default_options(newton_tol=NEWTON_TOL, max_newton=1, max_cg=16)
        for _ in range(2):
            ctx.fft_homog_solve(mat, Fbar, F, n_increments=N_INC, options=probe,
                                allow=(fh.FH_ERR_NOT_CONVERGED,))
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"probe_newton": "ok", "shape": list(shape)}), flush=True)
        ctx.close()
        return

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs; launches counted, not timed one by one ----
    ctx.fh_profile_enable(False)
    barrier(world, local)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    with ClockSampler(local) as clk:
        e0.record(stream)
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            pbar, st, _ = step()
            stats.append(st)
        e1.record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    barrier(world, local)
    counts_timed = ctx.fh_profile_read()
    elapsed_s = e0.elapsed_time(e1) / 1e3
    elapsed_s = max_over_ranks(world, elapsed_s, dev)
    per_step = elapsed_s / args.steps

    # ---- end to end through the public API with host buffers ----
    e2e_s = None
    if not args.no_e2e:
        e2e_s = run_e2e(args, world, ctx, fh, torch, phase, params, Fbar, F, opts, dev, stream)

    # ---- one more solve with CUDA events around every launch: the per-kernel split ----
    ctx.fh_profile_enable(True)
    step()
    prof = ctx.fh_profile_read()
    ctx.fh_profile_enable(False)

    # ---- measured FP64 issue rate (the roofline of the FP64-bound passes) ----
    fp64 = probe_fp64(fh, local)

    # ---- cuFFT comparison and the 16^3 linear-elastic solve ----
    cmp = None
    if not args.no_cufft:
        cmp = run_matvec_comparison(ctx, fh, torch, mat, F, shape, dev, stream)
    small = None
    if rank == 0 and not args.no_cpu_baseline:
        small = run_small_strain_16(fh, torch, stream)
    if rank != 0:
        ctx.close()
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (from the profiled solve; launches that did work only) ----
    hbm_peak, hbm_src = peaks()
    classes = {c: v for c, v in prof.items() if v[0] > 0 and c != "idle"}
    dom = max(classes, key=lambda c: classes[c][1])
    launches_dom, ms_dom = classes[dom]
    avg_s = ms_dom / 1e3 / launches_dom
    bytes_l, flops_l = algorithmic_work(dom, *shape)
    fp64_ach = flops_l / avg_s / 1e12 if flops_l else None
    peak_tf = fp64["tflops"]
    roofline = {"bound": "alu", "kernel": dom, "achieved": fp64_ach, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": fp64_ach / peak_tf if fp64_ach else None,
                "traffic": committed_traffic(dom),
                "peak_source": fp64["source"] + " (x 2 flops per FMA), of measured",
                "achieved_counts": "algorithmic flops of one launch (5 L log2 L per complex length-L FFT, 2 per "
                                   "pointwise FMA) / its average CUDA-event duration in a profiled solve, launches "
                                   "that did work only",
                "avg_launch_ms": avg_s * 1e3, "launches": launches_dom,
                "algorithmic_flops_per_launch": flops_l, "algorithmic_bytes_per_launch": bytes_l,
                "hbm_gbs": bytes_l / avg_s / 1e9, "hbm_peak": hbm_peak, "hbm_peak_source": hbm_src,
                "hbm_frac": bytes_l / avg_s / 1e9 / hbm_peak,
                "fp64_pipe_frac": fp64_pipe_frac(dom, shape, avg_s, fp64["lane_ops_per_s"]),
                "fp64_probe": fp64}
    # CG iteration (matrix-vector product + vector update) effective bandwidth
    cg_cls = ("fwd_z", "fwd_y", "x_ghat", "inv_y", "inv_z", "cg_update", "cg_scalar")
    it_ms = sum(classes[c][1] / classes[c][0] for c in cg_cls[:6] if c in classes)
    it_bytes = cg_iteration_bytes(*shape)
    cg_iter = {"ms": it_ms, "algorithmic_bytes": it_bytes, "gbs": it_bytes / (it_ms / 1e3) / 1e9,
               "hbm_frac": it_bytes / (it_ms / 1e3) / 1e9 / hbm_peak,
               "fp64_ops": sum(fp64_ops(c, *shape) for c in cg_cls[:6]),
               "fp64_pipe_frac": sum(fp64_ops(c, *shape) for c in cg_cls[:6]) / (it_ms / 1e3) / fp64["lane_ops_per_s"],
               "note": "per-launch means of the six CG-iteration kernels in the profiled solve (launches that did "
                       "work only); algorithmic bytes as in the scope table's per-voxel count",
               "comparison": cmp}
    tot = sum(x[1] for x in prof.values())
    kernels = {c: {"launches": v[0], "ms_total": v[1], "share": v[1] / tot} for c, v in prof.items() if v[0]}

    # ---- CPU oracle on a bounded sample (rank 0 only, at N = 1) ----
    cpu = None
    if world == 1 and not args.no_cpu_baseline and shape == (N_GRID,) * 3:
        t_cg, t_newton, it = oracle_sample(phase, params, Fbar, n_cg_iters=6)
        st = stats[-1]
        est = st["n_newton"] * t_newton + st["n_cg"] * t_cg
        cpu = {"value": est, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
               "extrapolated": True,
               "sample": f"extrapolated from a sample: one Newton iteration at 128^3 with {it} CG products on the "
                         f"host ({t_newton:.2f} s Newton overhead, {t_cg:.3f} s per CG iteration), times this run's "
                         f"counts ({st['n_newton']} Newton, {st['n_cg']} CG)",
               "full_solve_recorded": oracle_full_solve_record()}

    st = stats[-1]
    line = {
        "metric": METRIC, "value": per_step, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if shape == (N_GRID,) * 3 else WORKLOAD.replace("128^3", "x".join(map(str, shape))),
                   "grid": list(shape), "l2": l2_note(shape)},
        "replicas": world,
        "timing": "CUDA events around the K solves, no per-launch events inside the timed region",
        "result": {"newton_iterations": st["n_newton"], "cg_iterations": st["n_cg"], "pbar": pbar.tolist()},
        "e2e": ({"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(n), "d2h_bytes_per_step": int(9 * n * 8)}
                if e2e_s is not None else None),
        "gpu_launches": int(sum(v[0] for v in counts_timed.values())),
        "gpu_launches_idle": int(counts_timed["idle"][0]),
        "roofline": roofline,
        "cg_iteration": cg_iter,
        "kernels": kernels,
        "small_strain_16": small,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "wall_s_timed": t_wall,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch", type=int, default=0,
                    help="solve this many uneven linear-elastic cells batched and one by one (not the bench line)")
    ap.add_argument("--probe-newton", action="store_true",
                    help="run one Newton iteration with 16 CG products (for ncu launch lists) and exit")
    ap.add_argument("--no-cufft", action="store_true")
    ap.add_argument("--differentiation", action="store_true",
                    help="config 4: SIMP 64^3 tangent and sensitivities (not the bench line)")
    ap.add_argument("--examples", action="store_true",
                    help="time the paper's 2D examples (SVK square, J2 disks, Eshelby tangent); not the bench line")
    ap.add_argument("--df64", action="store_true",
                    help="the 128^3 solve with double-float CG transforms beside FP64 (an option; not the bench "
                         "line); with --batch, the batch also with double-float CG products")
    ap.add_argument("--only", nargs="+", default=None,
                    choices=("svk_square", "svk_scaling", "j2_biaxial", "eshelby"),
                    help="with --examples: run only these examples (for launch lists)")
    ap.add_argument("--warm-start", action="store_true",
                    help="learned warm start vs zero guess on held-out cells of --shape (not the bench line)")
    ap.add_argument("--shape", type=int, nargs=3, default=[N_GRID] * 3,
                    help="grid of the solve (smaller cases are for profiling, not bench lines)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.batch:
        run_batch(args, world, rank, local)
        return
    if args.warm_start:
        run_warm_start(args, world, rank, local)
        return
    if args.examples:
        run_examples(args, world, rank, local)
        return
    if args.differentiation:
        run_differentiation(args, world, rank, local)
        return
    if args.df64:
        run_df64(args, world, rank, local)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
