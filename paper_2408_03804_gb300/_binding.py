"""ctypes binding of libfft_homog.so (argument marshalling only).

Every computation runs in the CUDA library; this module only converts torch
tensors to device pointers, host arrays to C arrays and return codes to
exceptions. It fails loudly when the library has not been built: there is no
CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_void_p

import numpy as np

from . import build as _build

FH_OK = 0
FH_ERR_ARG = 1
FH_ERR_CUDA = 2
FH_ERR_NOT_CONVERGED = 3
FH_ERR_NONPHYSICAL = 4
FH_ERR_TIMEOUT = 5
FH_ERR_UNSUPPORTED = 6

LINEAR_ELASTIC = 0
NEO_HOOKEAN = 1
SVK = 2
J2 = 3

TANGENT_STORED = 0
TANGENT_JVP = 1

INIT_REFERENCE = 0
INIT_GIVEN = 1

LAUNCH_GRAPH = 0
LAUNCH_PLAIN = 1

ARITH_FP64 = 0
ARITH_DF64 = 1

_ERR_NAMES = {1: "FH_ERR_ARG", 2: "FH_ERR_CUDA", 3: "FH_ERR_NOT_CONVERGED", 4: "FH_ERR_NONPHYSICAL",
              5: "FH_ERR_TIMEOUT", 6: "FH_ERR_UNSUPPORTED"}

# every symbol include/fft_homog.h declares
EXPORTS = ["fh_default_options", "fh_create", "fh_destroy", "fh_last_error_string", "fh_constitutive",
           "fh_project", "fh_matvec", "fft_homog_solve", "fh_profile_enable", "fh_profile_read", "fh_project_static", "fft_homog_tangent", "fft_homog_sensitivity", "fft_homog_stress_sensitivity",
           "fh_batch_create", "fh_batch_destroy", "fft_homog_solve_batched", "fh_autotune", "fh_probe_fp64", "fh_df64_roundtrip", "fh_twiddle_tables",
           "fh_fno_param_count", "fh_fno_create", "fh_fno_destroy", "fh_fno_set_params", "fh_fno_forward",
           "fh_fno_loss_grad", "fh_fno_adam", "fh_fno_make_target", "fh_fno_warm_start", "fh_fno_test_skip_mma"]

PROF_NCLASS = 14
PROF_CLASSES = ["fwd_z", "fwd_y", "x_ghat", "inv_y", "inv_z", "constitutive", "jvp", "cg_scalar", "cg_update",
                "newton_update", "fill", "reduce", "contract", "idle"]


class FhError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {message}")
        self.code = code


class FhMaterial(ctypes.Structure):
    _fields_ = [("kind", c_int), ("n_phase", c_int), ("phase", c_void_p), ("params", POINTER(c_double)),
                ("scale", c_void_p), ("plastic", POINTER(c_double)), ("history", c_void_p)]


class FhOptions(ctypes.Structure):
    _fields_ = [("newton_tol", c_double), ("cg_tol", c_double), ("max_newton", c_int), ("max_cg", c_int),
                ("init", c_int), ("tangent_mode", c_int), ("check_every", c_int), ("launch_mode", c_int),
                ("lengths", c_double * 3), ("matvec_arith", c_int), ("reserved", c_int)]


class FhCell(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("phase", c_void_p), ("scale", c_void_p),
                ("F", c_void_p)]


class FhStats(ctypes.Structure):
    _fields_ = [("n_newton", c_int), ("n_cg", c_int), ("capacity", c_int), ("n_recorded", c_int),
                ("newton_residuals", POINTER(c_double)), ("cg_iterations", POINTER(c_int)),
                ("time_ms", c_double), ("cg_graph_replays", c_int), ("cg_graph_captures", c_int)]


_lib = None


def library_path() -> str:
    return _build.lib_path()


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the library (once). Raises if it is missing: build it first."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} is missing (run paper_2408_03804_gb300.build)")
    lib = ctypes.CDLL(path)
    lib.fh_default_options.argtypes = [POINTER(FhOptions)]
    lib.fh_default_options.restype = None
    lib.fh_create.argtypes = [POINTER(c_void_p), c_int, c_int, c_int, c_void_p]
    lib.fh_create.restype = c_int
    lib.fh_destroy.argtypes = [c_void_p]
    lib.fh_destroy.restype = None
    lib.fh_last_error_string.argtypes = []
    lib.fh_last_error_string.restype = ctypes.c_char_p
    lib.fh_constitutive.argtypes = [c_void_p, POINTER(FhMaterial), c_void_p, c_void_p, c_void_p, POINTER(c_double)]
    lib.fh_constitutive.restype = c_int
    lib.fh_project.argtypes = [c_void_p, c_void_p, c_void_p, c_double, POINTER(c_double)]
    lib.fh_project.restype = c_int
    lib.fh_matvec.argtypes = [c_void_p, POINTER(FhMaterial), c_void_p, c_void_p, c_void_p, c_void_p,
                              POINTER(c_double), c_int]
    lib.fh_matvec.restype = c_int
    lib.fft_homog_solve.argtypes = [c_void_p, POINTER(FhMaterial), POINTER(c_double), c_int, POINTER(FhOptions),
                                    c_void_p, POINTER(c_double), POINTER(FhStats)]
    lib.fft_homog_solve.restype = c_int
    lib.fh_profile_enable.argtypes = [c_void_p, c_int]
    lib.fh_profile_enable.restype = c_int
    lib.fh_profile_read.argtypes = [c_void_p, POINTER(ctypes.c_longlong), POINTER(c_double)]
    lib.fh_profile_read.restype = c_int
    lib.fh_project_static.argtypes = [c_void_p, c_void_p, c_int, c_int, c_int, c_double, POINTER(c_double),
                                      c_void_p]
    lib.fh_project_static.restype = c_int
    lib.fft_homog_tangent.argtypes = [c_void_p, POINTER(FhMaterial), c_void_p, POINTER(FhOptions),
                                      POINTER(c_double)]
    lib.fft_homog_tangent.restype = c_int
    lib.fft_homog_sensitivity.argtypes = [c_void_p, POINTER(FhMaterial), POINTER(FhOptions), c_int, c_int, c_int,
                                          c_int, c_void_p, c_void_p]
    lib.fft_homog_sensitivity.restype = c_int
    lib.fft_homog_stress_sensitivity.argtypes = [c_void_p, POINTER(FhMaterial), c_void_p, POINTER(FhOptions), c_int,
                                                 c_int, c_void_p, c_void_p]
    lib.fft_homog_stress_sensitivity.restype = c_int
    lib.fh_batch_create.argtypes = [POINTER(c_void_p), POINTER(FhCell), c_int, c_void_p]
    lib.fh_batch_create.restype = c_int
    lib.fh_batch_destroy.argtypes = [c_void_p]
    lib.fh_batch_destroy.restype = None
    lib.fft_homog_solve_batched.argtypes = [c_void_p, c_int, c_int, POINTER(c_double), POINTER(c_double), c_int,
                                            POINTER(FhOptions), POINTER(c_double), POINTER(c_int), POINTER(c_int),
                                            POINTER(c_int)]
    lib.fft_homog_solve_batched.restype = c_int
    lib.fh_autotune.argtypes = [c_void_p, c_int, POINTER(c_double), POINTER(c_int)]
    lib.fh_autotune.restype = c_int
    lib.fh_probe_fp64.argtypes = [c_int, c_int, ctypes.c_longlong, c_void_p, POINTER(c_double), POINTER(c_double)]
    lib.fh_probe_fp64.restype = c_int
    lib.fh_df64_roundtrip.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, ctypes.c_longlong, c_void_p]
    lib.fh_df64_roundtrip.restype = c_int
    lib.fh_twiddle_tables.argtypes = [POINTER(c_double), c_int]
    lib.fh_twiddle_tables.restype = c_int
    lib.fh_fno_param_count.argtypes = []
    lib.fh_fno_param_count.restype = ctypes.c_longlong
    lib.fh_fno_create.argtypes = [POINTER(c_void_p), c_int, c_int, c_int, c_int, c_int, c_void_p]
    lib.fh_fno_create.restype = c_int
    lib.fh_fno_destroy.argtypes = [c_void_p]
    lib.fh_fno_destroy.restype = None
    lib.fh_fno_set_params.argtypes = [c_void_p, c_void_p]
    lib.fh_fno_set_params.restype = c_int
    lib.fh_fno_forward.argtypes = [c_void_p, c_int, POINTER(c_void_p), POINTER(c_double), POINTER(c_void_p)]
    lib.fh_fno_forward.restype = c_int
    lib.fh_fno_loss_grad.argtypes = [c_void_p, POINTER(c_void_p), POINTER(c_double), c_void_p]
    lib.fh_fno_loss_grad.restype = c_int
    lib.fh_fno_adam.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float,
                                ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    lib.fh_fno_adam.restype = c_int
    lib.fh_fno_make_target.argtypes = [c_void_p, c_void_p, POINTER(c_double), c_void_p]
    lib.fh_fno_make_target.restype = c_int
    lib.fh_fno_warm_start.argtypes = [c_void_p, c_void_p, c_void_p, POINTER(c_double), c_void_p]
    lib.fh_fno_warm_start.restype = c_int
    lib.fh_fno_test_skip_mma.argtypes = [c_void_p, c_int]
    lib.fh_fno_test_skip_mma.restype = c_int
    _lib = lib
    return lib


def _check(rc: int, allow=()) -> int:
    if rc != FH_OK and rc not in allow:
        raise FhError(rc, load().fh_last_error_string().decode())
    return rc


def _ptr(t) -> int:
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _dvec(values, n=None):
    a = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(-1))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values")
    return a, a.ctypes.data_as(POINTER(c_double))


def default_options(**kw) -> FhOptions:
    o = FhOptions()
    load().fh_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "lengths":
            for i in range(3):
                o.lengths[i] = float(v[i])
        else:
            setattr(o, k, v)
    return o


def fh_project_static(A, out, scale: float = 1.0, lengths=None, stream=None):
    """out = scale * G(A) without any device allocation (no fh_ctx needed).

    For callers that may not allocate GPU memory; the grid must have at most
    32768 voxels. A and out are contiguous CUDA float64 tensors (9, nx, ny, nz).
    """
    import torch

    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    nx, ny, nz = A.shape[1:]
    La = _dvec(lengths, 3) if lengths is not None else (None, None)
    return _check(load().fh_project_static(_ptr(A), _ptr(out), nx, ny, nz, float(scale), La[1], c_void_p(stream)))


def fh_df64_roundtrip(x, hi=None, lo=None, out=None, stream=None):
    """The double-float split of a CUDA float64 tensor x as the FH_ARITH_DF64 kernels make it:
    (hi, lo) float32 tensors and hi + lo joined back to float64 (returned as (hi, lo, out))."""
    import torch

    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    hi = torch.empty(x.shape, dtype=torch.float32, device=x.device) if hi is None else hi
    lo = torch.empty(x.shape, dtype=torch.float32, device=x.device) if lo is None else lo
    out = torch.empty_like(x) if out is None else out
    _check(load().fh_df64_roundtrip(_ptr(x), _ptr(hi), _ptr(lo), _ptr(out), int(x.numel()), c_void_p(stream)))
    return hi, lo, out


def fh_twiddle_tables():
    """The library's twiddle tables (host only): a complex numpy array of 2 T entries, w_L^m as
    (cos, -sin) at offset(L) + m and its tangent form (rho, tau) at T + offset(L) + m."""
    lib = load()
    n = lib.fh_twiddle_tables(None, 0)
    buf = (c_double * (2 * n))()
    if lib.fh_twiddle_tables(buf, n) != n:
        raise FhError(FH_ERR_ARG, "fh_twiddle_tables: unexpected size")
    a = np.frombuffer(buf, dtype=np.float64).copy().reshape(n, 2)
    return a[:, 0] + 1j * a[:, 1]


def fh_probe_fp64(ctas_per_sm: int = 4, chains: int = 8, iters: int = 1 << 18, stream=None):
    """Measured FP64 FMA issue rate of the current device: (ms, lane operations) of one timed launch."""
    import torch

    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    ms, ops = c_double(), c_double()
    _check(load().fh_probe_fp64(int(ctas_per_sm), int(chains), int(iters), c_void_p(stream), ctypes.byref(ms),
                                ctypes.byref(ops)))
    return ms.value, ops.value


class Material:
    """A material description: kind, device phase map and host parameter table."""

    def __init__(self, kind: int, phase, params, scale=None, plastic=None, history=None):
        import torch

        self.kind = int(kind)
        if not isinstance(phase, torch.Tensor):
            phase = torch.as_tensor(np.ascontiguousarray(phase, dtype=np.uint8))
        self.phase = phase.to(device="cuda", dtype=torch.uint8).contiguous()
        self.params, _ = _dvec(params)
        if self.params.size % 2:
            raise ValueError("params must hold (lambda, mu) pairs")
        self.scale = None
        if scale is not None:
            if not isinstance(scale, torch.Tensor):
                scale = torch.as_tensor(np.ascontiguousarray(scale, dtype=np.float64))
            self.scale = scale.to(device="cuda", dtype=torch.float64).contiguous()
        self.plastic = None
        if plastic is not None:
            self.plastic, _ = _dvec(plastic)
        self.history = history  # CUDA float64 tensor (10, nx, ny, nz) for J2, updated in place by solves
        self._c = FhMaterial(self.kind, self.params.size // 2, self.phase.data_ptr(),
                             self.params.ctypes.data_as(POINTER(c_double)),
                             self.scale.data_ptr() if self.scale is not None else None,
                             self.plastic.ctypes.data_as(POINTER(c_double)) if self.plastic is not None else None,
                             _ptr(history) if history is not None else None)

    @property
    def c(self):
        return ctypes.byref(self._c)


class Context:
    """An fh_ctx bound to a grid and a CUDA stream (default: torch's current stream)."""

    def __init__(self, nx: int, ny: int, nz: int, stream=None):
        import torch

        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.shape = (nx, ny, nz)
        self.stream = stream
        h = c_void_p()
        _check(lib.fh_create(ctypes.byref(h), nx, ny, nz, c_void_p(stream)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().fh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- entry points (same names as the C-ABI) ----
    def fh_constitutive(self, mat: Material, F, P=None, K=None, want_pbar=True, allow_nonphysical=False):
        pbar = np.zeros(9)
        rc = load().fh_constitutive(self._h, mat.c, _ptr(F), _ptr(P), _ptr(K),
                                    pbar.ctypes.data_as(POINTER(c_double)) if want_pbar else None)
        _check(rc, allow=(FH_ERR_NONPHYSICAL,) if allow_nonphysical else ())
        return (pbar, rc) if allow_nonphysical else pbar

    def fh_project(self, A, out, scale: float = 1.0, lengths=None):
        La = _dvec(lengths, 3) if lengths is not None else (None, None)
        _check(load().fh_project(self._h, _ptr(A), _ptr(out), float(scale), La[1]))

    def fh_matvec(self, p, y, K=None, mat: Material | None = None, F=None, lengths=None, arith: int = ARITH_FP64):
        La = _dvec(lengths, 3) if lengths is not None else (None, None)
        _check(load().fh_matvec(self._h, mat.c if mat is not None else None, _ptr(F), _ptr(K), _ptr(p), _ptr(y),
                                La[1], int(arith)))

    def fh_autotune(self, reps: int = 3):
        """Time candidate tile shapes of the projection passes and keep the fastest.

        Returns (ms per projection, (z lines per CTA, y columns, x columns)).
        """
        ms = c_double()
        ch = (c_int * 3)()
        _check(load().fh_autotune(self._h, int(reps), ctypes.byref(ms), ch))
        return ms.value, tuple(ch)

    def fh_profile_enable(self, enable: bool = True):
        _check(load().fh_profile_enable(self._h, 1 if enable else 0))

    def fh_profile_read(self):
        """{class name: (launches, device ms)} since the last fh_profile_enable."""
        counts = (ctypes.c_longlong * PROF_NCLASS)()
        ms = (c_double * PROF_NCLASS)()
        _check(load().fh_profile_read(self._h, counts, ms))
        return {PROF_CLASSES[i]: (int(counts[i]), float(ms[i])) for i in range(PROF_NCLASS)}

    def fft_homog_tangent(self, mat: Material, F, options: FhOptions | None = None):
        """Homogenized tangent as a 9x9 array, C[ab, cd] = dPbar_ab / dFbar_cd."""
        C = np.zeros(81)
        _check(load().fft_homog_tangent(self._h, mat.c, _ptr(F),
                                        ctypes.byref(options) if options is not None else None,
                                        C.ctypes.data_as(POINTER(c_double))))
        return C.reshape(9, 9)

    def fft_homog_sensitivity(self, mat: Material, ijkl, dscale, out, options: FhOptions | None = None):
        """dCbar_ijkl / d rho per voxel into out (CUDA float64 tensor of the grid shape)."""
        i, j, k, l = (int(v) for v in ijkl)
        _check(load().fft_homog_sensitivity(self._h, mat.c, ctypes.byref(options) if options is not None else None,
                                            i, j, k, l, _ptr(dscale), _ptr(out)))

    def fft_homog_stress_sensitivity(self, mat: Material, F, ij, dscale, out, options: FhOptions | None = None):
        """dPbar_ij / d rho per voxel at the converged state F into out (CUDA float64 tensor of the grid shape)."""
        i, j = (int(v) for v in ij)
        _check(load().fft_homog_stress_sensitivity(self._h, mat.c, _ptr(F),
                                                   ctypes.byref(options) if options is not None else None, i, j,
                                                   _ptr(dscale), _ptr(out)))

    def fft_homog_solve(self, mat: Material, Fbar, F, n_increments: int = 1, options: FhOptions | None = None,
                        capacity: int = 512, allow=()):
        """Solve in place on F; returns (Pbar, stats dict, return code)."""
        fb, fbp = _dvec(Fbar, 9)
        pbar = np.zeros(9)
        res = np.zeros(capacity)
        cgi = np.zeros(capacity, dtype=np.int32)
        st = FhStats(0, 0, capacity, 0, res.ctypes.data_as(POINTER(c_double)),
                     cgi.ctypes.data_as(POINTER(c_int)), 0.0)
        rc = load().fft_homog_solve(self._h, mat.c, fbp, int(n_increments),
                                    ctypes.byref(options) if options is not None else None, _ptr(F),
                                    pbar.ctypes.data_as(POINTER(c_double)), ctypes.byref(st))
        _check(rc, allow=allow)
        stats = {"n_newton": st.n_newton, "n_cg": st.n_cg, "time_ms": st.time_ms,
                 "newton_residuals": res[:st.n_recorded].tolist(), "cg_iterations": cgi[:st.n_recorded].tolist(),
                 "cg_graph_replays": st.cg_graph_replays, "cg_graph_captures": st.cg_graph_captures}
        return pbar, stats, rc


class Batch:
    """An fh_batch: many cells of possibly different grids solved together.

    cells: list of (phase, scale or None) with phase a uint8 array or CUDA
    tensor of the cell's grid shape. The batch owns one CUDA float64 field per
    cell (``self.F[i]``, shape (9, nx, ny, nz)).
    """

    def __init__(self, cells, stream=None):
        import torch

        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.phase, self.scale, self.F = [], [], []
        arr = (FhCell * len(cells))()
        for i, (ph, sc) in enumerate(cells):
            if not isinstance(ph, torch.Tensor):
                ph = torch.as_tensor(np.ascontiguousarray(ph, dtype=np.uint8))
            ph = ph.to(device="cuda", dtype=torch.uint8).contiguous()
            if sc is not None:
                if not isinstance(sc, torch.Tensor):
                    sc = torch.as_tensor(np.ascontiguousarray(sc, dtype=np.float64))
                sc = sc.to(device="cuda", dtype=torch.float64).contiguous()
            F = torch.zeros((9,) + tuple(ph.shape), dtype=torch.float64, device="cuda")
            self.phase.append(ph)
            self.scale.append(sc)
            self.F.append(F)
            nx, ny, nz = ph.shape
            arr[i] = FhCell(nx, ny, nz, ph.data_ptr(), sc.data_ptr() if sc is not None else None, F.data_ptr())
        h = c_void_p()
        _check(lib.fh_batch_create(ctypes.byref(h), arr, len(cells), c_void_p(stream)))
        self._h = h
        self.n = len(cells)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().fh_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def fft_homog_solve_batched(self, kind, params, Fbar, n_increments=1, options=None, allow=()):
        """Returns (Pbar (n, 9), status (n,), newton (n,), cg (n,), return code)."""
        pa, pp = _dvec(params)
        fb, fbp = _dvec(Fbar, 9)
        pbar = np.zeros((self.n, 9))
        st = np.zeros(self.n, dtype=np.int32)
        nw = np.zeros(self.n, dtype=np.int32)
        cg = np.zeros(self.n, dtype=np.int32)
        rc = load().fft_homog_solve_batched(self._h, int(kind), pa.size // 2, pp, fbp, int(n_increments),
                                            ctypes.byref(options) if options is not None else None,
                                            pbar.ctypes.data_as(POINTER(c_double)),
                                            st.ctypes.data_as(POINTER(c_int)), nw.ctypes.data_as(POINTER(c_int)),
                                            cg.ctypes.data_as(POINTER(c_int)))
        _check(rc, allow=allow)
        return pbar, st, nw, cg, rc


def _ptr_array(tensors):
    arr = (c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = _ptr(t)
    return arr


class Fno:
    """An fh_fno: the learned warm-start network (include/fh_fno.h).

    Grids are nx x ny x nz with every extent >= 24; batches hold up to
    ``max_batch`` cells. Phase maps are CUDA uint8 tensors of the grid shape,
    predictions and targets CUDA float32 tensors (9, nx, ny, nz), parameter
    vectors CUDA float32 tensors of ``n_params`` entries.
    """

    def __init__(self, nx: int, ny: int, nz: int, max_batch: int = 1, train: bool = False, stream=None):
        import torch

        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.shape = (nx, ny, nz)
        self.n_params = int(lib.fh_fno_param_count())
        h = c_void_p()
        _check(lib.fh_fno_create(ctypes.byref(h), nx, ny, nz, int(max_batch), 1 if train else 0, c_void_p(stream)))
        self._h = h

    def test_skip_mma(self, skip: bool = True):
        """Failure-detection test hook: the tcgen05 projection issues no MMA, so its bounded wait runs out."""
        _check(load().fh_fno_test_skip_mma(self._h, 1 if skip else 0))

    def set_params(self, theta):
        _check(load().fh_fno_set_params(self._h, _ptr(theta)))

    def forward(self, phases, Fbar, q=None):
        """phases: list of B uint8 maps; Fbar: (B, 9); q: list of B outputs or None."""
        fb, fbp = _dvec(Fbar, 9 * len(phases))
        qa = _ptr_array(q) if q is not None else None
        _check(load().fh_fno_forward(self._h, len(phases), _ptr_array(phases), fbp, qa))

    def loss_grad(self, targets, grad=None) -> float:
        """Loss of the last forward pass; the parameter gradient into ``grad`` if given."""
        L = c_double()
        _check(load().fh_fno_loss_grad(self._h, _ptr_array(targets), ctypes.byref(L), _ptr(grad)))
        return L.value

    def adam(self, theta, grad, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
             eps: float = 1e-8, wd: float = 0.0):
        _check(load().fh_fno_adam(self._h, _ptr(theta), _ptr(grad), _ptr(m), _ptr(v), int(t), float(lr),
                                  float(beta1), float(beta2), float(eps), float(wd)))

    def make_target(self, F, Fbar, target):
        fb, fbp = _dvec(Fbar, 9)
        _check(load().fh_fno_make_target(self._h, _ptr(F), fbp, _ptr(target)))

    def warm_start(self, ctx: "Context", phase, Fbar, F):
        """F = Fbar + G(s q): the start field for fft_homog_solve with init = INIT_GIVEN."""
        fb, fbp = _dvec(Fbar, 9)
        _check(load().fh_fno_warm_start(self._h, ctx._h, _ptr(phase), fbp, _ptr(F)))

    def close(self):
        if getattr(self, "_h", None):
            load().fh_fno_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
