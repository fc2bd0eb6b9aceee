"""The C-ABI library builds, loads and exports every symbol its header declares.

No compute call is made here (this machine may have no GPU); only entry
points that reject their arguments before touching the device are called.
"""

import ctypes
import os
import re

import pytest

from paper_2408_03804_gb300 import _binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _binding.load()


def _declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*FH_API\s+[\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("fh_", "fft_homog"))))


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert set(declared) == set(_binding.EXPORTS), declared
    for name in declared:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_only_declared_symbols_are_exported(lib):
    out = os.popen(f"nm -D --defined-only {_binding.library_path()}").read()
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    ours = {s for s in exported if s.startswith(("fh_", "fft_homog"))}
    assert ours == set(_binding.EXPORTS)


def test_default_options(lib):
    o = _binding.default_options()
    assert o.newton_tol == 1e-8 and o.cg_tol == 0.0 and o.max_newton == 50 and o.max_cg == 5000
    assert o.check_every == 16 and list(o.lengths) == [1.0, 1.0, 1.0]
    assert o.launch_mode == _binding.LAUNCH_GRAPH and o.matvec_arith == _binding.ARITH_FP64
    assert ctypes.sizeof(_binding.FhOptions) == 72


@pytest.mark.parametrize("shape", [(4, 4, 3), (4, 4, 5), (513, 4, 4), (4, 1024, 4), (4, 4, 10), (0, 4, 4),
                                   (4, 0, 4), (4, 4, 18), (4, 4, 512)])
def test_create_rejects_unsupported_grids_without_touching_the_device(lib, shape):
    h = ctypes.c_void_p()
    rc = lib.fh_create(ctypes.byref(h), *shape, None)
    assert rc == _binding.FH_ERR_ARG
    assert b"3*2^a" in lib.fh_last_error_string()
    assert not h.value


def test_null_arguments_are_rejected(lib):
    assert lib.fh_create(None, 4, 4, 4, None) == _binding.FH_ERR_ARG
    assert lib.fft_homog_solve(None, None, None, 1, None, None, None, None) == _binding.FH_ERR_ARG
    assert lib.fh_project(None, None, None, 1.0, None) == _binding.FH_ERR_ARG
    lib.fh_destroy(None)
