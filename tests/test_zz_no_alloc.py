"""fh_project_static: the projection for callers that cannot allocate GPU memory.

Code hosted inside another application that owns the device's memory, or a
loop that must not allocate once running, cannot create an fh_ctx (its
scratch comes from cudaMalloc). fh_project_static serves them from a static
device array instead. These tests call it through the C-ABI twice in a row
(the second call on a smaller grid, so the shared array still holds the
first call's data) and require the same result as the allocating
fh_project, within the tolerance the operator tests use (1e-12 relative).
A third call writes its result over its input (out is A), which the header
allows. They also check that a grid above the static limit is refused with
an error, and that a call allocates no device memory: once a first call has
loaded its kernels, a second call leaves both the driver's free-memory count
and PyTorch's allocated bytes unchanged.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""

import numpy as np
import pytest

from gpu_helpers import dev, host, require_gpu

pytestmark = pytest.mark.gpu

OP_TOL = 1e-12


def test_static_projection_matches_fh_project_on_two_calls_in_a_row():
    torch = require_gpu()
    import paper_2408_03804_gb300 as fh
    from paper_2408_03804_gb300 import _binding

    lib = fh.load()
    cases = [((32, 32, 32), (1.0, 1.0, 1.0), 1.0), ((8, 16, 4), (1.0, 2.0, 0.5), -0.75)]
    rng = np.random.default_rng(2024)
    for shape, lengths, scale in cases:
        A = dev(rng.standard_normal((9,) + shape))
        ref = torch.empty_like(A)
        with fh.Context(*shape) as ctx:
            ctx.fh_project(A, ref, scale=scale, lengths=lengths)
        out = torch.full_like(A, float("nan"))
        La = np.asarray(lengths, dtype=np.float64)
        rc = lib.fh_project_static(A.data_ptr(), out.data_ptr(), *shape, scale,
                                   La.ctypes.data_as(_binding.POINTER(_binding.c_double)),
                                   _binding.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == fh.FH_OK, lib.fh_last_error_string()
        r, o = host(ref), host(out)
        assert np.isfinite(o).all()
        assert np.abs(o - r).max() <= OP_TOL * np.abs(r).max()
    # in place: out is A (same grid as the last call, fresh data)
    shape, lengths, scale = cases[-1]
    A = dev(rng.standard_normal((9,) + shape))
    ref = torch.empty_like(A)
    with fh.Context(*shape) as ctx:
        ctx.fh_project(A, ref, scale=scale, lengths=lengths)
    La = np.asarray(lengths, dtype=np.float64)
    rc = lib.fh_project_static(A.data_ptr(), A.data_ptr(), *shape, scale,
                               La.ctypes.data_as(_binding.POINTER(_binding.c_double)),
                               _binding.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == fh.FH_OK, lib.fh_last_error_string()
    r, o = host(ref), host(A)
    assert np.abs(o - r).max() <= OP_TOL * np.abs(r).max()


def test_static_projection_allocates_no_device_memory():
    torch = require_gpu()
    import paper_2408_03804_gb300 as fh

    lib = fh.load()
    shape = (16, 16, 16)
    A = dev(np.random.default_rng(7).standard_normal((9,) + shape))
    out = torch.empty_like(A)
    stream = torch.cuda.current_stream().cuda_stream
    # the first call on this grid loads its kernels (module memory) and the static tables
    assert lib.fh_project_static(A.data_ptr(), out.data_ptr(), *shape, 1.0, None, stream) == fh.FH_OK
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    first = host(out)
    assert lib.fh_project_static(A.data_ptr(), out.data_ptr(), *shape, 1.0, None, stream) == fh.FH_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert np.array_equal(host(out), first)


def test_static_projection_rejects_grids_above_its_limit():
    torch = require_gpu()
    import paper_2408_03804_gb300 as fh

    lib = fh.load()
    A = torch.zeros((9, 64, 32, 32), dtype=torch.float64, device="cuda")  # 65536 voxels > 32768
    rc = lib.fh_project_static(A.data_ptr(), A.data_ptr(), 64, 32, 32, 1.0, None, None)
    assert rc == fh.FH_ERR_ARG
    assert b"static scratch limit" in lib.fh_last_error_string()
