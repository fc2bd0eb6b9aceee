"""GB300 (sm_103a) library for AD-enhanced Fourier-Galerkin homogenization.

Hot path of Pundir & Kammer, "Simplifying FFT-based methods for solid
mechanics with automatic differentiation": the matrix-free Newton-Krylov
solve of the periodic cell problem (Eq. 1, Appendix A Algorithm 1) with
stress and tangent from forward-mode dual numbers (Eqs. 2-3) and the
homogenized stress (Eq. 4). All compute runs in the CUDA library under
``csrc/`` behind the C-ABI declared in ``include/fft_homog.h``; this package
is a thin ctypes binding (``_binding``) plus the in-tree build (``build``).
"""

from ._binding import (  # noqa: F401
    ARITH_DF64, ARITH_FP64, FH_ERR_ARG, FH_ERR_CUDA, FH_ERR_NONPHYSICAL, FH_ERR_NOT_CONVERGED, FH_ERR_TIMEOUT, FH_ERR_UNSUPPORTED, FH_OK,
    INIT_GIVEN, INIT_REFERENCE, J2, LAUNCH_GRAPH, LAUNCH_PLAIN, LINEAR_ELASTIC, NEO_HOOKEAN, SVK, TANGENT_JVP, TANGENT_STORED, EXPORTS,
    Batch, Context, FhError, Fno, Material, default_options, fh_df64_roundtrip, fh_probe_fp64, fh_twiddle_tables, library_path, load,
)
