"""CPU oracle for the Fourier-Galerkin Newton-Krylov homogenization method.

TEST INFRASTRUCTURE. This package is a plain, slow, FP64 NumPy/SciPy
restatement of what the GPU library computes, written from the paper
(Pundir & Kammer, "Simplifying FFT-based methods for solid mechanics with
automatic differentiation"): the equilibrium equation in Fourier form
(Eq. 1), stress and tangent from an energy density (Eqs. 2-3), the
Newton-Krylov solver (Appendix A, Algorithm 1) and the homogenized stress
(Eq. 4). Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product library never does, and the two share
no code. Inputs come from ``rve_inputs``, which holds no method arithmetic.

Modules
-------
spectral   wave vectors and the compatibility projection G (Eq. 1)
materials  closed-form energies, stresses and tangents (Eqs. 2-3)
solver     Newton-Krylov solve with a conjugate-gradient inner loop (Alg. 1)
laminate   exact laminate solutions (an independent pin of the solver)
brute      dense energy minimisation on tiny grids (an independent pin)
homogenize homogenized tangent (Eq. 4) and modulus sensitivities (Section 4.4.2)

Readings of the paper taken here where it is silent or garbled are listed in
each function's docstring; every function is pinned by a ``-m "not gpu"``
test against something other than itself.
"""

from . import spectral, materials, solver, laminate, brute, homogenize  # noqa: F401
