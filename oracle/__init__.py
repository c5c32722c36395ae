"""FP64 CPU oracle for the tensor-product nth-order FEM Poisson solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports it and shares no code, tables or constants with it.

The oracle computes what the fast solver computes, from the plain definitions
(Zlotnik & Zlotnik, "On fast Fourier solvers for the tensor product high-order
FEM for a generalized Poisson equation"):

* ``fem1d``   -- reference-element matrices A, C (Section 2, exact rationals),
                 assembled 1D operators, dense generalized eigendecomposition,
                 the element eigenproblems and the dispersion relation of
                 Section 3 (used only as pins).
* ``solve``   -- the N-D operator L of Section 4 and its inverse by dense
                 axis-wise products with the C-orthonormal 1D eigenbases
                 (algorithm (a) without any FFT), the operator apply, the
                 spectral coefficients and the gradients with respect to the
                 right-hand side and the coefficients.
* ``harness`` -- Gauss-quadrature load vectors (Section 5), manufactured
                 solutions and the mesh max-norm of Section 5.

Everything is float64 except the exact rational construction of A and C.
"""

from . import fem1d, solve, harness  # noqa: F401
