"""Plain FP64 CPU oracle for the fused matrix-free Jacobi-CG.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library
never calls it and shares no code with it.

Contents
--------
* ``fem``      -- 1D Gauss-Lobatto / Gauss rules, Lagrange tables, geometry
                  (Cartesian, the sine-deformed map or its tri-quadratic
                  interpolant per cell), element matrices of the
                  Laplacian (Eq. 5), element-by-element assembly into a sparse
                  matrix (Eq. 4), Dirichlet identity rows, the manufactured
                  right-hand side, sampled operator rows and the L2 error.
* ``cg``       -- textbook Jacobi-preconditioned CG (Algorithm 1) and the
                  merged-vector-operation PCG (Algorithm 5), generic over the
                  scalar type so that both also run in exact rationals.
* ``fastdiag`` -- exact discrete solve of the Cartesian problem by fast
                  diagonalisation of the Kronecker-sum operator.
"""
from . import fem, cg, fastdiag  # noqa: F401
