"""Plain FP64 CPU oracle for the vertex-patch smoother with a local p-multigrid solver.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it, and it shares no code with the CUDA library: every matrix here
is assembled explicitly from its definition, with dense linear algebra.

Modules
  rules    1D Gauss / Gauss-Lobatto rules (Golub-Welsch) and Lagrange bases
  fem      Q1 geometry, element matrices, load vectors, global assembly
  patch    vertex patches, p-levels, p-transfers, smoothers, V-cycle (Alg. 2),
           multiplicative colour-major sweep (Alg. 1)
  gmg      h-hierarchy, h-transfers, global GMG V-cycle, dense coarse Cholesky, PCG
  lanczos  counter-based start vectors, Lanczos, Sturm bisection, Chebyshev bounds
"""
