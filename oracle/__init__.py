"""FP64 CPU oracle for the Gauss-Newton Hessian-action path (test infrastructure).

This package is a plain, slow, obviously-correct restatement of what the CUDA
path computes.  It is test infrastructure: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product path never calls it and the
two share no code.

Modules
  fem        structured P1 meshes, generic element matrices, CSR assembly,
             pointwise observation operator     (Sections 2.3, 5.1, Appendix C)
  inverse    forward / adjoint / gradient / Gauss-Newton Hessian action,
             bilaplacian prior, cost            (Section 5.1, Appendix A)
  algorithms inexact Newton-CG (Algorithm 1), double-pass randomized
             eigensolver with PreCholQR (Algorithms 2, 4), single-pass
             variant (Algorithm 3), Laplace sampling (Section 4.3),
             pointwise variance (Section 4.4)

Every linear solve is a sparse direct factorisation (scipy SuperLU), i.e. a
library primitive, so oracle results are exact up to rounding.

Parity pins (tests/test_oracle_*.py) tie each function to something other
than itself: closed-form element matrices, a second independent derivation of
the stencil, the linear exact solution for m = 0, manufactured-solution
O(h^2) convergence, finite-difference gradient and Hessian checks, symmetry,
dense generalized eigendecomposition on tiny grids, and the exact covariance
of the linear sampling maps.
"""
