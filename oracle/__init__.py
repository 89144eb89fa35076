"""CPU FP64 oracle for the additive sweeping preconditioner (Liu & Ying, 2016).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
and reference legs of ``bench.py`` use it.  It shares no code with the CUDA
path: it reads plain numpy arrays (velocity, right-hand sides) produced by the
``workloads`` generator and computes everything from the paper's definitions,
in complex128, with numpy/scipy primitives (sparse assembly, LAPACK banded LU
with partial pivoting ``zgbtrf``/``zgbtrs``, dense ``numpy.linalg`` solves).

Modules and what they follow:

* :mod:`oracle.pml`        -- sigma(x) and s(x) = (1 + i sigma/omega)^-1, Section 2
  (1D PML functions) and the auxiliary profiles of Sections 2.1.1-2.1.3 / 3.1.
* :mod:`oracle.operator`   -- the discrete Helmholtz operator A: Eq. (2) (1D),
  Eq. (4) (2D), Eq. (5) (3D), with the PML put on every side as in the
  experiments of Sections 3.2 and 4.2.
* :mod:`oracle.partition`  -- the layers X_p and the padded grids X_q^M, X_p^R,
  X_p^L (Section 2, Section 3.1 "Auxiliary domains").
* :mod:`oracle.subproblems` -- H_q^M, H_p^R, H_p^L and the auxiliary Green's
  operators G~ (Section 3.1 "Auxiliary problems" / "Auxiliary Green's operators"),
  each factored once by banded LU in the quasi-1D ordering (Algorithm 1).
* :mod:`oracle.sweeping`   -- Algorithm 2 (accumulated boundary values, O(m)
  subproblem solves) and the naive O(m^2) superposition of Section 2.1.
* :mod:`oracle.nested_dissection` -- Section 4's solver of the 3D slab
  subproblems: unknowns grouped along x3, nested dissection of the column grid,
  dense frontal matrices (pinned against a sparse direct solve).
* :mod:`oracle.fgmres`     -- right-preconditioned flexible GMRES with restart,
  zero initial guess, modified Gram-Schmidt and Givens rotations (the Krylov
  solver of Section 3.2).

Pins (tests under ``tests/`` marked ``not gpu``) tie each function to facts the
paper or mathematics fix independently of this code: closed-form eigenpairs of
the PML-free operator, complex symmetry of the row-scaled operator (Section 3.1,
practical remark 4), dense brute-force solves, the boundary-value-problem form
of G~^R / G~^L, the naive-vs-accumulated identity of Section 2.2, the m=1
special case (preconditioner = A^-1), FGMRES against a dense solve, and the
nested-dissection slab solve against a sparse direct solve.
"""

from . import pml, operator, partition, subproblems, sweeping, fgmres, nested_dissection  # noqa: F401
