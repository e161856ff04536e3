"""Plain FP64 CPU oracle for the p-multigrid gamma-cycle line-smoother solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from here.
The product path (the CUDA library and its Python binding) never imports,
links or executes this package, and the package shares no code with it: the
one module both sides read is ``paper_2504_10710_gb300.inputs``, which only
describes seeded synthetic problems and holds none of the method's arithmetic.

Each function follows the paper step by step, in FP64 NumPy, vectorised over
elements and lines only (no blocking, fusion or reordering of the math):

  gll.py        Def. 2.1 (GLL quadrature), Def. 2.2 (Lagrange basis),
                interpolation between orders (Sec. 3.3).
  discretize.py Sec. 2.2 eq. (discreteBilinear): geometry factors, mass,
                matrix-free stiffness apply, dense assembly; Sec. 2.3 lifting.
  lines.py      Def. 3.1 / 3.2 line systems: the line blocks R A P of each grid
                line (banded, solved by a library banded Cholesky), and their
                band-1 part; Algorithm 1, Prop. 3.7, Thm. 3.8, Cor. 3.9 (cyclic
                reduction as a direct multigrid); the damped smoothing step.
  multigrid.py  Sec. 3.3: level hierarchy, P_l / R_l = P_l^T, Def. 3.12 /
                Algorithm 2 (gamma-cycle), exact coarsest solve.
  krylov.py     Outer solvers: flexible CG, plain PCG, right-preconditioned
                GMRES (the paper's choice, Sec. 3).
  solve.py      End-to-end solve of a workload.

Readings of ambiguous passages are stated where they are used.
Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, exactness properties, brute force on tiny inputs, library
routines, or the paper's printed iteration counts (Table 1).
"""
