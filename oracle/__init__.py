"""Plain FP64 CPU oracle for the space-time dG-IgA heat-equation solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library.

What it computes (Hofer, Langer, Neumueller, arXiv:1802.09277):

* ``bspline``  -- open uniform knot vectors and Cox-de Boor B-splines (Sec. 2.1).
* ``assemble`` -- the 1D space matrices M1, K1, the SUPG-weighted time matrices
  K_t, M_t, the jump coupling N_t (Eq. 2.6 and the text after it), the global
  block lower-bidiagonal space-time matrix L_h (Eq. 2.4, Eq. 2.5) as a scipy
  CSR matrix, one block row of it applied factor by factor without assembly
  (for grids too large to assemble), load vectors, and the dG error norm
  (Sec. 2.2).
* ``solve``    -- the exact solution of L_h u = f (sparse LU), the damped
  block-Jacobi smoother of Sec. 3.1 with sparse-LU slab solves, a time-only
  V-cycle that merges slab pairs with Galerkin coarse operators, the
  plain multigrid iteration and right-preconditioned FGMRES.
* ``minres``   -- the inexact spatial solves of Sec. 3.3-3.5: the real Schur
  form with standardised 2x2 blocks, the symmetric block systems and
  preconditioners of Theorems 3.2/3.3, preconditioned MinRes, and the slab
  solve of Eq. 3.1 / Algorithm 1 with MinRes block solves.

Every function is written from the paper's definitions and is deliberately
slow: no blocking, no fusion, no fast diagonalisation.  Every function is
pinned by a ``-m "not gpu"`` test to something other than itself (printed
tables, closed forms, identities, library routines, convergence rates).
"""
