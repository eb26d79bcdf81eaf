"""Plain FP64 CPU oracle for the DG-Jacobian spaND + s-step GMRES solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this tree;
only the tests, the smoke check and the CPU-baseline leg of the benchmark call
it.  It is written to be checked against the paper by eye: NumPy/SciPy library
calls (LU, pivoted QR, dense solves, eigenvalues) serve as steps, with no
blocking or fusion beyond what each passage states.

Modules and the passages they follow (arXiv 2101.01763):
  dg       Sec. 2.1.2, Eqs. 3-8: modal DG residual R, mass M, analytic dR/du,
           CFL time step; A = M/dtau + dR/du and b = -R (Eq. 5).
  nd       Sec. 2.2.1 and Sec. 3.3: nested dissection of the (i, j) element grid,
           interiors / separators / interfaces per level, merges.
  spand    Sec. 2.2.1, Eqs. 10-12: per-level elimination, interface scaling and
           RRQR sparsification; the resulting preconditioner and its transpose.
  gmres    Algorithm 1 (classical GMRES) and Algorithm 2 (s-step GMRES with
           single-reduce re-orthogonalization, Newton basis, Sec. 3.4).
  adjoint  dense adjoint of the linear solve (derivative of L = w^T x).

Parity status: every function is pinned by tests under tests/ (closed forms,
invariants, finite differences, brute force, library special cases); the
Newton-shift choice is pinned only up to its Ritz set.
"""
