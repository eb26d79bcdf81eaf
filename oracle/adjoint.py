"""Adjoint of the linear solve x = A^-1 b for a scalar loss L(x) (oracle).

With g = dL/dx:  lambda = A^-T g,  dL/db = lambda,  dL/dA = -lambda x^T, kept on
the block-sparsity pattern of A (block (r, c) = -lambda_r x_c^T).  The
iterative form solves A^T lambda = g by s-step GMRES preconditioned with the
transposed spaND operator (apply_transpose); the dense form uses a dense solve.
"""
import numpy as np

from . import spand
from .gmres import sstep_gmres


def pattern_outer(row_ptr, col, lam, x, B):
    """-lam_r x_c^T for every stored block (r, c): [nnzb, B, B]."""
    K = len(row_ptr) - 1
    rows = np.repeat(np.arange(K), np.diff(row_ptr))
    L = lam.reshape(K, B)
    Xv = x.reshape(K, B)
    return -np.einsum("ki,kj->kij", L[rows], Xv[col])


def adjoint_iterative(Asp, F, x, g, row_ptr, col, B, s=4, restart=60, tol=1e-10, max_iters=600):
    AT = Asp.T.tocsr()
    lam, st = sstep_gmres(lambda v: AT @ v, lambda v: spand.apply_transpose(F, v), g,
                          s=s, restart=restart, tol=tol, max_iters=max_iters)
    return lam, pattern_outer(row_ptr, col, lam, x, B), st


def adjoint_dense(A_dense, x, g, row_ptr, col, B):
    lam = np.linalg.solve(A_dense.T, g)
    return lam, pattern_outer(row_ptr, col, lam, x, B)
