"""Seeded block matrices on the O-grid pattern with low-rank face couplings.

A test input, not a DG Jacobian: every element e of an n_theta x n_r grid
carries a dense, well-conditioned B x B diagonal block, and every face
neighbour pair (e, f) a coupling block U_e C_ef V_f^T, where U_e and V_e are
B x k with orthonormal columns drawn once per element and C_ef is k x k.
Row spaces of every block that leaves element e lie in span(U_e) and column
spaces of every block that enters it in span(V_e).  Sums and products of such
blocks keep that structure, so the couplings of any cluster of elements to the
rest of the grid, before or after eliminating other clusters, have rank at most
2k per element.  The pattern is the DG one: each element with its face
neighbours (periodic in theta, open in r), columns ascending.
"""
import numpy as np


def grid_pattern(n_theta, n_r):
    """row_ptr [K+1], col [nnzb] (int32) of the face-neighbour block pattern."""
    K = n_theta * n_r
    rows = []
    for e in range(K):
        i, j = divmod(e, n_theta)
        nb = {e, i * n_theta + (j + 1) % n_theta, i * n_theta + (j - 1) % n_theta}
        if i > 0:
            nb.add(e - n_theta)
        if i < n_r - 1:
            nb.add(e + n_theta)
        rows.append(sorted(nb))
    row_ptr = np.zeros(K + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c in r], dtype=np.int32)
    return row_ptr, col


def lowrank_coupled(n_theta, n_r, B, k, seed, coupling=0.3):
    """(row_ptr, col, val[nnzb, B, B] row-major blocks) with rank-k face couplings.

    Diagonal blocks are B x B Gaussian / sqrt(B) plus 4 I (well conditioned);
    coupling blocks U_e C_ef V_f^T with C_ef Gaussian times `coupling`.
    """
    rng = np.random.default_rng(seed)
    row_ptr, col = grid_pattern(n_theta, n_r)
    K = n_theta * n_r

    def orth(m):
        q, _ = np.linalg.qr(rng.standard_normal((B, m)))
        return q

    U = [orth(k) for _ in range(K)]
    V = [orth(k) for _ in range(K)]
    val = np.empty((len(col), B, B))
    for e in range(K):
        for t in range(row_ptr[e], row_ptr[e + 1]):
            f = int(col[t])
            if f == e:
                val[t] = rng.standard_normal((B, B)) / np.sqrt(B) + 4.0 * np.eye(B)
            else:
                C = coupling * rng.standard_normal((k, k))
                val[t] = U[e] @ C @ V[f].T
    return row_ptr, col, val
