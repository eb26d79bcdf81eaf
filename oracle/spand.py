"""Sparsified nested dissection (spaND) factorization and apply (oracle).

Follows Sec. 2.2.1 of arXiv 2101.01763 level by level, l = 0 .. D:
  1. Eliminate the interiors of level l by row-pivoted block LU (Eq. 10):
       A_ss = P L U,  Y_sn = L^-1 P^T A_sn,  X_ns = A_ns U^-1,
       A_nn <- A_nn - X_ns Y_sn for every pair of neighbours of s.
  2. Scale every remaining cluster (interface) with its own PLU (Eq. 11),
     splitting diag(U) evenly: with Dg = diag(U),
       L~ = L |Dg|^(1/2),  U~ = |Dg|^(-1/2) U,  A_ss = P L~ U~,
     then A_sn <- L~^-1 P^T A_sn, A_ns <- A_ns U~^-1 and A_ss <- I.
  3. Compute every interface's Q first: column-pivoted QR (LAPACK geqp3 via
     SciPy) of W = [A_sn A_ns^T] (neighbour blocks in cluster order); keep the
     rank r = #{k : |R_kk| > eps |R_00|} (reading: the paper asks only for
     ||W_f|| = O(eps)).  Then compress every block: A_ij <- Q_ic^T A_ij Q_jc
     (Eq. 12 and the text after it); the f parts are dropped.  An interface
     with no neighbours is left unsparsified.
  4. Merge the clusters into the next level's clusters.
The product of the recorded operators is the preconditioner (A ~ prod F_i);
apply() runs the forward ops in order and the backward ops in reverse, and
apply_transpose() applies the transposed operators in the opposite order.

Vectors live in "slots": a level-0 cluster owns the DOFs of its elements; a
sparsified cluster keeps its first r slots for the coarse unknowns and the
rest hold its f part; a merged cluster concatenates its children's kept slots.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .nd import build_hierarchy


class SpandFactor:
    def __init__(self):
        self.ops = []          # forward-ordered operators
        self.N = 0
        self.ranks = []        # per level: list of (n_s, r) for sparsified interfaces
        self.flops = 0.0
        self.top_size = 0
        self.spars_log = []    # with record=True: per sparsified interface (level, W, Q, |diag R|, r)


def _lu(A):
    lu, piv = sla.lu_factor(A, check_finite=True)
    n = A.shape[0]
    perm = np.arange(n)
    for k, p in enumerate(piv):           # LAPACK row interchanges -> permutation
        perm[k], perm[p] = perm[p], perm[k]
    L = np.tril(lu, -1) + np.eye(n)
    U = np.triu(lu)
    return perm, L, U                      # A[perm] = L U


def _linv_pt(perm, L, M):
    """L^-1 P^T M, with A[perm] = L U  (P^T M = M[perm])."""
    return sla.solve_triangular(L, M[perm], lower=True, unit_diagonal=True)


def _m_uinv(U, M):
    """M U^-1."""
    return sla.solve_triangular(U, M.T, trans="T", lower=False).T


def factor(bsr, n_theta, n_r, D, eps, hierarchy=None, record=False):
    """Factor A (block-CSR tuple (row_ptr, col, val[nnzb,B,B])) with tolerance eps.

    record=True keeps, for every sparsified interface, the matrix W it was
    compressed from, its Q, |diag R| and the kept rank (F.spars_log), so that
    tests can check the truncation against W itself."""
    row_ptr, col, val = bsr
    K = len(row_ptr) - 1
    B = val.shape[1]
    A = sp.bsr_matrix((val, col, row_ptr), shape=(K * B, K * B)).tocsr()
    tree, levels = hierarchy if hierarchy is not None else build_hierarchy(n_theta, n_r, D)
    F = SpandFactor()
    F.N = K * B
    # ---- level-0 clusters and blocks
    cl = [np.concatenate([np.arange(e * B, (e + 1) * B) for e in c["elems"]]) for c in levels[0]]
    cl_of = np.empty(K, dtype=np.int64)
    for ci, c in enumerate(levels[0]):
        cl_of[c["elems"]] = ci
    pairs = set()
    for e in range(K):
        for k in range(row_ptr[e], row_ptr[e + 1]):
            pairs.add((int(cl_of[e]), int(cl_of[col[k]])))
    blocks = {}
    for a, b in sorted(pairs):
        blocks[(a, b)] = A[cl[a]][:, cl[b]].toarray()
    for l in range(D + 1):
        info = levels[l]
        alive = set(range(len(info)))
        # ---- 1. eliminate interiors (Eq. 10)
        for s in [i for i in range(len(info)) if info[i]["interior"]]:
            ns = sorted(n for (a, n) in blocks if a == s and n != s)
            ss = len(cl[s])
            if ss == 0:
                alive.discard(s)
                for n in ns:
                    blocks.pop((s, n), None)
                    blocks.pop((n, s), None)
                blocks.pop((s, s), None)
                continue
            perm, L, U = _lu(blocks.pop((s, s)))
            Y = {n: _linv_pt(perm, L, blocks.pop((s, n))) for n in ns}
            X = {n: _m_uinv(U, blocks.pop((n, s))) for n in ns}
            F.flops += 2.0 / 3.0 * ss ** 3
            for n1 in ns:
                F.flops += 2.0 * ss ** 2 * len(cl[n1])
                for n2 in ns:
                    upd = X[n1] @ Y[n2]
                    F.flops += 2.0 * len(cl[n1]) * len(cl[n2]) * ss
                    blocks[(n1, n2)] = blocks[(n1, n2)] - upd if (n1, n2) in blocks else -upd
            F.ops.append(("elim", cl[s].copy(), perm, L, U,
                          [(cl[n].copy(), X[n], Y[n]) for n in ns]))
            alive.discard(s)
            if l == D:
                F.top_size += ss
        surv = sorted(alive)
        if l == D:
            assert not surv and not blocks
            break
        # ---- 2. scale interfaces (Eq. 11)
        SL, SU = {}, {}
        for s in surv:
            perm, L, U = _lu(blocks[(s, s)])
            d = np.sqrt(np.abs(np.diag(U)))
            SL[s] = (perm, L, d)
            SU[s] = (U, d)
            F.ops.append(("scale", cl[s].copy(), perm, L, U, d))
            F.flops += 2.0 / 3.0 * len(cl[s]) ** 3
        for (a, b) in list(blocks):
            if a == b:
                blocks[(a, b)] = np.eye(len(cl[a]))
                continue
            perm, L, d = SL[a]
            M = _linv_pt(perm, L, blocks[(a, b)]) / d[:, None]
            U, db = SU[b]
            blocks[(a, b)] = _m_uinv(U, M) * db[None, :]
        # ---- 3. all Q first, then compress (Eq. 12)
        Q, rank = {}, {}
        lvl_ranks = []
        for s in surv:
            ns = sorted(n for (a, n) in blocks if a == s and n != s)
            n_s = len(cl[s])
            if not ns or n_s == 0:
                Q[s], rank[s] = np.eye(n_s), n_s
                continue
            W = np.hstack([blocks[(s, n)] for n in ns] + [blocks[(n, s)].T for n in ns])
            Qs, R, _ = sla.qr(W, pivoting=True, mode="full")
            dR = np.abs(np.diag(R))
            r = int(np.count_nonzero(dR > eps * dR[0])) if dR.size else 0
            Q[s], rank[s] = Qs, r
            F.flops += 2.0 * W.shape[1] * n_s ** 2 - 2.0 / 3.0 * n_s ** 3 if W.shape[1] >= n_s else 0.0
            lvl_ranks.append((n_s, r))
            if record:
                F.spars_log.append(dict(level=l, W=W, Q=Qs, dR=dR, r=r))
            F.ops.append(("spars", cl[s].copy(), Qs))
        F.ranks.append(lvl_ranks)
        for (a, b) in list(blocks):
            if a == b:
                blocks[(a, b)] = np.eye(rank[a])
            else:
                F.flops += 2.0 * blocks[(a, b)].shape[0] * blocks[(a, b)].shape[1] * (rank[a] + rank[b])
                blocks[(a, b)] = Q[a][:, :rank[a]].T @ blocks[(a, b)] @ Q[b][:, :rank[b]]
        for s in surv:
            cl[s] = cl[s][:rank[s]]
        # ---- 4. merge into the next level's clusters
        nxt = levels[l + 1]
        parent = {}
        new_cl = []
        for pi, pc in enumerate(nxt):
            kids = [surv[ch] for ch in pc["children"]]
            for k_ in kids:
                parent[k_] = pi
            new_cl.append(np.concatenate([cl[k_] for k_ in kids]) if kids else np.zeros(0, np.int64))
        offs = {}
        for pi, pc in enumerate(nxt):
            o = 0
            for ch in pc["children"]:
                offs[surv[ch]] = o
                o += len(cl[surv[ch]])
        new_blocks = {}
        for (a, b), M in blocks.items():
            pa, pb = parent[a], parent[b]
            if (pa, pb) not in new_blocks:
                new_blocks[(pa, pb)] = np.zeros((len(new_cl[pa]), len(new_cl[pb])))
            new_blocks[(pa, pb)][offs[a]:offs[a] + M.shape[0], offs[b]:offs[b] + M.shape[1]] = M
        cl, blocks = new_cl, new_blocks
    return F


def apply(F, r):
    """z = M^-1 r: forward ops in order, then backward ops in reverse."""
    w = np.array(r, dtype=float, copy=True)
    for op in F.ops:
        kind, sl = op[0], op[1]
        if kind == "elim":
            _, _, perm, L, U, nb = op
            y = _linv_pt(perm, L, w[sl])
            w[sl] = y
            for sn, Xn, _ in nb:
                w[sn] -= Xn @ y
        elif kind == "scale":
            _, _, perm, L, U, d = op
            w[sl] = _linv_pt(perm, L, w[sl]) / d
        else:
            w[sl] = op[2].T @ w[sl]
    for op in reversed(F.ops):
        kind, sl = op[0], op[1]
        if kind == "elim":
            _, _, perm, L, U, nb = op
            t = w[sl].copy()
            for sn, _, Yn in nb:
                t -= Yn @ w[sn]
            w[sl] = sla.solve_triangular(U, t, lower=False)
        elif kind == "scale":
            _, _, perm, L, U, d = op
            w[sl] = sla.solve_triangular(U, w[sl] * d, lower=False)
        else:
            w[sl] = op[2] @ w[sl]
    return w


def apply_transpose(F, r):
    """z = M^-T r: transposed backward ops in forward order, then transposed forward ops in reverse."""
    w = np.array(r, dtype=float, copy=True)
    for op in F.ops:
        kind, sl = op[0], op[1]
        if kind == "elim":
            _, _, perm, L, U, nb = op
            t = sla.solve_triangular(U, w[sl], trans="T", lower=False)
            w[sl] = t
            for sn, _, Yn in nb:
                w[sn] -= Yn.T @ t
        elif kind == "scale":
            _, _, perm, L, U, d = op
            w[sl] = d * sla.solve_triangular(U, w[sl], trans="T", lower=False)
        else:
            w[sl] = op[2].T @ w[sl]
    for op in reversed(F.ops):
        kind, sl = op[0], op[1]
        if kind == "elim":
            _, _, perm, L, U, nb = op
            t = w[sl].copy()
            for sn, Xn, _ in nb:
                t -= Xn.T @ w[sn]
            v = sla.solve_triangular(L, t, trans="T", lower=True, unit_diagonal=True)
            out = np.empty_like(v)
            out[perm] = v
            w[sl] = out
        elif kind == "scale":
            _, _, perm, L, U, d = op
            v = sla.solve_triangular(L, w[sl] / d, trans="T", lower=True, unit_diagonal=True)
            out = np.empty_like(v)
            out[perm] = v
            w[sl] = out
        else:
            w[sl] = op[2] @ w[sl]
    return w


def factor_bytes(F, itemsize=8):
    """Bytes of the stored operators one apply reads (both sweeps), counted from the factor."""
    tot = 0
    for op in F.ops:
        if op[0] == "elim":
            n = len(op[1])
            tot += 2 * n * n + sum(2 * len(sn) * n for sn, _, _ in op[5])
        elif op[0] == "scale":
            n = len(op[1])
            tot += 2 * n * n
        else:
            tot += 2 * op[2].size
    return tot * itemsize
