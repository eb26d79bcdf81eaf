"""Classical GMRES (Algorithm 1) and s-step GMRES (Algorithm 2) (oracle).

Both solve A x = b with right preconditioning, A M^-1 u = b, x = x0 + M^-1 Q y
(reading: the paper does not state the preconditioning side).  Convergence is
tested on ||b - A x|| / ||b|| (the Givens estimate inside a cycle, confirmed by
the true residual at every restart).

Algorithm 2 reading (the paper gives a skeleton and cites Yamazaki et al. 2020
for details).  With Q_f the final orthonormal columns and P the pending block
(orthogonalized once), each iteration:
  * generates s vectors V from the last column with the Newton recurrence
    v_{k+1} = A M^-1 v_k - theta_k v_k (conjugate pairs as real two-steps),
  * forms ONE Gram product G = [Q_f, P, V]^T [P, V]   (the single reduction),
  * re-orthogonalizes and re-normalizes P from G (block CGS + CholQR with the
    Pythagorean Gram correction G_PP - X_P^T X_P) - the lagged second pass,
  * assembles the Hessenberg columns of the now-final block with
    H_new = (T B - H_old T_top) T_cc^-1 and applies Givens rotations,
  * checks convergence,
  * orthogonalizes and normalizes V against all final columns (first pass).
At the end of a cycle one more reduction finalizes the last block.  Newton
shifts are the Ritz values of s classical GMRES steps of the first cycle (those
steps also supply the first s Hessenberg columns), in real Leja order; the
monomial basis uses zero shifts.
"""
import numpy as np
import scipy.linalg as sla


class GmresStats:
    def __init__(self):
        self.iters = 0           # Hessenberg columns used (linear iterations)
        self.restarts = 0
        self.true_relres = np.inf
        self.history = []        # (iteration, estimated relative residual)
        self.orth_err = []       # ||Q^T Q - I||_F per cycle
        self.shifts = None
        self.converged = False
        self.reductions = 0


def _givens(a, b):
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


class _LSQ:
    """Incremental Givens QR of the (m+1) x m Hessenberg matrix."""

    def __init__(self, m, beta):
        self.R = np.zeros((m + 1, m))
        self.cs = np.zeros(m)
        self.sn = np.zeros(m)
        self.g = np.zeros(m + 1)
        self.g[0] = beta
        self.k = 0

    def add(self, h):
        k = self.k
        h = np.array(h[:k + 2], dtype=float)
        for i in range(k):
            t = self.cs[i] * h[i] + self.sn[i] * h[i + 1]
            h[i + 1] = -self.sn[i] * h[i] + self.cs[i] * h[i + 1]
            h[i] = t
        c, s = _givens(h[k], h[k + 1])
        self.cs[k], self.sn[k] = c, s
        h[k] = c * h[k] + s * h[k + 1]
        h[k + 1] = 0.0
        self.R[:k + 1, k] = h[:k + 1]
        self.g[k + 1] = -s * self.g[k]
        self.g[k] = c * self.g[k]
        self.k += 1
        return abs(self.g[k + 1])

    def solve(self):
        k = self.k
        if k == 0:
            return np.zeros(0)
        return sla.solve_triangular(self.R[:k, :k], self.g[:k], lower=False)


def gmres(Aop, Mop, b, x0=None, tol=1e-8, restart=40, max_iters=400):
    """Algorithm 1 (MGS Arnoldi + Givens), restarted."""
    st = GmresStats()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=float)
    bn = np.linalg.norm(b)
    while True:
        r = b - Aop(x)
        beta = np.linalg.norm(r)
        st.true_relres = beta / bn
        if st.true_relres <= tol or st.iters >= max_iters:
            st.converged = st.true_relres <= tol
            return x, st
        m = min(restart, max_iters - st.iters)
        Q = np.zeros((b.size, m + 1))
        Q[:, 0] = r / beta
        lsq = _LSQ(m, beta)
        k = 0
        for j in range(m):
            v = Aop(Mop(Q[:, j]))
            h = np.zeros(j + 2)
            for i in range(j + 1):
                h[i] = v @ Q[:, i]
                v = v - h[i] * Q[:, i]
            h[j + 1] = np.linalg.norm(v)
            if h[j + 1] > 0:
                Q[:, j + 1] = v / h[j + 1]
            est = lsq.add(h)
            k = j + 1
            st.iters += 1
            st.history.append((st.iters, est / bn))
            if est / bn <= tol or h[j + 1] == 0:
                break
        y = lsq.solve()
        x = x + Mop(Q[:, :k] @ y)
        st.restarts += 1


def leja_order(theta):
    """Real Leja ordering of Ritz values: conjugate pairs adjacent, +imag first."""
    theta = [complex(t) for t in theta]
    rem = list(range(len(theta)))
    out = []

    def take(i):
        t = theta[i]
        rem.remove(i)
        if abs(t.imag) > 0:
            out.append(complex(t.real, abs(t.imag)))
            j = min(rem, key=lambda q: abs(theta[q] - t.conjugate()))
            rem.remove(j)
            out.append(complex(t.real, -abs(t.imag)))
        else:
            out.append(complex(t.real, 0.0))

    i0 = max(rem, key=lambda q: (abs(theta[q]), theta[q].imag))
    take(i0)
    while rem:
        def score(q):
            return sum(np.log(abs(theta[q] - o) + 1e-300) for o in out)
        best = max(rem, key=lambda q: (score(q), theta[q].imag))
        take(best)
    return out


def change_of_basis(shifts):
    """B ((s+1) x s) with A M^-1 [w_0..w_{s-1}] = [w_0..w_s] B for the Newton recurrence."""
    s = len(shifts)
    B = np.zeros((s + 1, s))
    for k, t in enumerate(shifts):
        B[k, k] = t.real
        B[k + 1, k] = 1.0
        if t.imag < 0:                       # second of a conjugate pair
            B[k - 1, k] = -t.imag ** 2
    return B


def _mpk(Aop, Mop, w0, shifts):
    s = len(shifts)
    V = np.zeros((w0.size, s + 1))
    V[:, 0] = w0
    for k, t in enumerate(shifts):
        v = Aop(Mop(V[:, k])) - t.real * V[:, k]
        if t.imag < 0:
            v = v + t.imag ** 2 * V[:, k - 1]
        V[:, k + 1] = v
    return V[:, 1:]


def _chol_upper(G):
    try:
        return np.linalg.cholesky(G).T
    except np.linalg.LinAlgError:
        raise FloatingPointError("CholQR breakdown: Gram matrix not positive definite")


def sstep_gmres(Aop, Mop, b, x0=None, s=4, restart=40, tol=1e-8, max_iters=400,
                basis="newton", shifts=None):
    """Algorithm 2 with lagged single-reduce BCGS2 + CholQR2 (see module docstring)."""
    st = GmresStats()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=float)
    bn = np.linalg.norm(b)
    if restart % s:
        raise ValueError("restart must be a multiple of s")
    first_cycle = True
    while True:
        r = b - Aop(x)
        beta = np.linalg.norm(r)
        st.true_relres = beta / bn
        if st.true_relres <= tol or st.iters >= max_iters:
            st.converged = st.true_relres <= tol
            return x, st
        m = min(restart, max_iters - st.iters)
        m -= m % s
        if m == 0:
            st.converged = False
            return x, st
        Qf = np.zeros((b.size, m + 1))
        Qf[:, 0] = r / beta
        H = np.zeros((m + 1, m))
        lsq = _LSQ(m, beta)
        c = 0                                  # last final column
        pend = None                            # (P, R1, S1, t0, c_start)
        done = False
        if basis == "newton" and shifts is None:
            # s classical GMRES steps supply the Ritz values and H[:, :s] (the first
            # cycle that runs them to completion fixes the shifts for later cycles)
            for j in range(s):
                v = Aop(Mop(Qf[:, j]))
                for i in range(j + 1):
                    H[i, j] = v @ Qf[:, i]
                    v = v - H[i, j] * Qf[:, i]
                H[j + 1, j] = np.linalg.norm(v)
                Qf[:, j + 1] = v / H[j + 1, j] if H[j + 1, j] > 0 else 0.0
                est = lsq.add(H[:, j])
                st.iters += 1
                st.history.append((st.iters, est / bn))
                c = j + 1
                if est / bn <= tol or H[j + 1, j] == 0:
                    done = True
                    break
            if not done:
                shifts = leja_order(np.linalg.eigvals(H[:s, :s]))
        if shifts is None and not done:
            shifts = [0j] * s                  # monomial basis
        st.shifts = shifts
        Bm = change_of_basis(shifts) if shifts is not None else None
        first_cycle = False

        def finalize(pend, c, G_P, XP):
            """Second pass of the pending block; returns new c, S2 and the block's H columns."""
            P, R1, S1, t0, cs = pend
            S2 = _chol_upper(G_P - XP.T @ XP)
            QP = sla.solve_triangular(S2.T, (P - Qf[:, :c + 1] @ XP).T, lower=True).T
            Qf[:, c + 1:c + 1 + s] = QP
            T = np.zeros((c + s + 1, s + 1))
            T[:cs + 1, 0] = t0
            T[:c + 1, 1:] = R1 + XP @ S1
            T[c + 1:, 1:] = S2 @ S1
            Hn = T @ Bm - H[:c + s + 1, :cs] @ T[:cs, :s]
            Tcc = T[cs:cs + s, :s]
            Hn = sla.solve_triangular(Tcc.T, Hn.T, lower=True).T
            H[:c + s + 1, cs:cs + s] = Hn
            return c + s, S2

        while not done:
            if pend is not None and pend[4] + s + s > m:
                break
            if pend is None and c + s > m:
                break
            # ---- matrix powers from the last column
            w0 = pend[0][:, -1] if pend is not None else Qf[:, c]
            V = _mpk(Aop, Mop, w0, shifts)
            # ---- the single reduction
            Z = Qf[:, :c + 1] if pend is None else np.hstack([Qf[:, :c + 1], pend[0]])
            G = np.hstack([Z, V]).T @ (V if pend is None else np.hstack([pend[0], V]))
            st.reductions += 1
            if pend is not None:
                nf = c + 1
                XP = G[:nf, :s]
                GPP = G[nf:nf + s, :s]
                XV = G[:nf, s:]
                GPV = G[nf:nf + s, s:]
                GVV = G[nf + s:, s:]
                cs_new = c + s                         # start column of V's block
                c_old = c
                c, S2 = finalize(pend, c, GPP, XP)
                t0 = np.concatenate([XP[:, -1], S2[:, -1]])
                for j in range(c_old, c):
                    est = lsq.add(H[:, j])
                    st.iters += 1
                    st.history.append((st.iters, est / bn))
                if est / bn <= tol:
                    done = True
                    break
                QPV = sla.solve_triangular(S2.T, GPV - XP.T @ XV, lower=True)
                R1 = np.vstack([XV, QPV])
            else:
                nf = c + 1
                R1 = G[:nf, :]
                GVV = G[nf:, :]
                cs_new = c
                t0 = np.zeros(c + 1)
                t0[c] = 1.0
            S1 = _chol_upper(GVV - R1.T @ R1)
            P = sla.solve_triangular(S1.T, (V - Qf[:, :c + 1] @ R1).T, lower=True).T
            pend = (P, R1, S1, t0, cs_new)
        if not done and pend is not None:
            # ---- flush: finalize the last block of the cycle
            Z = np.hstack([Qf[:, :c + 1], pend[0]])
            G = Z.T @ pend[0]
            st.reductions += 1
            nf = c + 1
            c_old = c
            c, _ = finalize(pend, c, G[nf:, :], G[:nf, :])
            for j in range(c_old, c):
                est = lsq.add(H[:, j])
                st.iters += 1
                st.history.append((st.iters, est / bn))
        k = lsq.k
        Qk = Qf[:, :k + 1]
        st.orth_err.append(float(np.linalg.norm(Qk.T @ Qk - np.eye(k + 1))))
        y = lsq.solve()
        x = x + Mop(Qf[:, :k] @ y)
        st.restarts += 1
