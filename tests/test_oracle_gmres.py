"""Pins for GMRES (Algorithm 1) and s-step GMRES (Algorithm 2)."""
import numpy as np
import pytest

from oracle import adjoint, dg, spand
from oracle.gmres import change_of_basis, gmres, leja_order, sstep_gmres
from synth import get_config, modal_state, naca_ogrid


def _tiny(n=150, seed=0, shift=3.0):
    rng = np.random.default_rng(seed)
    A = shift * np.eye(n) + rng.standard_normal((n, n)) / np.sqrt(n)
    return A, rng.standard_normal(n)


def test_gmres_matches_dense_solve():
    A, b = _tiny()
    x, st = gmres(lambda v: A @ v, lambda v: v, b, tol=1e-12, restart=30, max_iters=300)
    assert st.converged
    assert np.linalg.norm(x - np.linalg.solve(A, b)) / np.linalg.norm(x) < 1e-10


def test_gmres_iterate_is_krylov_minimizer():
    """Algorithm 1 after k steps (x0 = 0, right preconditioning): x_k = M z with z minimising
    ||b - A M z|| over span{b, (AM) b, ..., (AM)^(k-1) b}, here by brute force: an orthonormal
    basis of the explicit Krylov matrix and a dense least-squares solve."""
    A, b = _tiny(n=120, seed=21)
    M = np.diag(1.0 + 0.3 * np.sin(np.arange(120)))
    AM = A @ M
    for k in (1, 3, 7, 12):
        K = np.empty((120, k))
        K[:, 0] = b / np.linalg.norm(b)
        for j in range(1, k):
            v = AM @ K[:, j - 1]
            K[:, j] = v / np.linalg.norm(v)
        Qk, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(AM @ Qk, b, rcond=None)
        x_ref = M @ (Qk @ y)
        x, st = gmres(lambda v: A @ v, lambda v: M @ v, b, tol=0.0, restart=k, max_iters=k)
        assert st.iters == k
        assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-9


@pytest.mark.parametrize("basis", ["newton", "monomial"])
@pytest.mark.parametrize("s", [2, 4, 5])
def test_sstep_iterates_equal_gmres(basis, s):
    """Same Krylov space, same minimisation: iterates coincide at k = s, 2s, ... (Sec. 2.3)."""
    A, b = _tiny(n=160, seed=s)
    M = np.diag(1.0 + 0.1 * np.arange(160) / 160)
    for k in (s, 2 * s, 3 * s, 5 * s):
        x1, _ = gmres(lambda v: A @ v, lambda v: M @ v, b, tol=0.0, restart=k, max_iters=k)
        x2, st = sstep_gmres(lambda v: A @ v, lambda v: M @ v, b, s=s, restart=k, tol=0.0,
                             max_iters=k, basis=basis)
        assert st.iters == k
        assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) <= 1e-10


def test_single_reduction_per_block():
    A, b = _tiny(n=100, seed=9)
    _, st = sstep_gmres(lambda v: A @ v, lambda v: v, b, s=4, restart=24, tol=0.0, max_iters=24)
    # Newton: 4 Arnoldi columns, then 5 MPK blocks (one reduction each) + one flush
    assert st.reductions == 5 + 1
    _, st = sstep_gmres(lambda v: A @ v, lambda v: v, b, s=4, restart=24, tol=0.0, max_iters=24,
                        basis="monomial")
    assert st.reductions == 6 + 1


def test_leja_order_pairs_adjacent():
    th = [1.0 + 2j, 1.0 - 2j, 3.0, -0.5, 0.2 + 0.1j, 0.2 - 0.1j]
    o = leja_order(th)
    assert abs(o[0] - (1.0 + 2j)) < 1e-15 or abs(o[0] - 3.0) < 1e-15
    assert abs(abs(o[0]) - max(abs(t) for t in th)) < 1e-12
    for k, t in enumerate(o):
        if t.imag > 0:
            assert o[k + 1] == t.conjugate()
    assert sorted(o, key=lambda z: (z.real, z.imag)) == sorted(th, key=lambda z: (z.real, z.imag))


def test_change_of_basis_reproduces_newton_recurrence():
    rng = np.random.default_rng(4)
    n = 40
    A = rng.standard_normal((n, n))
    sh = leja_order([0.5 + 0.3j, 0.5 - 0.3j, -1.0, 2.0])
    W = np.zeros((n, 5))
    W[:, 0] = rng.standard_normal(n)
    for k, t in enumerate(sh):
        W[:, k + 1] = A @ W[:, k] - t.real * W[:, k] + (t.imag ** 2 * W[:, k - 1] if t.imag < 0 else 0)
    assert np.allclose(A @ W[:, :4], W @ change_of_basis(sh), atol=1e-10)


def test_orthogonality_newton_reortho():
    """Fig. 6: Newton basis + re-orthogonalization keeps ||Q^T Q - I||_F <= 1e-10."""
    A, b = _tiny(n=300, seed=7, shift=2.0)
    _, st = sstep_gmres(lambda v: A @ v, lambda v: v, b, s=4, restart=60, tol=1e-13, max_iters=60)
    assert max(st.orth_err) <= 1e-10


def test_c1_solution_matches_dense():
    c = get_config("C1")
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
    rhs, bsr, _ = dg.assemble(X, c.p, u, c.mach, c.alpha_deg, c.cfl)
    A = dg.bsr_to_scipy(*bsr).tocsr()
    F = spand.factor(bsr, c.n_theta, c.n_r, c.nd_depth, c.eps)
    x, st = sstep_gmres(lambda v: A @ v, lambda v: spand.apply(F, v), rhs, s=c.s,
                        restart=c.restart, tol=c.tol)
    assert st.converged and st.true_relres <= 1e-8
    xd = np.linalg.solve(A.toarray(), rhs)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-6
    # the paper's stress setting: crude eps -> several s-blocks and restarts
    F1 = spand.factor(bsr, c.n_theta, c.n_r, c.nd_depth, 0.5)
    x1, st1 = sstep_gmres(lambda v: A @ v, lambda v: spand.apply(F1, v), rhs, s=c.s,
                          restart=8, tol=1e-10, max_iters=400)
    assert st1.converged and np.linalg.norm(x1 - xd) / np.linalg.norm(xd) <= 1e-7


def test_adjoint_iterative_matches_dense_and_fd():
    rng = np.random.default_rng(11)
    X = naca_ogrid(8, 4, 13)
    u = modal_state(X, 1, 0.5, 2.0, 0.05, 13)
    rhs, bsr, _ = dg.assemble(X, 1, u, 0.5, 2.0, 10.0)
    rp, col, val = bsr
    A = dg.bsr_to_scipy(*bsr).tocsr()
    Ad = A.toarray()
    F = spand.factor(bsr, 8, 4, 2, 1e-2)
    x = np.linalg.solve(Ad, rhs)
    w = rng.standard_normal(rhs.size)
    lam, dA, st = adjoint.adjoint_iterative(A, F, x, w, rp, col, 16, tol=1e-12)
    lam_d, dA_d = adjoint.adjoint_dense(Ad, x, w, rp, col, 16)
    assert np.linalg.norm(lam - lam_d) / np.linalg.norm(lam_d) <= 1e-9
    assert np.allclose(dA, dA_d, rtol=1e-8, atol=1e-10 * np.abs(dA_d).max())
    # central FD of L = w^T A^-1 b on seeded entries (exact dense solves)
    for _ in range(16):
        k = rng.integers(len(col))
        i, j = rng.integers(16, size=2)
        h = 1e-6
        vp, vm = val.copy(), val.copy()
        vp[k, i, j] += h
        vm[k, i, j] -= h
        Lp = w @ np.linalg.solve(dg.bsr_to_dense(rp, col, vp), rhs)
        Lm = w @ np.linalg.solve(dg.bsr_to_dense(rp, col, vm), rhs)
        assert abs((Lp - Lm) / (2 * h) - dA_d[k, i, j]) <= 1e-6 * max(1.0, abs(dA_d[k, i, j]))
    # dL/db = lambda
    e = rng.integers(rhs.size)
    bp, bm = rhs.copy(), rhs.copy()
    bp[e] += 1e-6
    bm[e] -= 1e-6
    fd = (w @ np.linalg.solve(Ad, bp) - w @ np.linalg.solve(Ad, bm)) / 2e-6
    assert abs(fd - lam_d[e]) <= 1e-6 * max(1.0, abs(fd))
