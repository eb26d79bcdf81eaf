"""Pins for the spaND oracle (Sec. 2.2.1, Eqs. 10-12)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import dg, spand
from oracle.gmres import gmres
from oracle.nd import build_hierarchy
from synth import get_config, modal_state, naca_ogrid


def _system(nt, nr, p, seed, mach=0.5, amp=0.05):
    X = naca_ogrid(nt, nr, seed)
    u = modal_state(X, p, mach, 2.0, amp, seed)
    rhs, bsr, dtau = dg.assemble(X, p, u, mach, 2.0, 10.0)
    return rhs, bsr


@pytest.fixture(scope="module")
def c1():
    c = get_config("C1")
    rhs, bsr = _system(c.n_theta, c.n_r, c.p, c.seed)
    return c, rhs, bsr, dg.bsr_to_scipy(*bsr).tocsr()


def test_eps0_is_exact_direct_solve(c1):
    c, rhs, bsr, A = c1
    F = spand.factor(bsr, c.n_theta, c.n_r, c.nd_depth, 0.0)
    x = spand.apply(F, rhs)
    xd = np.linalg.solve(A.toarray(), rhs)
    Ad = A.toarray()
    berr = np.linalg.norm(Ad @ x - rhs) / (np.linalg.norm(Ad, 2) * np.linalg.norm(x) + np.linalg.norm(rhs))
    assert berr <= 1e-12
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-9


def test_eps0_inverse_brute_force_tiny():
    rhs, bsr = _system(8, 4, 1, 5)
    A = dg.bsr_to_dense(*bsr)
    F = spand.factor(bsr, 8, 4, 2, 0.0)
    Minv = np.column_stack([spand.apply(F, e) for e in np.eye(A.shape[0])])
    assert np.allclose(Minv @ A, np.eye(A.shape[0]), atol=1e-10)
    MinvT = np.column_stack([spand.apply_transpose(F, e) for e in np.eye(A.shape[0])])
    assert np.allclose(MinvT, Minv.T, atol=1e-11)


def test_transpose_apply_adjoint_identity(c1):
    c, rhs, bsr, A = c1
    F = spand.factor(bsr, c.n_theta, c.n_r, c.nd_depth, c.eps)
    rng = np.random.default_rng(0)
    v, w = rng.standard_normal(c.N), rng.standard_normal(c.N)
    lhs = spand.apply(F, v) @ w
    rhs_ = v @ spand.apply_transpose(F, w)
    assert abs(lhs - rhs_) <= 1e-10 * abs(lhs)


def test_scaling_split_is_balanced_and_exact():
    # Eq. 11: A_ss = P L~ U~ with |diag L~| = |diag U~| = |diag U|^(1/2)
    rng = np.random.default_rng(1)
    A = rng.standard_normal((12, 12)) + 4 * np.eye(12)
    perm, L, U = spand._lu(A)
    d = np.sqrt(np.abs(np.diag(U)))
    Lt = L * d[None, :]
    Ut = U / d[:, None]
    assert np.allclose(Lt @ Ut, A[perm], atol=1e-12)
    assert np.allclose(np.abs(np.diag(Lt)), np.abs(np.diag(Ut)), atol=1e-14)
    # the scaled diagonal block is the identity: |D|^-1/2 L^-1 P^T A U^-1 |D|^1/2 = I
    S = spand._linv_pt(perm, L, A) / d[:, None]
    S = spand._m_uinv(U, S) * d[None, :]
    assert np.allclose(S, np.eye(12), atol=1e-12)


def test_sparsification_residual_bound():
    # Eq. 12: ||[W_fn W_nf^T]||_2 <= eps |R_00| sqrt(n) for the relative RRQR cut
    rng = np.random.default_rng(2)
    n, m = 30, 90
    U_, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sv = 10.0 ** -np.linspace(0, 8, n)
    W = (U_ * sv) @ rng.standard_normal((n, m))
    Q, R, _ = sla.qr(W, pivoting=True, mode="full")
    for eps in (1e-2, 1e-4, 1e-6):
        d = np.abs(np.diag(R))
        r = int(np.count_nonzero(d > eps * d[0]))
        Wf = Q[:, r:].T @ W
        assert np.linalg.norm(Wf, 2) <= eps * d[0] * np.sqrt(n)
        assert r < n


def test_iterations_monotone_in_eps(c1):
    c, rhs, bsr, A = c1
    its = []
    tree_levels = build_hierarchy(c.n_theta, c.n_r, c.nd_depth)
    for eps in (0.3, 1e-1, 1e-2, 1e-4, 0.0):
        F = spand.factor(bsr, c.n_theta, c.n_r, c.nd_depth, eps, hierarchy=tree_levels)
        _, st = gmres(lambda v: A @ v, lambda v: spand.apply(F, v), rhs, tol=1e-10, restart=60, max_iters=60)
        assert st.converged
        its.append(st.iters)
    assert all(a >= b for a, b in zip(its, its[1:])), its
    assert its[-1] == 1


def test_ranks_shrink_with_eps(c1):
    c, rhs, bsr, A = c1
    r = []
    for eps in (1e-1, 1e-2, 1e-4):
        F = spand.factor(bsr, c.n_theta, c.n_r, c.nd_depth, eps)
        r.append(sum(b for lv in F.ranks for _, b in lv))
    assert r[0] <= r[1] <= r[2]
