"""Pins for the spaND oracle (Sec. 2.2.1, Eqs. 10-12)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import dg, spand
from oracle.gmres import gmres
from oracle.nd import build_hierarchy
from synth import get_config, modal_state, naca_ogrid
from synth.lowrank import lowrank_coupled


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


def _truncation_checks(F, eps):
    """Eq. 12 on every recorded interface, computed from W itself: Q orthogonal,
    every column of Q_f^T W at most eps |R_00| long (|R_00| = the largest column
    norm of W, the first pivot) and r minimal (dropping one more kept column
    leaves a column longer than that)."""
    for rec in F.spars_log:
        W, Q, r = rec["W"], rec["Q"], rec["r"]
        n = W.shape[0]
        assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-12 * n
        r00 = np.linalg.norm(W, axis=0).max()
        cut = eps * r00
        Wf = Q[:, r:].T @ W
        if r < n:
            assert np.linalg.norm(Wf, axis=0).max() <= cut * (1 + 1e-9) + 1e-14 * r00
            assert np.linalg.norm(Wf, 2) <= cut * np.sqrt(W.shape[1] - r) * (1 + 1e-9) + 1e-14 * r00
        if r > 0:
            assert np.linalg.norm(Q[:, r - 1:].T @ W, axis=0).max() > cut


def test_truncation_keeps_exact_rank_of_lowrank_couplings():
    # Sec. 2.2.1: when the couplings [A_sn A_ns^T] of an interface have exact
    # rank r, its f part carries nothing, eliminating f leaves A_nn unchanged and
    # spaND is an exact solver at any small eps.  Rank-k face couplings give
    # rank 2k per element of an interface (synth.lowrank), so a level-0
    # interface of n = B |s| unknowns keeps exactly 2k |s|.
    nt, nr, p, k = 16, 8, 1, 2
    B = 4 * (p + 1) ** 2
    bsr = lowrank_coupled(nt, nr, B, k, 7, coupling=3.0)
    A = dg.bsr_to_dense(*bsr)
    eps = 1e-12
    F = spand.factor(bsr, nt, nr, 2, eps, record=True)
    lv0 = F.ranks[0]
    assert len(lv0) >= 4
    for n_s, r in lv0:
        assert r == 2 * k * (n_s // B), (n_s, r)
    b = np.random.default_rng(0).standard_normal(A.shape[0])
    x = spand.apply(F, b)
    berr = np.linalg.norm(A @ x - b) / (np.linalg.norm(A, 2) * np.linalg.norm(x) + np.linalg.norm(b))
    assert berr <= 1e-12
    xt = spand.apply_transpose(F, b)
    assert np.linalg.norm(A.T @ xt - b) / np.linalg.norm(b) <= 1e-11
    _truncation_checks(F, eps)
    # a cut that drops one more direction per interface than the exact rank
    # leaves a visible error: the exactness above is the truncation's doing
    F2 = spand.factor(bsr, nt, nr, 2, 1e-5, record=True)
    assert sum(r for _, r in F2.ranks[0]) < sum(r for _, r in lv0)
    x2 = spand.apply(F2, b)
    assert np.linalg.norm(A @ x2 - b) / np.linalg.norm(b) > 1e-8


@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-4])
def test_truncation_bound_and_minimal_rank_on_dg_jacobian(c1, eps):
    # Eq. 12 with the relative cut: ||W_f|| = O(eps) column by column, and no
    # smaller rank meets the same bound
    c, rhs, bsr, A = c1
    F = spand.factor(bsr, c.n_theta, c.n_r, c.nd_depth, eps, record=True)
    assert F.spars_log and any(rec["r"] < rec["W"].shape[0] for rec in F.spars_log)
    _truncation_checks(F, eps)


def test_truncation_is_relative_to_r00(c1):
    # a cut relative to |R_00| is invariant under scaling of A (the interface
    # scaling of Eq. 11 scales W by sqrt(alpha)); an absolute cut is not
    c, rhs, bsr, A = c1
    rp, col, val = bsr
    ref = spand.factor(bsr, c.n_theta, c.n_r, c.nd_depth, c.eps).ranks
    for alpha in (1e-6, 1e6):
        got = spand.factor((rp, col, alpha * val), c.n_theta, c.n_r, c.nd_depth, c.eps).ranks
        assert got == ref


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
