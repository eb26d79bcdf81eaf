"""Adjoint of the solve (torch.autograd.Function around spaND + s-step GMRES).

dL/db = lambda = A^-T w and dL/dA = -lambda x^T on the block pattern, checked
against the oracle's dense adjoint and against central finite differences
(h = 1e-6) of L = w^T A^-1 b computed with eps = 0 direct solves on the GPU.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import adjoint, dg  # noqa: E402
from synth import modal_state, naca_ogrid  # noqa: E402


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__ as g
    g.build()
    import paper_2101_01763_gb300 as m
    return m


def _system(nt, nr, p, seed):
    X = naca_ogrid(nt, nr, seed)
    u = modal_state(X, p, 0.5, 2.0, 0.05, seed)
    return dg.assemble(X, p, u, 0.5, 2.0, 10.0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_matches_dense(sg, prec):
    rhs, (rp, col, val), _ = _system(16, 8, 1, 2101_0004)
    A = sg.BSR.from_host(rp, col, val)
    plan = sg.Plan(16, 8, 16, 2)
    w = np.random.default_rng(7).standard_normal(rhs.size)
    vt = A.val.clone().requires_grad_(True)
    b = torch.as_tensor(rhs, device="cuda").requires_grad_(True)
    x = sg.SpandSolve.apply(vt, b, A, plan, 1e-3, prec, 4, 40, 1e-12)
    L = torch.dot(torch.as_tensor(w, device="cuda"), x)
    L.backward()
    Ad = dg.bsr_to_dense(rp, col, val)
    lam_d, dA_d = adjoint.adjoint_dense(Ad, np.linalg.solve(Ad, rhs), w, rp, col, 16)
    gb = b.grad.cpu().numpy()
    assert np.linalg.norm(gb - lam_d) / np.linalg.norm(lam_d) <= 1e-6
    gA = vt.grad.cpu().numpy().reshape(-1, 16, 16).transpose(0, 2, 1)    # column-major blocks -> [k, r, c]
    assert np.abs(gA - dA_d).max() <= 1e-6 * np.abs(dA_d).max()


def test_adjoint_finite_differences(sg):
    rhs, (rp, col, val), _ = _system(32, 16, 2, 2101_0044)
    A = sg.BSR.from_host(rp, col, val)
    B = 36
    plan = sg.Plan(32, 16, B, 0)
    rng = np.random.default_rng(11)
    w = rng.standard_normal(rhs.size)
    wt = torch.as_tensor(w, device="cuda")
    vt = A.val.clone().requires_grad_(True)
    b = torch.as_tensor(rhs, device="cuda").requires_grad_(True)
    x = sg.SpandSolve.apply(vt, b, A, plan, 1e-3, "fp64", 4, 60, 1e-12)
    torch.dot(wt, x).backward()
    g = vt.grad

    def loss(val_flat):
        A2 = sg.BSR(A.K, A.B, A.row_ptr, A.col, val_flat)
        F = sg.Factor(plan, A2, 0.0, "fp64")           # exact direct solve
        return torch.dot(wt, F.apply(torch.as_tensor(rhs, device="cuda"))).item()

    h = 1e-6
    for _ in range(16):
        idx = int(rng.integers(A.val.numel()))
        vp, vm = A.val.clone(), A.val.clone()
        vp[idx] += h
        vm[idx] -= h
        fd = (loss(vp) - loss(vm)) / (2 * h)
        assert abs(fd - g[idx].item()) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, g[idx].item())
    # dL/db by FD on a few entries
    for _ in range(4):
        e = int(rng.integers(rhs.size))
        bp, bm = rhs.copy(), rhs.copy()
        bp[e] += h
        bm[e] -= h
        F = sg.Factor(plan, A, 0.0, "fp64")
        fd = (torch.dot(wt, F.apply(torch.as_tensor(bp, device="cuda"))).item()
              - torch.dot(wt, F.apply(torch.as_tensor(bm, device="cuda"))).item()) / (2 * h)
        assert abs(fd - b.grad[e].item()) <= 1e-6 * max(1.0, abs(fd))


def test_pattern_outer_matches_numpy(sg):
    rhs, (rp, col, val), _ = _system(8, 4, 1, 5)
    A = sg.BSR.from_host(rp, col, val)
    rng = np.random.default_rng(2)
    u, v = rng.standard_normal(rhs.size), rng.standard_normal(rhs.size)
    o = sg.pattern_outer(A, torch.as_tensor(u, device="cuda"), torch.as_tensor(v, device="cuda"), -2.0)
    got = o.cpu().numpy().reshape(-1, 16, 16).transpose(0, 2, 1)
    # the oracle's pattern_outer gives -u v^T per block, so -2 u v^T = 2 * that
    assert np.allclose(got, 2.0 * adjoint.pattern_outer(rp, col, u, v, 16), atol=1e-14)


def test_adjoint_c4_full_size_finite_differences(sg):
    """128 x 64 O-grid, p=2 (K=8192, N=294,912), L = w^T x with seeded Gaussian w.

    dL/db: A^T lambda = w to the solve tolerance (FP64 SpMV).  dL/dA on 64 seeded
    entries against the central difference [L(A+hE) - L(A-hE)] / 2h, h = 1e-6.
    Each L(A +- hE) - L(A) is evaluated without cancellation: with x0 = A^-1 b,
    the difference d = x(A +- hE) - x0 solves (A +- hE) d = -+h E x0 exactly, and
    that system is solved by GMRES preconditioned with the eps = 0 (direct) factor
    of A, so the quotient carries the solve's relative error, not L's.
    """
    from synth import get_config
    c = get_config("C4")
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
    dev = torch.device("cuda")
    rhs, A, _ = sg.assemble(torch.as_tensor(X, device=dev), c.p, torch.as_tensor(u, device=dev), c.mach,
                            c.alpha_deg, c.cfl)
    B = A.B
    plan = sg.Plan(c.n_theta, c.n_r, B, c.nd_depth)
    rng = np.random.default_rng(c.seed + 64)
    w = torch.as_tensor(rng.standard_normal(rhs.numel()), device=dev)
    vt = A.val.clone().requires_grad_(True)
    b = rhs.clone().requires_grad_(True)
    x = sg.SpandSolve.apply(vt, b, A, plan, c.eps, "mixed", c.s, c.restart, 1e-12)
    torch.dot(w, x).backward()
    lam, g = b.grad, vt.grad
    # dL/db = lambda solves A^T lambda = w
    r = sg.spmv(A, lam, transpose=True) - w
    assert (torch.linalg.norm(r) / torch.linalg.norm(w)).item() <= 1e-10
    # the direct (eps = 0) factor of A as an exact preconditioner
    F0 = sg.Factor(plan, A, 0.0, "fp64")
    x0, st0 = sg.sstep_gmres(A, F0, rhs, s=c.s, restart=c.restart, tol=1e-13)
    assert st0["converged"] and st0["iters"] <= 8
    rp, col = A.row_ptr.cpu().numpy(), A.col.cpu().numpy()
    h = 1e-6
    x0h = x0.cpu().numpy()
    for _ in range(64):
        idx = int(rng.integers(A.val.numel()))
        k, rem = divmod(idx, B * B)
        cc, rr = divmod(rem, B)                       # column-major block: index = rr + cc * B
        i = int(np.searchsorted(rp, k, side="right") - 1) * B + rr
        j = int(col[k]) * B + cc
        diffs = []
        for sgn in (1.0, -1.0):
            v2 = A.val.clone()
            v2[idx] += sgn * h
            A2 = sg.BSR(A.K, A.B, A.row_ptr, A.col, v2)
            e = torch.zeros_like(rhs)
            e[i] = -sgn * h * x0h[j]
            d, std = sg.sstep_gmres(A2, F0, e, s=c.s, restart=c.restart, tol=1e-12)
            assert std["converged"]
            diffs.append(torch.dot(w, d).item())
        fd = (diffs[0] - diffs[1]) / (2 * h)
        got = g[idx].item()
        assert abs(fd - got) <= 1e-6 * max(abs(fd), 1e-3 * g.abs().max().item()), (idx, fd, got)
    F0.close()
