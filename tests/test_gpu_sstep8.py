"""s-step GMRES at the large workload's solver settings (s = 8, restart 80) on
the GPU, through the C ABI (Algorithm 2, Sec. 2.3).

* Unpreconditioned iterates after k = 8, 16 and 32 columns of one cycle equal
  the oracle's Algorithm 2 to 1e-10 (Newton and monomial bases).
* A p = 3 system (32 x 16 O-grid, N = 32,768, the large workload's flow) with a
  deliberately weak preconditioner (CFL 100, eps = 0.5, tol 1e-10) runs more
  than 2s columns, so the Gram reduction, the lagged CGS2 + CholQR2 pass and
  the Hessenberg assembly of several s-blocks run; the FP64 and mixed solutions
  match a sparse direct solve.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dg, spand  # noqa: E402
from oracle.gmres import sstep_gmres as o_sstep  # noqa: E402
from synth import get_config, modal_state, naca_ogrid  # noqa: E402


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__ as g
    g.build()
    import paper_2101_01763_gb300 as m
    return m


def _system(c, cfl=None):
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
    return dg.assemble(X, c.p, u, c.mach, c.alpha_deg, c.cfl if cfl is None else cfl)


@pytest.mark.parametrize("basis", ["newton", "monomial"])
def test_sstep8_iterates_match_oracle(sg, basis):
    c = get_config("C1")
    rhs_o, bsr, _ = _system(c)
    A = sg.BSR.from_host(*bsr)
    S = dg.bsr_to_scipy(*bsr).tocsr()
    rhs = torch.as_tensor(rhs_o, device="cuda")
    for k in (8, 16, 32):
        xg, st = sg.sstep_gmres(A, None, rhs, s=8, restart=80, tol=0.0, max_iters=k, basis=basis)
        xo, so = o_sstep(lambda v: S @ v, lambda v: v, rhs_o, s=8, restart=80, tol=0.0, max_iters=k, basis=basis)
        assert st["iters"] == so.iters == k
        xg = xg.cpu().numpy()
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10, (k, basis)


@pytest.fixture(scope="module")
def p3case():
    c = get_config("C3").with_(n_theta=32, n_r=16)
    rhs_o, bsr, _ = _system(c, cfl=100.0)
    S = dg.bsr_to_scipy(*bsr).tocsr()
    import scipy.sparse.linalg as spla
    xr = spla.spsolve(S.tocsc(), rhs_o)
    return c, rhs_o, bsr, S, xr


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sstep8_p3_many_blocks(sg, p3case, prec):
    c, rhs_o, bsr, S, xr = p3case
    A = sg.BSR.from_host(*bsr)
    F = sg.Factor(sg.Plan(c.n_theta, c.n_r, c.B, c.nd_depth), A, 0.5, prec)
    x, st = sg.sstep_gmres(A, F, torch.as_tensor(rhs_o, device="cuda"), s=8, restart=80, tol=1e-10,
                           max_iters=400)
    x = x.cpu().numpy()
    assert st["converged"]
    assert st["iters"] > 16 and st["reductions"] >= 2, st          # several s-blocks ran
    relres = np.linalg.norm(S @ x - rhs_o) / np.linalg.norm(rhs_o)
    assert relres <= 1e-10
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-6
    if prec == "fp64":
        # the oracle's Algorithm 2 with the oracle's factor takes the same number of blocks
        Fo = spand.factor(bsr, c.n_theta, c.n_r, c.nd_depth, 0.5)
        _, so = o_sstep(lambda v: S @ v, lambda v: spand.apply(Fo, v), rhs_o, s=8, restart=80, tol=1e-10,
                        max_iters=400)
        assert abs(st["iters"] - so.iters) <= 8, (st["iters"], so.iters)
        assert st["orth_err"] <= 1e-10
