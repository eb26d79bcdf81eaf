"""Algorithm 1 (MGS GMRES, gmres_solve) on the GPU beside Algorithm 2, and the
per-phase stream times of both solvers.

Sec. 3.4: the s-step solver is compared with standard GMRES in a stress
setting (eps = 1e-1, tolerance 1e-10, at most 100 steps).  Checks: the GPU
MGS iterates equal the oracle's Algorithm 1 after k steps (unpreconditioned
C1 Jacobian, with and without restarts); in the stress setting both solvers
converge to the true FP64 residual target, the s-step one within a block of
the classical count, with fewer reductions; phase times are positive and sum
to at most the call's wall time.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dg  # noqa: E402
from oracle.gmres import gmres as o_gmres  # noqa: E402
from synth import get_config, modal_state, naca_ogrid  # noqa: E402


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__ as g
    g.build()
    import paper_2101_01763_gb300 as m
    return m


def _system(sg, name):
    c = get_config(name)
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
    rhs_o, bsr, _ = dg.assemble(X, c.p, u, c.mach, c.alpha_deg, c.cfl)
    A = sg.BSR.from_host(*bsr)
    return c, A, torch.as_tensor(rhs_o, device="cuda"), rhs_o, dg.bsr_to_scipy(*bsr).tocsr()


@pytest.fixture(scope="module")
def c1(sg):
    return _system(sg, "C1")


@pytest.mark.parametrize("k,restart", [(4, 4), (12, 12), (20, 8)])
def test_mgs_iterates_match_oracle(sg, c1, k, restart):
    c, A, rhs, rhs_o, S = c1
    xg, st = sg.gmres(A, None, rhs, restart=restart, tol=0.0, max_iters=k)
    xo, so = o_gmres(lambda v: S @ v, lambda v: v, rhs_o, tol=0.0, restart=restart, max_iters=k)
    assert st["iters"] == so.iters == k
    assert not st["converged"]
    xg = xg.cpu().numpy()
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-9
    if restart == k:
        # one reduction for each residual norm at the two restart checks, j + 2 for column j
        assert st["reductions"] == 2 + sum(j + 2 for j in range(k))


def _phase_sum(st):
    return st["t_spmv_ms"] + st["t_apply_ms"] + st["t_orth_ms"] + st["t_small_ms"]


@pytest.mark.parametrize("name,prec", [("C1", "fp64"), ("C2", "mixed")])
def test_stress_setting_both_solvers(sg, c1, name, prec):
    """eps = 1e-1 preconditioner, tolerance 1e-10 (the stress setting of Sec. 3.4)."""
    c, A, rhs, rhs_o, S = c1 if name == "C1" else _system(sg, name)
    F = sg.Factor(sg.Plan(c.n_theta, c.n_r, c.B, c.nd_depth), A, 0.1, prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xg, sg_st = sg.gmres(A, F, rhs, restart=60, tol=1e-10, max_iters=400)
    wall_g = 1e3 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    xs, ss_st = sg.sstep_gmres(A, F, rhs, s=4, restart=60, tol=1e-10, max_iters=400)
    wall_s = 1e3 * (time.perf_counter() - t0)
    bn = np.linalg.norm(rhs_o)
    for x, st, wall in ((xg, sg_st, wall_g), (xs, ss_st, wall_s)):
        assert st["converged"]
        assert np.linalg.norm(S @ x.cpu().numpy() - rhs_o) / bn <= 2e-10
        for key in ("t_spmv_ms", "t_apply_ms", "t_orth_ms", "t_small_ms"):
            assert st[key] > 0.0, key
        assert _phase_sum(st) <= wall + 0.5
    gi, si = sg_st["iters"], ss_st["iters"]
    if prec == "fp64":
        assert gi - 4 <= si <= gi + 8, (gi, si)   # same Krylov spaces; s-step checks per block
    assert ss_st["reductions"] < sg_st["reductions"]
    F.close()
