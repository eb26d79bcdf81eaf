"""Pseudo-time continuation on the GPU (dg_pseudo_time_march) against the oracle.

Sec. 2.1.2, Eqs. 5, 8, 9.  At C1 size every assembled state is compared with
the oracle's march (dense solves): residual norms, CFL numbers and dtau of
each step, and the final state.  The linear tolerance is 1e-12, so the two
trajectories differ by the solve error only.  At C2 size (the benchmark's
workload), the oracle evaluates R at the GPU's states, and the first update
is checked against the oracle's Jacobian.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dg, march  # noqa: E402
from synth import get_config, modal_state, naca_ogrid  # noqa: E402
from synth.state import uniform_modal_state  # noqa: E402


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__ as g
    g.build()
    import paper_2101_01763_gb300 as m
    return m


def _case(name):
    c = get_config(name)
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u0 = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
    return c, X, u0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_march_c1_matches_oracle(sg, prec):
    c, X, u0 = _case("C1")
    steps, cfl0, cfl_inf = 6, 100.0, 1e6
    uo, ho = march.march(X, c.p, u0, c.mach, c.alpha_deg, cfl0, cfl_inf, steps)
    plan = sg.Plan(c.n_theta, c.n_r, c.B, c.nd_depth)
    dev = torch.device("cuda")
    ug, hg = sg.march(torch.as_tensor(X, device=dev), c.p, torch.as_tensor(u0, device=dev), c.mach, c.alpha_deg,
                      plan, cfl0=cfl0, cfl_inf=cfl_inf, max_steps=steps, rtol=0.0, eps=c.eps, precision=prec,
                      s=c.s, restart=c.restart, tol=1e-12, max_iters=400)
    assert hg["steps"] == steps
    assert np.allclose(hg["res"], ho["res"], rtol=1e-8, atol=0)
    assert np.allclose(hg["cfl"], ho["cfl"], rtol=1e-8, atol=0)
    assert np.allclose(hg["dtau"], ho["dtau"], rtol=1e-8, atol=0)
    assert np.all(hg["gmres_iters"] > 0)
    u = ug.cpu().numpy()
    assert np.max(np.abs(u - uo)) <= 1e-9 * np.max(np.abs(uo))


def test_march_newton_limit_and_stop(sg):
    """Large CFL^0: quadratic convergence to rtol, stopping before a further solve."""
    c, X, u0 = _case("C1")
    plan = sg.Plan(c.n_theta, c.n_r, c.B, c.nd_depth)
    dev = torch.device("cuda")
    ug, hg = sg.march(torch.as_tensor(X, device=dev), c.p, torch.as_tensor(u0, device=dev), c.mach, c.alpha_deg,
                      plan, cfl0=1e4, cfl_inf=1e14, max_steps=12, rtol=1e-11, eps=0.0, precision="fp64",
                      s=c.s, restart=c.restart, tol=1e-13, max_iters=400)
    r = hg["res"]
    assert r[-1] <= 1e-11 * r[0] and np.all(r[:-1] > 1e-11 * r[0])    # stopped at the first state below rtol
    assert hg["steps"] == len(r) - 1 <= 8
    uo, ho = march.march(X, c.p, u0, c.mach, c.alpha_deg, 1e4, 1e14, hg["steps"])
    big = ho["res"] > 1e-8 * ho["res"][0]
    assert np.allclose(r[big], ho["res"][big], rtol=1e-6, atol=0)
    R = dg.residual(X, c.p, ug.cpu().numpy(), c.mach, c.alpha_deg)
    assert np.linalg.norm(R) <= 1e-11 * r[0] * 1.01


def test_march_free_stream_stays(sg):
    """A uniform free stream with far field everywhere is steady: R is round-off
    and the march leaves the state where it is."""
    c = get_config("C1")
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u0 = uniform_modal_state(c.n_theta * c.n_r, c.p, c.mach, c.alpha_deg)
    plan = sg.Plan(c.n_theta, c.n_r, c.B, c.nd_depth)
    dev = torch.device("cuda")
    ut = torch.as_tensor(u0, device=dev)
    ug, hg = sg.march(torch.as_tensor(X, device=dev), c.p, ut, c.mach, c.alpha_deg, plan, cfl0=10.0,
                      cfl_inf=1e6, max_steps=2, rtol=0.0, eps=c.eps, precision="fp64", s=c.s,
                      restart=c.restart, tol=1e-8, bc="farfield")
    assert np.all(hg["res"] <= 1e-10)
    assert torch.max(torch.abs(ug - ut)).item() <= 1e-12


def test_march_c2_states_against_oracle(sg):
    """C2 (64 x 32, p = 2, N = 73,728), mixed form, 3 steps from CFL^0 = 10."""
    c, X, u0 = _case("C2")
    plan = sg.Plan(c.n_theta, c.n_r, c.B, c.nd_depth)
    dev = torch.device("cuda")
    Xd = torch.as_tensor(X, device=dev)
    u1, h1 = sg.march(Xd, c.p, torch.as_tensor(u0, device=dev), c.mach, c.alpha_deg, plan, cfl0=c.cfl,
                      cfl_inf=1e6, max_steps=1, rtol=0.0, eps=c.eps, precision="mixed", s=c.s,
                      restart=c.restart, tol=1e-10, max_iters=c.max_iters)
    u3, h3 = sg.march(Xd, c.p, torch.as_tensor(u0, device=dev), c.mach, c.alpha_deg, plan, cfl0=c.cfl,
                      cfl_inf=1e6, max_steps=3, rtol=0.0, eps=c.eps, precision="mixed", s=c.s,
                      restart=c.restart, tol=1e-10, max_iters=c.max_iters)
    # R at u^0, u^1 and u^3 by the oracle
    for h, n, u in ((h1, 0, u0), (h1, 1, u1.cpu().numpy()), (h3, 3, u3.cpu().numpy())):
        Ro = dg.residual(X, c.p, u, c.mach, c.alpha_deg)
        assert abs(h["res"][n] - np.linalg.norm(Ro)) <= 1e-9 * np.linalg.norm(Ro)
    assert h3["res"][3] < h3["res"][0]
    assert h3["res"][0] == h1["res"][0]
    assert np.allclose(h3["res"][:2], h1["res"], rtol=1e-7, atol=0)    # same first step up to the solve error
    # the first update solves the oracle's Newton-step system (Eq. 5) to the solve tolerance
    rhs, blocks, dtau = dg.assemble(X, c.p, u0, c.mach, c.alpha_deg, c.cfl)
    assert abs(dtau - h1["dtau"][0]) <= 1e-12 * dtau
    A = dg.bsr_to_scipy(*blocks).tocsr()
    du = (u1.cpu().numpy() - u0).reshape(-1)
    assert np.linalg.norm(A @ du - rhs) <= 1e-8 * np.linalg.norm(rhs)
