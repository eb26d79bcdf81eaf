"""Pins for the pseudo-time continuation oracle (Sec. 2.1.2, Eqs. 5, 8, 9).

The march is pinned by what its limits must do, not by retyping it:
  * CFL -> infinity turns each step into Newton's method on R(u) = 0, so the
    residual must fall quadratically once it is small (a wrong Jacobian, a
    wrong sign of du or an inverted ramp gives linear convergence or none);
  * CFL -> 0 turns a step into explicit Euler in pseudo-time,
    du = -dtau M^-1 R + O(dtau^2) (pins the M/dtau term and the sign);
  * the steady state is a fixed point, and a uniform free stream (far field
    everywhere) is already steady;
  * the dense solve and the spaND-preconditioned s-step GMRES oracle give the
    same trajectory (library special case of the step's definition).
"""
import numpy as np
import pytest

from oracle import dg, gmres, march, spand
from synth import get_config, modal_state, naca_ogrid
from synth.state import uniform_modal_state


@pytest.fixture(scope="module")
def c1():
    c = get_config("C1")
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u0 = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
    return c, X, u0


def test_newton_limit_converges_quadratically(c1):
    c, X, u0 = c1
    u, h = march.march(X, c.p, u0, c.mach, c.alpha_deg, 1e4, 1e14, 12, rtol=1e-13)
    r = h["res"]
    assert r[-1] <= 1e-12 * r[0]
    # quadratic phase: r_{n+1} <= C r_n^2 for the steps that start below 1e-4 r_0 and end
    # above the round-off floor (a linear rate would need a contraction below 50 a)
    pairs = [(a, b) for a, b in zip(r[:-1], r[1:]) if a <= 1e-4 * r[0] and b > 1e-13]
    assert len(pairs) >= 1
    for a, b in pairs:
        assert b <= 50.0 * a * a, (a, b)
    # observed order log(r_{n+1}/r_n) / log(r_n/r_{n-1}) on the last steps above the floor
    q = r[r > 1e-13]
    order = np.log(q[-1] / q[-2]) / np.log(q[-2] / q[-3])
    assert order >= 1.5, order
    # CFL^1 = CFL^0 (Eq. 9 at n = 1) and the ramp grows while R falls
    assert h["cfl"][0] == h["cfl"][1] == 1e4
    assert np.all(np.diff(h["cfl"]) >= 0)


def test_steady_state_is_a_fixed_point(c1):
    c, X, u0 = c1
    u, h = march.march(X, c.p, u0, c.mach, c.alpha_deg, 1e4, 1e14, 12, rtol=1e-13)
    R = dg.residual(X, c.p, u, c.mach, c.alpha_deg)
    assert np.linalg.norm(R) <= 1e-12 * h["res"][0]
    u2, h2 = march.march(X, c.p, u, c.mach, c.alpha_deg, 1e4, 1e14, 2)
    assert np.max(np.abs(u2 - u)) <= 1e-12 * np.max(np.abs(u))


def test_small_cfl_is_explicit_euler(c1):
    c, X, u0 = c1
    for cfl in (1e-4, 1e-5):
        u1, h = march.march(X, c.p, u0, c.mach, c.alpha_deg, cfl, cfl, 1)
        dtau = h["dtau"][0]
        Mk = dg.mass_blocks(X, c.p)
        R = dg.residual(X, c.p, u0, c.mach, c.alpha_deg)
        expl = -dtau * np.linalg.solve(Mk, R)          # per element, each of the 4 variables
        du = u1 - u0
        err = np.linalg.norm(du - expl) / np.linalg.norm(expl)
        # the O(dtau) term: relative error shrinks in proportion to dtau
        assert err <= 5e3 * dtau, (cfl, dtau, err)


def test_free_stream_is_steady():
    c = get_config("C1")
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u0 = uniform_modal_state(c.n_theta * c.n_r, c.p, c.mach, c.alpha_deg)
    u, h = march.march(X, c.p, u0, c.mach, c.alpha_deg, 10.0, 1e6, 3, bc_mode="farfield")
    assert h["res"][0] <= 1e-12
    assert np.max(np.abs(u - u0)) <= 1e-12


def test_spand_gmres_solver_matches_dense(c1):
    c, X, u0 = c1

    def solver(rhs, blocks):
        F = spand.factor(blocks, c.n_theta, c.n_r, c.nd_depth, c.eps)
        A = dg.bsr_to_scipy(*blocks).tocsr()
        x, st = gmres.sstep_gmres(lambda v: A @ v, lambda v: spand.apply(F, v), rhs, s=c.s,
                                  restart=c.restart, tol=1e-13)
        assert st.converged
        return x

    ua, ha = march.march(X, c.p, u0, c.mach, c.alpha_deg, 100.0, 1e6, 3)
    ub, hb = march.march(X, c.p, u0, c.mach, c.alpha_deg, 100.0, 1e6, 3, solver=solver)
    assert np.allclose(ha["res"], hb["res"], rtol=1e-9, atol=0)
    assert np.max(np.abs(ua - ub)) <= 1e-9 * np.max(np.abs(ua))
