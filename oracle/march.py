"""Pseudo-time continuation to the steady state (oracle; test infrastructure).

Sec. 2.1.2 of arXiv 2101.01763.  Pseudo-time step n (n = 0, 1, ...):
  * CFL number by the residual ratio (Eq. 9):
        CFL^n = min(CFL^0 ||R^0|| / ||R^{n-1}||, CFL^inf),   n >= 1,
    and CFL^0 itself at n = 0;
  * dtau^n = min_k CFL^n / lam_k (Eq. 8) and the Newton-step system
        (M/dtau^n + dR/du|^n) du = -R^n (Eq. 5);
  * u^{n+1} = u^n + du.
Readings (the paper gives the formulas only): ||.|| is the 2-norm of all
residual coefficients; the march stops before a solve once
||R^n|| <= rtol ||R^0|| or after max_steps solves; a zero ||R^{n-1}|| gives
CFL^inf.  The linear solve is the plain definition du = A^-1 (-R) (dense LU),
or the oracle's spaND-preconditioned s-step GMRES when `solver` asks for it.
"""
import numpy as np

from . import dg


def cfl_ramp(cfl0, cfl_inf, r0, r_prev):
    """CFL^n of Eq. 9 from ||R^0|| and ||R^{n-1}||."""
    if r_prev <= 0.0:
        return cfl_inf
    return min(cfl0 * r0 / r_prev, cfl_inf)


def _solve_dense(rhs, blocks):
    rp, col, val = blocks
    return np.linalg.solve(dg.bsr_to_dense(rp, col, val), rhs)


def march(X, p, uhat, mach, alpha_deg, cfl0, cfl_inf, max_steps, rtol=0.0, bc_mode="wall", solver=None):
    """Run the continuation from uhat [K, Np, 4].

    solver(rhs, (row_ptr, col, val)) -> du; default: dense solve.
    Returns (u [K, Np, 4], history) with history = dict(res [steps+1],
    cfl [steps+1], dtau [steps+1]): the residual norm, CFL number and dtau of
    every assembled state u^0 .. u^steps (the last state is assembled and
    not solved).
    """
    solve = solver or _solve_dense
    u = np.array(uhat, dtype=np.float64, copy=True)
    res, cfls, dts = [], [], []
    cfl = cfl0
    for n in range(max_steps + 1):
        rhs, blocks, dtau = dg.assemble(X, p, u, mach, alpha_deg, cfl, bc_mode)
        r = float(np.linalg.norm(rhs))
        res.append(r)
        cfls.append(cfl)
        dts.append(dtau)
        if n == max_steps or r <= rtol * res[0]:
            break
        du = solve(rhs, blocks)
        u = u + du.reshape(u.shape)
        cfl = cfl_ramp(cfl0, cfl_inf, res[0], r)
    return u, {"res": np.array(res), "cfl": np.array(cfls), "dtau": np.array(dts)}
