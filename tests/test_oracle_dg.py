"""Pins for the DG oracle (Sec. 2.1.2, Eqs. 3-8) against closed forms and invariants."""
import numpy as np
import pytest

from oracle import dg
from synth import get_config, modal_state, naca_ogrid, uniform_modal_state


def _annulus(n_theta, n_r, r0=1.0, r1=3.0):
    """Exact ring grid (clockwise j, outward i) for closed-form geometry checks."""
    th = -2 * np.pi * np.arange(n_theta) / n_theta
    r = np.linspace(r0, r1, n_r + 1)
    X = np.stack([r[:, None] * np.cos(th)[None, :], r[:, None] * np.sin(th)[None, :]], -1)
    return X


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_gauss_exact_on_monomials(q):
    t, w = dg.gauss(q)
    for d in range(2 * q):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(w @ t ** d - exact) < 1e-14
    d = 2 * q
    assert abs(w @ t ** d - 2.0 / (d + 1)) > 1e-6      # degree 2q is not exact


@pytest.mark.parametrize("p", [1, 2, 3])
def test_basis_orthonormal(p):
    # closed form: int_[-1,1]^2 psi_i psi_j = delta_ij (rule with 8 points is exact here)
    t, w = np.polynomial.legendre.leggauss(8)
    xi, eta = np.meshgrid(t, t, indexing="xy")
    W = np.outer(w, w).ravel()
    psi, _, _ = dg.basis2d(p, xi.ravel(), eta.ravel())
    G = psi.T @ (W[:, None] * psi)
    assert np.allclose(G, np.eye((p + 1) ** 2), atol=1e-13)
    # mode index m = b*(p+1) + a: mode 1 is linear in xi only
    assert np.allclose(psi[:, 1], np.sqrt(1.5) * xi.ravel() / np.sqrt(2.0))


def test_mass_affine_is_det_identity():
    # parallelogram element: constant |J|, so M = |J| I (orthonormal basis)
    p = 2
    X = _annulus(8, 2)
    X[:] = 0.0
    # build a 2x8 grid of identical parallelograms by shearing a regular lattice
    for i in range(3):
        for j in range(8):
            X[i, j] = np.array([0.7 * i + 0.2 * (-j), 0.5 * (-j) + 0.1 * i])
    M = dg.mass_blocks(X, p)
    a = X[0, 1] - X[0, 0]
    b = X[1, 0] - X[0, 0]
    detJ = abs(a[0] * b[1] - a[1] * b[0]) / 4.0
    for k in range(7):                       # skip the wrapped column j = 7 -> 0
        assert np.allclose(M[k], detJ * np.eye(9), atol=1e-13)


def test_freestream_preservation():
    c = get_config("C1")
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u0 = uniform_modal_state(c.K, c.p, c.mach, c.alpha_deg)
    R = dg.residual(X, c.p, u0, c.mach, c.alpha_deg, bc_mode="farfield")
    assert np.abs(R).max() <= 1e-12
    R = dg.residual(X, c.p, u0, c.mach, c.alpha_deg, bc_mode="wall")
    rows = np.nonzero(np.abs(R).max(axis=(1, 2)) > 1e-12)[0] // c.n_theta
    assert set(rows.tolist()) == {0}             # only wall-adjacent elements


def test_rusanov_consistency_and_symmetry():
    rng = np.random.default_rng(3)
    U = np.array([1.1, 0.4, -0.2, 2.6]) + 0.05 * rng.standard_normal((7, 4))
    th = rng.uniform(0, 2 * np.pi, 7)
    nx, ny = np.cos(th), np.sin(th)
    F, _, _ = dg.rusanov(U, U, nx, ny)
    Fx, Fy = dg.flux(U)
    assert np.allclose(F, Fx * nx[:, None] + Fy * ny[:, None], atol=1e-14)
    V = U[::-1].copy()
    Fa, _, _ = dg.rusanov(U, V, nx, ny)
    Fb, _, _ = dg.rusanov(V, U, -nx, -ny)
    assert np.allclose(Fa, -Fb, atol=1e-14)      # conservation across a face


def test_flux_jacobian_fd():
    rng = np.random.default_rng(5)
    U = np.array([1.2, 0.5, 0.1, 2.8])
    nx, ny = 0.6, 0.8
    A = dg.flux_normal_jacobian(U[None], np.array([nx]), np.array([ny]))[0]
    for w in range(4):
        h = 1e-6
        Up, Um = U.copy(), U.copy()
        Up[w] += h
        Um[w] -= h
        fp = dg.flux(Up)[0] * nx + dg.flux(Up)[1] * ny
        fm = dg.flux(Um)[0] * nx + dg.flux(Um)[1] * ny
        assert np.allclose(A[:, w], (fp - fm) / (2 * h), rtol=1e-8, atol=1e-9)
    del rng


def test_mode0_residual_telescopes_to_boundary_flux():
    # R_{k,0} = 1/2 oint F*.n (grad psi_0 = 0); interior faces cancel in the sum
    c = get_config("C1")
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
    R = dg.residual(X, c.p, u, c.mach, c.alpha_deg, bc_mode="farfield")
    tot = R[:, 0, :].sum(axis=0)
    # independent boundary integral: outer and airfoil rings, far-field ghost
    t, w = np.polynomial.legendre.leggauss(c.p + 2)
    Uinf = dg.freestream(c.mach, c.alpha_deg)
    n_r, nt = c.n_r, c.n_theta
    acc = np.zeros(4)
    for ring, i_el, eta, outward_sign in ((n_r, n_r - 1, 1.0, 1.0), (0, 0, -1.0, -1.0)):
        for j in range(nt):
            a, b = X[ring, j], X[ring, (j + 1) % nt]
            tv = b - a
            n = outward_sign * np.array([-tv[1], tv[0]]) / np.linalg.norm(tv)
            psi = dg.basis2d(c.p, t, np.full_like(t, eta))[0]
            UL = psi @ u[i_el * nt + j]
            F, _, _ = dg.rusanov(UL, np.tile(Uinf, (len(t), 1)), np.full(len(t), n[0]), np.full(len(t), n[1]))
            acc += 0.5 * np.linalg.norm(tv) / 2 * (w @ F)
    assert np.allclose(tot, acc, rtol=1e-11, atol=1e-12)


def test_pseudo_time_step_closed_form():
    p, cfl = 2, 10.0
    X = _annulus(8, 3)
    u0 = uniform_modal_state(24, p, 0.5, 2.0)
    dt = dg.pseudo_time_step(X, p, u0, cfl)
    U = dg.freestream(0.5, 2.0)
    speed = np.hypot(U[1], U[2]) / U[0] + 1.0       # |v| + c with c_inf = 1
    C = dg.element_corners(X)
    area = 0.5 * np.abs(sum(C[:, a, 0] * C[:, (a + 1) % 4, 1] - C[:, (a + 1) % 4, 0] * C[:, a, 1]
                            for a in range(4)))      # shoelace = bilinear quad area
    perim = sum(np.linalg.norm(C[:, (a + 1) % 4] - C[:, a], axis=-1) for a in range(4))
    assert np.isclose(dt, np.min(cfl / (speed * (2 * p + 1) * perim / area)), rtol=1e-12)


def _fd_check(X, p, u, mach, alpha, cols, bc="wall"):
    rhs, bsr, dtau = dg.assemble(X, p, u, mach, alpha, 10.0, bc_mode=bc)
    J = dg.bsr_to_dense(*bsr)
    B = 4 * (p + 1) ** 2
    M = dg.mass_blocks(X, p)
    for k in range(M.shape[0]):
        J[k * B:(k + 1) * B, k * B:(k + 1) * B] -= np.kron(M[k], np.eye(4)) / dtau
    uf = u.reshape(-1)
    worst = 0.0
    for jc in cols:
        h = 1e-7 * max(1.0, abs(uf[jc]))
        up, um = uf.copy(), uf.copy()
        up[jc] += h
        um[jc] -= h
        fd = (dg.residual(X, p, up.reshape(u.shape), mach, alpha, bc).ravel()
              - dg.residual(X, p, um.reshape(u.shape), mach, alpha, bc).ravel()) / (2 * h)
        worst = max(worst, np.linalg.norm(J[:, jc] - fd) / np.linalg.norm(fd))
    return worst, rhs


def test_jacobian_fd_all_columns_tiny():
    X = naca_ogrid(6, 4, 11)
    u = modal_state(X, 1, 0.5, 2.0, 0.05, 11)
    worst, rhs = _fd_check(X, 1, u, 0.5, 2.0, range(u.size))
    assert worst <= 1e-6
    assert np.allclose(rhs, -dg.residual(X, 1, u, 0.5, 2.0).ravel())


def test_jacobian_fd_seeded_columns_c1():
    c = get_config("C1")
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
    cols = np.random.default_rng(c.seed).choice(u.size, 64, replace=False)
    worst, _ = _fd_check(X, c.p, u, c.mach, c.alpha_deg, cols)
    assert worst <= 1e-6


def test_jacobian_fd_p3_farfield():
    X = naca_ogrid(8, 4, 21)
    u = modal_state(X, 3, 0.8, 1.0, 0.1, 21)
    cols = np.random.default_rng(0).choice(u.size, 48, replace=False)
    worst, _ = _fd_check(X, 3, u, 0.8, 1.0, cols, bc="farfield")
    assert worst <= 1e-6


def test_bsr_pattern_counts():
    for nt, nr in ((16, 8), (64, 32)):
        rp, col = dg.bsr_pattern(nt, nr)
        assert rp[-1] == 5 * nt * nr - 2 * nt
        for r in range(nt * nr):
            assert list(col[rp[r]:rp[r + 1]]) == sorted(col[rp[r]:rp[r + 1]])
