"""Modal DG discretisation of 2D Euler and the Newton-step system (oracle).

Follows Sec. 2.1.2 of arXiv 2101.01763:
  * Eq. 3: u = sum_i u_hat_i psi_i with a modal basis; here the tensor
    orthonormal Legendre basis psi_m(xi, eta) = P~_a(xi) P~_b(eta),
    m = b*(p+1) + a, P~_a = sqrt((2a+1)/2) P_a.
  * Eq. 7 (residual, sign as printed):
        R_i = - int_D F(u) . grad psi_i dV + oint_dD F*(u) . n psi_i dA
    with the Rusanov numerical flux F*.n = (F(uL)+F(uR)).n/2 - lam (uR-uL)/2,
    lam = max(|vL.n| + cL, |vR.n| + cR).  (The paper's flux is Roe; the workload
    fixes Rusanov.)
  * Eq. 6: M = int psi_i psi_j dV (times I_4).
  * Eq. 8: dtau = min_k CFL / lam_k with
        lam_k = max_{quad pts}(|v| + c) * (2p+1) * |dD_k| / |D_k|.
  * Eq. 5: A = M/dtau + dR/du, b = -R.  dR/du is the exact derivative of the
    discrete R (the paper uses AD); here it is derived by hand, with the
    branch of the max taken on the L side on ties and d|x|/dx = +1 at x = 0.

Quadrature: Gauss-Legendre, q = p+2 points per direction in the volume and
on edges (exact for the mass matrix and for the free-stream identity on
bilinear quads).  Boundary conditions: far field (ghost = free stream) on the
outer ring; slip wall (ghost with reflected normal momentum) on the airfoil,
or far field there too with bc_mode = "farfield".

DOF index inside element e: m*4 + v.  Output A is block-CSR with blocks
val[k, r, c] (row-major inside a block), row_ptr [K+1], col [nnzb] ascending.
"""
import numpy as np
from numpy.polynomial import legendre as npleg

GAMMA = 1.4


# ----------------------------------------------------------------- basis / quadrature
def gauss(q):
    return npleg.leggauss(q)


def legendre_orthonormal(p, t):
    """Values and derivatives [len(t), p+1] of sqrt((2a+1)/2) P_a(t)."""
    t = np.asarray(t, dtype=float)
    V = np.zeros((t.size, p + 1))
    D = np.zeros((t.size, p + 1))
    for a in range(p + 1):
        c = np.zeros(a + 1)
        c[a] = np.sqrt((2 * a + 1) / 2.0)
        V[:, a] = npleg.legval(t, c)
        D[:, a] = npleg.legval(t, npleg.legder(c)) if a > 0 else 0.0
    return V, D


def basis2d(p, xi, eta):
    """psi, dpsi/dxi, dpsi/deta at points (xi[k], eta[k]) -> [npts, Np]."""
    Vx, Dx = legendre_orthonormal(p, xi)
    Ve, De = legendre_orthonormal(p, eta)
    np_ = (p + 1) ** 2
    psi = np.zeros((len(xi), np_))
    pxi = np.zeros_like(psi)
    peta = np.zeros_like(psi)
    for b in range(p + 1):
        for a in range(p + 1):
            m = b * (p + 1) + a
            psi[:, m] = Vx[:, a] * Ve[:, b]
            pxi[:, m] = Dx[:, a] * Ve[:, b]
            peta[:, m] = Vx[:, a] * De[:, b]
    return psi, pxi, peta


def volume_points(p):
    t, w = gauss(p + 2)
    xi = np.tile(t, len(t))          # xi fastest
    eta = np.repeat(t, len(t))
    W = np.tile(w, len(w)) * np.repeat(w, len(w))
    return xi, eta, W


# ----------------------------------------------------------------- geometry
def element_corners(X):
    n_r = X.shape[0] - 1
    jp = np.roll(np.arange(X.shape[1]), -1)
    return np.stack([X[:n_r], X[:n_r, jp], X[1:, jp], X[1:]], axis=2).reshape(-1, 4, 2)


def bilinear_derivs(C, xi, eta):
    """dx/dxi, dx/deta [K, npts, 2] of the bilinear map through corners C[K,4,2]."""
    xi = xi[None, :, None]
    eta = eta[None, :, None]
    c0, c1, c2, c3 = (C[:, i, None, :] for i in range(4))
    dxi = 0.25 * (-(1 - eta) * c0 + (1 - eta) * c1 + (1 + eta) * c2 - (1 + eta) * c3)
    deta = 0.25 * (-(1 - xi) * c0 - (1 + xi) * c1 + (1 + xi) * c2 + (1 - xi) * c3)
    return dxi, deta


# ----------------------------------------------------------------- Euler physics
def primitives(U, gamma=GAMMA):
    rho = U[..., 0]
    ux = U[..., 1] / rho
    uy = U[..., 2] / rho
    p = (gamma - 1.0) * (U[..., 3] - 0.5 * rho * (ux * ux + uy * uy))
    return rho, ux, uy, p


def flux(U, gamma=GAMMA):
    rho, ux, uy, p = primitives(U, gamma)
    E = U[..., 3]
    Fx = np.stack([rho * ux, rho * ux * ux + p, rho * ux * uy, (E + p) * ux], axis=-1)
    Fy = np.stack([rho * uy, rho * ux * uy, rho * uy * uy + p, (E + p) * uy], axis=-1)
    return Fx, Fy


def flux_normal_jacobian(U, nx, ny, gamma=GAMMA):
    """d(F.n)/dU [..., 4, 4] for the Euler flux."""
    rho, ux, uy, p = primitives(U, gamma)
    E = U[..., 3]
    g1 = gamma - 1.0
    vn = ux * nx + uy * ny
    phi = 0.5 * g1 * (ux * ux + uy * uy)
    H = (E + p) / rho
    z = np.zeros_like(rho)
    one = np.ones_like(rho)
    A = np.stack([
        np.stack([z, nx * one, ny * one, z], -1),
        np.stack([phi * nx - ux * vn, vn + ux * nx - g1 * ux * nx, ux * ny - g1 * uy * nx, g1 * nx * one], -1),
        np.stack([phi * ny - uy * vn, uy * nx - g1 * ux * ny, vn + uy * ny - g1 * uy * ny, g1 * ny * one], -1),
        np.stack([vn * (phi - H), H * nx - g1 * ux * vn, H * ny - g1 * uy * vn, gamma * vn], -1),
    ], -2)
    return A


def wave_speed(U, nx, ny, gamma=GAMMA):
    """a = |v.n| + c and da/dU."""
    rho, ux, uy, p = primitives(U, gamma)
    c = np.sqrt(gamma * p / rho)
    vn = ux * nx + uy * ny
    sg = np.where(vn >= 0.0, 1.0, -1.0)
    dvn = np.stack([-vn / rho, nx / rho * np.ones_like(rho), ny / rho * np.ones_like(rho), np.zeros_like(rho)], -1)
    g1 = gamma - 1.0
    dp = np.stack([0.5 * g1 * (ux * ux + uy * uy), -g1 * ux, -g1 * uy, g1 * np.ones_like(rho)], -1)
    drho = np.zeros(dp.shape)
    drho[..., 0] = 1.0
    dc = (gamma / (2.0 * c * rho))[..., None] * dp - (c / (2.0 * rho))[..., None] * drho
    return np.abs(vn) + c, sg[..., None] * dvn + dc


def rusanov(UL, UR, nx, ny, gamma=GAMMA):
    """F*.n and its derivatives with respect to UL and UR ([..., 4, 4])."""
    FxL, FyL = flux(UL, gamma)
    FxR, FyR = flux(UR, gamma)
    FnL = FxL * nx[..., None] + FyL * ny[..., None]
    FnR = FxR * nx[..., None] + FyR * ny[..., None]
    aL, daL = wave_speed(UL, nx, ny, gamma)
    aR, daR = wave_speed(UR, nx, ny, gamma)
    takeL = aL >= aR
    lam = np.where(takeL, aL, aR)
    dU = UR - UL
    F = 0.5 * (FnL + FnR) - 0.5 * lam[..., None] * dU
    I4 = np.eye(4)
    dlamL = np.where(takeL[..., None], daL, 0.0)
    dlamR = np.where(takeL[..., None], 0.0, daR)
    dFL = 0.5 * flux_normal_jacobian(UL, nx, ny, gamma) + 0.5 * lam[..., None, None] * I4 \
        - 0.5 * dU[..., :, None] * dlamL[..., None, :]
    dFR = 0.5 * flux_normal_jacobian(UR, nx, ny, gamma) - 0.5 * lam[..., None, None] * I4 \
        - 0.5 * dU[..., :, None] * dlamR[..., None, :]
    return F, dFL, dFR


def freestream(mach, alpha_deg, gamma=GAMMA):
    a = np.deg2rad(alpha_deg)
    u, v = mach * np.cos(a), mach * np.sin(a)
    p = 1.0 / gamma
    return np.array([1.0, u, v, p / (gamma - 1.0) + 0.5 * (u * u + v * v)])


# ----------------------------------------------------------------- faces
def _faces(X):
    """Face lists: (L, R or -1, L local face, R local face, nx, ny, half length, kind).

    Local faces: 0 = east (xi=+1), 1 = west (xi=-1), 2 = north (eta=+1), 3 = south (eta=-1).
    kind: 0 interior, 1 airfoil boundary, 2 outer boundary.
    """
    n_r, n_t = X.shape[0] - 1, X.shape[1]
    out = []
    i, j = np.meshgrid(np.arange(n_r), np.arange(n_t), indexing="ij")
    i, j = i.ravel(), j.ravel()
    jp = (j + 1) % n_t
    # angular faces: L=(i,j) east, R=(i,j+1) west; edge X[i,j+1] -> X[i+1,j+1]
    t = X[i + 1, jp] - X[i, jp]
    out.append((i * n_t + j, i * n_t + jp, 0, 1, t[:, 1], -t[:, 0], 0))
    # radial faces: L=(i,j) north, R=(i+1,j) south; edge X[i+1,j] -> X[i+1,j+1]
    sel = i < n_r - 1
    ii, jj, jjp = i[sel], j[sel], jp[sel]
    t = X[ii + 1, jjp] - X[ii + 1, jj]
    out.append((ii * n_t + jj, (ii + 1) * n_t + jj, 2, 3, -t[:, 1], t[:, 0], 0))
    # airfoil: (0,j) south; edge X[0,j] -> X[0,j+1]
    jj = np.arange(n_t)
    t = X[0, (jj + 1) % n_t] - X[0, jj]
    out.append((jj, -np.ones_like(jj), 3, -1, t[:, 1], -t[:, 0], 1))
    # outer: (n_r-1, j) north; edge X[n_r,j] -> X[n_r,j+1]
    t = X[n_r, (jj + 1) % n_t] - X[n_r, jj]
    out.append(((n_r - 1) * n_t + jj, -np.ones_like(jj), 2, -1, -t[:, 1], t[:, 0], 2))
    faces = []
    for L, R, fl, fr, nx, ny, kind in out:
        ln = np.hypot(nx, ny)
        faces.append(dict(L=L, R=R, fl=fl, fr=fr, nx=nx / ln, ny=ny / ln, hl=0.5 * ln, kind=kind))
    return faces


def face_basis(p, face, t):
    one = np.ones_like(t)
    if face == 0:
        return basis2d(p, one, t)[0]
    if face == 1:
        return basis2d(p, -one, t)[0]
    if face == 2:
        return basis2d(p, t, one)[0]
    return basis2d(p, t, -one)[0]


# ----------------------------------------------------------------- residual + Jacobian
def _evaluate(X, p, uhat, mach, alpha_deg, bc_mode, want_jac, gamma=GAMMA):
    K = uhat.shape[0]
    np_ = (p + 1) ** 2
    C = element_corners(X)
    xi, eta, W = volume_points(p)
    psi, pxi, peta = basis2d(p, xi, eta)
    dxi, deta = bilinear_derivs(C, xi, eta)
    det = dxi[..., 0] * deta[..., 1] - deta[..., 0] * dxi[..., 1]
    # det * grad psi
    Gx = deta[..., 1, None] * pxi[None] - dxi[..., 1, None] * peta[None]
    Gy = -deta[..., 0, None] * pxi[None] + dxi[..., 0, None] * peta[None]
    U = np.einsum("qm,kmv->kqv", psi, uhat)
    Fx, Fy = flux(U, gamma)
    R = -np.einsum("q,kqm,kqv->kmv", W, Gx, Fx) - np.einsum("q,kqm,kqv->kmv", W, Gy, Fy)
    blocks = []   # (row element, col element, [F, Np,4, Np,4])
    if want_jac:
        Ax = flux_normal_jacobian(U, np.ones(U.shape[:2]), np.zeros(U.shape[:2]), gamma)
        Ay = flux_normal_jacobian(U, np.zeros(U.shape[:2]), np.ones(U.shape[:2]), gamma)
        Jv = -np.einsum("q,kqi,kqvw,qj->kivjw", W, Gx, Ax, psi) \
            - np.einsum("q,kqi,kqvw,qj->kivjw", W, Gy, Ay, psi)
        blocks.append((np.arange(K), np.arange(K), Jv))
    te, we = gauss(p + 2)
    Uinf = freestream(mach, alpha_deg, gamma)
    for f in _faces(X):
        L, Rr = f["L"], f["R"]
        psiL = face_basis(p, f["fl"], te)
        UL = np.einsum("qm,fmv->fqv", psiL, uhat[L])
        nx = np.repeat(f["nx"][:, None], len(te), 1)
        ny = np.repeat(f["ny"][:, None], len(te), 1)
        wall = f["kind"] == 1 and bc_mode == "wall"
        if f["kind"] == 0:
            psiR = face_basis(p, f["fr"], te)
            UR = np.einsum("qm,fmv->fqv", psiR, uhat[Rr])
        elif wall:
            Wm = np.zeros(UL.shape[:2] + (4, 4))
            Wm[..., 0, 0] = 1.0
            Wm[..., 3, 3] = 1.0
            Wm[..., 1, 1] = 1.0 - 2.0 * nx * nx
            Wm[..., 1, 2] = -2.0 * nx * ny
            Wm[..., 2, 1] = -2.0 * nx * ny
            Wm[..., 2, 2] = 1.0 - 2.0 * ny * ny
            UR = np.einsum("fqvw,fqw->fqv", Wm, UL)
        else:
            UR = np.broadcast_to(Uinf, UL.shape).copy()
        Fs, dFL, dFR = rusanov(UL, UR, nx, ny, gamma)
        hw = f["hl"][:, None] * we[None, :]
        np.add.at(R, L, np.einsum("fq,qm,fqv->fmv", hw, psiL, Fs))
        if f["kind"] == 0:
            np.add.at(R, Rr, -np.einsum("fq,qm,fqv->fmv", hw, psiR, Fs))
        if want_jac:
            if wall:
                dFL = dFL + np.einsum("fqvu,fquw->fqvw", dFR, Wm)
            blocks.append((L, L, np.einsum("fq,qi,fqvw,qj->fivjw", hw, psiL, dFL, psiL)))
            if f["kind"] == 0:
                blocks.append((L, Rr, np.einsum("fq,qi,fqvw,qj->fivjw", hw, psiL, dFR, psiR)))
                blocks.append((Rr, L, -np.einsum("fq,qi,fqvw,qj->fivjw", hw, psiR, dFL, psiL)))
                blocks.append((Rr, Rr, -np.einsum("fq,qi,fqvw,qj->fivjw", hw, psiR, dFR, psiR)))
    out = dict(R=R, blocks=blocks, det=det, W=W, psi=psi, U=U, C=C)
    return out


def residual(X, p, uhat, mach, alpha_deg, bc_mode="wall", gamma=GAMMA):
    """R [K, Np, 4] (Eq. 7)."""
    return _evaluate(X, p, uhat, mach, alpha_deg, bc_mode, False, gamma)["R"]


def mass_blocks(X, p):
    """M_k [K, Np, Np] = int psi_i psi_j |J| (Eq. 6), without the I_4 factor."""
    C = element_corners(X)
    xi, eta, W = volume_points(p)
    psi, _, _ = basis2d(p, xi, eta)
    dxi, deta = bilinear_derivs(C, xi, eta)
    det = dxi[..., 0] * deta[..., 1] - deta[..., 0] * dxi[..., 1]
    return np.einsum("q,kq,qi,qj->kij", W, det, psi, psi)


def pseudo_time_step(X, p, uhat, cfl, gamma=GAMMA):
    """dtau = min_k CFL/lam_k (Eq. 8), lam_k = max(|v|+c) (2p+1) |dD_k|/|D_k|."""
    C = element_corners(X)
    xi, eta, W = volume_points(p)
    psi, _, _ = basis2d(p, xi, eta)
    dxi, deta = bilinear_derivs(C, xi, eta)
    det = dxi[..., 0] * deta[..., 1] - deta[..., 0] * dxi[..., 1]
    area = det @ W
    perim = sum(np.linalg.norm(C[:, (a + 1) % 4] - C[:, a], axis=-1) for a in range(4))
    U = np.einsum("qm,kmv->kqv", psi, uhat)
    rho, ux, uy, pr = primitives(U, gamma)
    smax = np.max(np.sqrt(ux * ux + uy * uy) + np.sqrt(gamma * pr / rho), axis=1)
    lam = smax * (2 * p + 1) * perim / area
    return float(np.min(cfl / lam))


def bsr_pattern(n_theta, n_r):
    """row_ptr [K+1], col [nnzb]: each element with its face neighbours, ascending."""
    K = n_theta * n_r
    rows = []
    for e in range(K):
        i, j = divmod(e, n_theta)
        nb = {e, i * n_theta + (j + 1) % n_theta, i * n_theta + (j - 1) % n_theta}
        if i > 0:
            nb.add(e - n_theta)
        if i < n_r - 1:
            nb.add(e + n_theta)
        rows.append(sorted(nb))
    row_ptr = np.zeros(K + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c in r], dtype=np.int32)
    return row_ptr, col


def assemble(X, p, uhat, mach, alpha_deg, cfl, bc_mode="wall", gamma=GAMMA):
    """Return rhs [N], (row_ptr, col, val[nnzb,B,B]) and dtau for A = M/dtau + dR/du (Eq. 5)."""
    n_r, n_t = X.shape[0] - 1, X.shape[1]
    K = n_r * n_t
    np_ = (p + 1) ** 2
    B = 4 * np_
    ev = _evaluate(X, p, uhat, mach, alpha_deg, bc_mode, True, gamma)
    dtau = pseudo_time_step(X, p, uhat, cfl, gamma)
    row_ptr, col = bsr_pattern(n_t, n_r)
    keys = np.repeat(np.arange(K), np.diff(row_ptr)).astype(np.int64) * K + col
    val = np.zeros((len(col), B, B))
    for r, c, blk in ev["blocks"]:
        pos = np.searchsorted(keys, r.astype(np.int64) * K + c)
        assert np.all(keys[pos] == r.astype(np.int64) * K + c)
        np.add.at(val, pos, blk.reshape(-1, B, B))
    Mk = mass_blocks(X, p)
    diag = np.searchsorted(keys, np.arange(K, dtype=np.int64) * (K + 1))
    val[diag] += np.einsum("kij,vw->kivjw", Mk, np.eye(4)).reshape(K, B, B) / dtau
    rhs = -ev["R"].reshape(-1)
    return rhs, (row_ptr, col, val), dtau


def bsr_to_dense(row_ptr, col, val):
    K = len(row_ptr) - 1
    B = val.shape[1]
    A = np.zeros((K * B, K * B))
    for r in range(K):
        for k in range(row_ptr[r], row_ptr[r + 1]):
            A[r * B:(r + 1) * B, col[k] * B:(col[k] + 1) * B] = val[k]
    return A


def bsr_to_scipy(row_ptr, col, val):
    import scipy.sparse as sp
    K = len(row_ptr) - 1
    B = val.shape[1]
    return sp.bsr_matrix((val, col, row_ptr), shape=(K * B, K * B))
