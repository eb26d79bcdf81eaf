"""Seeded modal DG states for the Euler workloads.

Format: u_hat[K, Np, 4] float64, Np = (p+1)^2, mode m = b*(p+1) + a for the
tensor Legendre mode of degree a in xi and b in eta, variables (rho, rho*u,
rho*v, E).  The constant mode of the orthonormal Legendre basis on [-1,1]^2 is
1/2, so a cell-average state U is stored as u_hat[k, 0] = 2*U.

Non-dimensionalisation: rho_inf = 1, p_inf = 1/gamma (so c_inf = 1) and
v_inf = M (cos alpha, sin alpha).
"""
import numpy as np

GAMMA = 1.4


def freestream_conserved(mach, alpha_deg, gamma=GAMMA):
    a = np.deg2rad(alpha_deg)
    rho, p = 1.0, 1.0 / gamma
    u, v = mach * np.cos(a), mach * np.sin(a)
    return np.array([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def uniform_modal_state(K, p, mach, alpha_deg, gamma=GAMMA):
    np_ = (p + 1) ** 2
    u = np.zeros((K, np_, 4))
    u[:, 0, :] = 2.0 * freestream_conserved(mach, alpha_deg, gamma)[None, :]
    return u


def _smooth_field(rng, xy, n_waves=4):
    k = rng.uniform(0.3, 3.0, size=n_waves)
    th = rng.uniform(0.0, 2.0 * np.pi, size=n_waves)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n_waves)
    a = rng.uniform(0.5, 1.0, size=n_waves)
    f = np.zeros(xy.shape[0])
    for t in range(n_waves):
        f += a[t] * np.sin(k[t] * (np.cos(th[t]) * xy[:, 0] + np.sin(th[t]) * xy[:, 1]) + ph[t])
    return f / a.sum()                                   # |f| <= 1


def modal_state(X, p, mach, alpha_deg, amp, seed, gamma=GAMMA):
    """Free stream with seeded smooth primitive perturbations of relative size amp.

    The element mean is the perturbed primitive state at the element centroid
    (four smooth seeded fields for rho, u, v, p); higher modes carry small seeded
    values (a tenth of amp, damped with the mode degree).
    """
    rng = np.random.default_rng(seed + 7919)
    n_r, n_theta = X.shape[0] - 1, X.shape[1]
    jp = np.roll(np.arange(n_theta), -1)
    cen = 0.25 * (X[:n_r, :, :] + X[:n_r, jp, :] + X[1:, jp, :] + X[1:, :, :]).reshape(-1, 2)
    K = cen.shape[0]
    a = np.deg2rad(alpha_deg)
    d = [_smooth_field(rng, cen) for _ in range(4)]
    rho = 1.0 * (1.0 + amp * d[0])
    u = mach * np.cos(a) * (1.0 + amp * d[1])
    v = mach * np.sin(a) + amp * mach * d[2]
    pr = (1.0 / gamma) * (1.0 + amp * d[3])
    E = pr / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    U = np.stack([rho, rho * u, rho * v, E], axis=1)
    np_ = (p + 1) ** 2
    uh = np.zeros((K, np_, 4))
    uh[:, 0, :] = 2.0 * U
    scale = np.array([1.0, mach, mach, 1.0 / (gamma - 1.0)])
    for m in range(1, np_):
        deg = m % (p + 1) + m // (p + 1)
        g = np.clip(rng.standard_normal((K, 4)), -2.0, 2.0)
        uh[:, m, :] = 2.0 * 0.1 * amp * scale[None, :] * g / (1.0 + deg)
    return uh
