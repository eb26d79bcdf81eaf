"""Seeded O-grid around a closed NACA-4-digit thickness curve.

Node (i, j): i = 0..n_r is the radial layer (0 = airfoil, n_r = outer circle of
radius 20 chords), j = 0..n_theta-1 runs clockwise around the airfoil starting
at the trailing edge (periodic).  Element (i, j), i < n_r, has corners
(i,j), (i,j+1), (i+1,j+1), (i+1,j) and index e = i*n_theta + j, the (i, j)
integer mapping of Sec. 3.3.  With j clockwise and i outward the bilinear map
of every element has a positive Jacobian determinant (checked here).
"""
import numpy as np


def _naca_thickness(x, t=0.12):
    # closed-trailing-edge NACA 4-digit half thickness
    return 5.0 * t * (0.2969 * np.sqrt(np.maximum(x, 0.0)) - 0.1260 * x - 0.3516 * x ** 2
                      + 0.2843 * x ** 3 - 0.1036 * x ** 4)


def naca_ogrid(n_theta, n_r, seed, thickness=0.12, radius=20.0, jitter=0.10):
    """Return nodes [n_r+1, n_theta, 2] (float64)."""
    rng = np.random.default_rng(seed)
    phi = 2.0 * np.pi * np.arange(n_theta) / n_theta
    xa = 0.5 * (1.0 + np.cos(phi))                     # cosine clustering at LE/TE
    ya = -np.sign(np.sin(phi)) * _naca_thickness(xa, thickness)
    ya[np.abs(np.sin(phi)) < 1e-14] = 0.0
    center = np.array([0.5, 0.0])
    xo = center[0] + radius * np.cos(phi)
    yo = center[1] - radius * np.sin(phi)
    g = 1.0 + 4.0 / n_r                                # geometric radial stretching
    s = (g ** np.arange(n_r + 1) - 1.0) / (g ** n_r - 1.0)
    X = np.empty((n_r + 1, n_theta, 2))
    X[:, :, 0] = xa[None, :] + s[:, None] * (xo - xa)[None, :]
    X[:, :, 1] = ya[None, :] + s[:, None] * (yo - ya)[None, :]
    # seeded jitter of interior nodes: +-jitter x the shortest adjacent edge
    if jitter > 0 and n_r > 1:
        Xi = X[1:n_r]
        d_r = np.minimum(np.linalg.norm(X[2:] - X[1:-1], axis=-1),
                         np.linalg.norm(X[1:-1] - X[:-2], axis=-1))
        d_t = np.minimum(np.linalg.norm(np.roll(Xi, -1, axis=1) - Xi, axis=-1),
                         np.linalg.norm(np.roll(Xi, 1, axis=1) - Xi, axis=-1))
        h = np.minimum(d_r, d_t)
        off = rng.uniform(-1.0, 1.0, size=Xi.shape) * (jitter * h)[..., None]
        X[1:n_r] = Xi + off
    _check_positive(X)
    return X


def element_corners(X):
    """Corners [K, 4, 2] in the order (i,j), (i,j+1), (i+1,j+1), (i+1,j)."""
    n_r = X.shape[0] - 1
    jp = np.roll(np.arange(X.shape[1]), -1)
    c0 = X[:n_r, :, :]
    c1 = X[:n_r, jp, :]
    c2 = X[1:, jp, :]
    c3 = X[1:, :, :]
    return np.stack([c0, c1, c2, c3], axis=2).reshape(-1, 4, 2)


def _check_positive(X):
    C = element_corners(X)

    def cross(a, b):
        return a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]

    # the Jacobian determinant of a bilinear map is affine in (xi, eta) separately;
    # positive at the four corners => positive on the element
    dets = (cross(C[:, 1] - C[:, 0], C[:, 3] - C[:, 0]),
            cross(C[:, 1] - C[:, 0], C[:, 2] - C[:, 1]),
            cross(C[:, 2] - C[:, 3], C[:, 2] - C[:, 1]),
            cross(C[:, 2] - C[:, 3], C[:, 3] - C[:, 0]))
    if not all(np.all(d > 0) for d in dets):
        raise ValueError("O-grid has a non-positive element Jacobian")
