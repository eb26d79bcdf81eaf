"""The five synthetic workloads (C1-C5) shaped like the paper's 2D airfoil runs.

The paper (Sec. 3.1, Table 1) runs a p=1 NACA0012 O-mesh at M=0.3, alpha=2 deg
with spaND eps=1e-3 and ~32-element leaves.  Here every workload is a seeded
synthetic O-grid of n_theta x n_r bilinear quads; the grid, state and solver
settings below stand in for the SU2 mesh and flow field, which are not
available.
"""
from dataclasses import dataclass, field, replace
import math


@dataclass(frozen=True)
class Config:
    name: str
    p: int              # polynomial degree of the tensor Legendre basis
    n_theta: int        # elements around the airfoil (periodic direction)
    n_r: int            # elements in the radial direction
    mach: float
    alpha_deg: float
    amp: float          # relative amplitude of the seeded perturbation
    cfl: float
    eps: float          # spaND truncation tolerance
    s: int              # s-step block size
    restart: int        # basis vectors per GMRES cycle
    tol: float          # relative residual target
    seed: int
    max_iters: int = 600
    extra: dict = field(default_factory=dict)

    @property
    def K(self):
        return self.n_theta * self.n_r

    @property
    def B(self):
        return 4 * (self.p + 1) ** 2

    @property
    def N(self):
        return self.K * self.B

    @property
    def nd_depth(self):
        """D = ceil(log2(K/32)): leaves of about 32 elements (Table 1 ratio)."""
        return max(1, int(math.ceil(math.log2(self.K / 32.0))))

    @property
    def levels(self):
        return self.nd_depth + 1

    def with_(self, **kw):
        return replace(self, **kw)


CONFIGS = {
    "C1": Config("C1", p=1, n_theta=16, n_r=8, mach=0.5, alpha_deg=2.0, amp=0.05,
                 cfl=10.0, eps=1e-2, s=4, restart=40, tol=1e-8, seed=2101_0001),
    "C2": Config("C2", p=2, n_theta=64, n_r=32, mach=0.5, alpha_deg=2.0, amp=0.05,
                 cfl=10.0, eps=1e-3, s=4, restart=60, tol=1e-8, seed=2101_0002),
    "C3": Config("C3", p=3, n_theta=256, n_r=128, mach=0.8, alpha_deg=2.0, amp=0.10,
                 cfl=10.0, eps=1e-3, s=8, restart=80, tol=1e-8, seed=2101_0003),
    "C4": Config("C4", p=2, n_theta=128, n_r=64, mach=0.5, alpha_deg=2.0, amp=0.05,
                 cfl=10.0, eps=1e-3, s=4, restart=60, tol=1e-8, seed=2101_0004),
}


def get_config(name):
    return CONFIGS[name]


def batch_configs(n=24, seed=2101_0500):
    """C5: independent systems with grids, degrees and flow angles drawn per system."""
    import numpy as np
    grids = [(32, 16), (64, 32), (96, 48), (192, 96)]
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed + i)
        nt, nr = grids[int(rng.integers(0, len(grids)))]
        p = int(rng.integers(1, 4))
        out.append(Config(f"C5_{i}", p=p, n_theta=nt, n_r=nr,
                          mach=float(rng.uniform(0.3, 0.8)),
                          alpha_deg=float(rng.uniform(0.0, 4.0)), amp=0.05,
                          cfl=10.0, eps=1e-3, s=4, restart=60, tol=1e-8, seed=seed + i))
    return out
