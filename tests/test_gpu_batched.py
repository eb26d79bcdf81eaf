"""Batched factorization and solve of independent systems (grids, degrees and
flow angles differ per system) against the one-system path and the dense
solve.

The batched factorization runs each level's phases as one launch over all
systems; per cluster it does the same arithmetic as the one-system path, so
ranks must agree exactly and applies to rounding.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dg  # noqa: E402
from synth import modal_state, naca_ogrid  # noqa: E402

# (n_theta, n_r, p, mach, alpha): depths 2..4, block sizes 16 / 36 / 64
SYSTEMS = [(16, 8, 1, 0.5, 2.0), (24, 12, 2, 0.35, 1.0), (16, 8, 3, 0.7, 3.5), (32, 16, 1, 0.6, 0.5),
           (12, 6, 2, 0.45, 2.5)]


@pytest.fixture(scope="module")
def sg():
    import __graft_entry__ as g
    g.build()
    import paper_2101_01763_gb300 as m
    return m


@pytest.fixture(scope="module")
def systems(sg):
    out = []
    dev = torch.device("cuda")
    for q, (nt, nr, p, mach, alpha) in enumerate(SYSTEMS):
        X = naca_ogrid(nt, nr, 2101_0500 + q)
        u = modal_state(X, p, mach, alpha, 0.05, 2101_0500 + q)
        rhs, A, _ = sg.assemble(torch.as_tensor(X, device=dev), p, torch.as_tensor(u, device=dev), mach, alpha, 10.0)
        plan = sg.Plan(nt, nr, A.B, 0)
        out.append(dict(rhs=rhs, A=A, plan=plan))
    return out


def _dense(A):
    return dg.bsr_to_dense(A.row_ptr.cpu().numpy(), A.col.cpu().numpy(), A.blocks_rowmajor())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_factor_matches_single(sg, systems, prec):
    Fb = sg.factor_batched([s["plan"] for s in systems], [s["A"] for s in systems], 1e-3, prec)
    rng = np.random.default_rng(3)
    for s, fb in zip(systems, Fb):
        f1 = sg.Factor(s["plan"], s["A"], 1e-3, prec)
        st1, stb = f1.stats(), fb.stats()
        assert stb["levels"] == st1["levels"]
        assert stb["sum_r"] == st1["sum_r"] and stb["n_sparsified"] == st1["n_sparsified"]
        assert stb["top_size"] == st1["top_size"] and stb["factor_bytes"] == st1["factor_bytes"]
        for tr in (False, True):
            r = torch.as_tensor(rng.standard_normal(s["rhs"].numel()), device="cuda")
            z1 = f1.apply(r, transpose=tr)
            zb = fb.apply(r, transpose=tr)
            tol = 1e-12 if prec == "fp64" else 1e-5
            assert (torch.linalg.norm(zb - z1) / torch.linalg.norm(z1)).item() <= tol
        f1.close()
    for fb in Fb[::-1]:                          # any order; memory goes with the last handle
        fb.close()


def test_batched_eps0_is_exact_per_system(sg, systems):
    Fb = sg.factor_batched([s["plan"] for s in systems], [s["A"] for s in systems], 0.0, "fp64")
    for s, fb in zip(systems, Fb):
        Ad = _dense(s["A"])
        b = s["rhs"].cpu().numpy()
        x = fb.apply(s["rhs"]).cpu().numpy()
        # normwise backward error in the infinity norm
        be = np.abs(Ad @ x - b).max() / (np.abs(Ad).sum(axis=1).max() * np.abs(x).max() + np.abs(b).max())
        assert be <= 1e-12
    # close the middle handles first: the others keep working
    for q in (2, 1, 3):
        Fb[q].close()
    z = Fb[4].apply(systems[4]["rhs"])
    assert torch.isfinite(z).all()
    Fb[0].close()
    Fb[4].close()


def test_batched_solve_matches_dense(sg, systems):
    Fb = sg.factor_batched([s["plan"] for s in systems], [s["A"] for s in systems], 1e-3, "mixed")
    xs, stats, status = sg.sstep_gmres_batched([s["A"] for s in systems], Fb, [s["rhs"] for s in systems],
                                               s=4, restart=60, tol=1e-10)
    assert status == [0] * len(systems)
    for s, x, st in zip(systems, xs, stats):
        assert st["converged"] and st["true_relres"] <= 1e-10
        Ad = _dense(s["A"])
        xd = np.linalg.solve(Ad, s["rhs"].cpu().numpy())
        assert np.linalg.norm(x.cpu().numpy() - xd) / np.linalg.norm(xd) <= 1e-6
    # the same solves one at a time give the same iterates (deterministic kernels)
    for q in (0, 2):
        x1, st1 = sg.sstep_gmres(systems[q]["A"], Fb[q], systems[q]["rhs"], s=4, restart=60, tol=1e-10)
        assert st1["iters"] == stats[q]["iters"]
        assert (torch.linalg.norm(x1 - xs[q]) / torch.linalg.norm(x1)).item() <= 1e-12
    for fb in Fb:
        fb.close()


def test_batched_argument_errors(sg, systems):
    with pytest.raises(sg.SpandError):
        sg.factor_batched([systems[0]["plan"]], [systems[1]["A"]], 1e-3, "mixed")   # plan / matrix mismatch
    with pytest.raises(sg.SpandError):
        sg.factor_batched([s["plan"] for s in systems[:2]], [s["A"] for s in systems[:2]], -1.0, "mixed")
