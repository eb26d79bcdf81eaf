"""The matrix-powers step of Algorithm 2 with the preconditioner fused into the
SpMV chain (sstep_matrix_powers), against the oracle's Newton-basis
recurrence on the same matrix and the same preconditioner.

FP64 factor at eps > 0 (ranks equal to the oracle's, so M^-1 is the same
operator to rounding): every basis vector equals the oracle's to 1e-10
relative, for real shifts, a conjugate pair and the monomial basis, forward and
transposed.  Mixed factor: the same recurrence with the FP32 preconditioner's
output read in place, against the same recurrence run through separate
spand_apply and bsr_spmv calls (1e-12).  Bad shift orders are refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dg, spand  # noqa: E402
from oracle.gmres import _mpk  # noqa: E402
from synth import get_config, modal_state, naca_ogrid  # noqa: E402


@pytest.fixture(scope="module")
def case():
    import __graft_entry__ as g
    g.build()
    import paper_2101_01763_gb300 as sg
    c = get_config("C1")
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
    rhs_o, bsr, _ = dg.assemble(X, c.p, u, c.mach, c.alpha_deg, c.cfl)
    A = sg.BSR.from_host(*bsr)
    S = dg.bsr_to_scipy(*bsr).tocsr()
    Fo = spand.factor(bsr, c.n_theta, c.n_r, c.nd_depth, c.eps)
    plan = sg.Plan(c.n_theta, c.n_r, c.B, c.nd_depth)
    return sg, c, A, S, Fo, plan


SHIFTS = [
    [0.3, 1.1, 2.0, 0.7],                         # real shifts
    [0.5 + 0.4j, 0.5 - 0.4j, 1.2, 0.9],           # a conjugate pair first
    [0.0, 0.0, 0.0, 0.0],                         # monomial
]


@pytest.mark.parametrize("shifts", SHIFTS)
@pytest.mark.parametrize("transpose", [False, True])
def test_matrix_powers_match_oracle_fp64(case, shifts, transpose):
    sg, c, A, S, Fo, plan = case
    F = sg.Factor(plan, A, c.eps, "fp64")
    v0 = np.random.default_rng(5).standard_normal(c.N)
    V = sg.matrix_powers(A, F, torch.as_tensor(v0, device="cuda"), shifts, transpose=transpose).cpu().numpy()
    if transpose:
        Vo = _mpk(lambda v: S.T @ v, lambda v: spand.apply_transpose(Fo, v), v0, [complex(t) for t in shifts])
    else:
        Vo = _mpk(lambda v: S @ v, lambda v: spand.apply(Fo, v), v0, [complex(t) for t in shifts])
    for k in range(len(shifts)):
        assert np.linalg.norm(V[:, k] - Vo[:, k]) / np.linalg.norm(Vo[:, k]) <= 1e-10, k


def test_matrix_powers_mixed_reads_fp32_output_in_place(case):
    sg, c, A, S, Fo, plan = case
    F = sg.Factor(plan, A, c.eps, "mixed")
    shifts = SHIFTS[1]
    v0 = torch.as_tensor(np.random.default_rng(6).standard_normal(c.N), device="cuda")
    V = sg.matrix_powers(A, F, v0, shifts)
    # the same recurrence through the public apply (FP32 sweep, FP64 output) and SpMV
    ref, prev, cur = [], None, v0
    for t in shifts:
        t = complex(t)
        y = sg.spmv(A, F.apply(cur)) - t.real * cur
        if t.imag < 0:
            y = y + t.imag ** 2 * prev
        ref.append(y)
        prev, cur = cur, y
    for k in range(len(shifts)):
        assert (torch.linalg.norm(V[:, k] - ref[k]) / torch.linalg.norm(ref[k])).item() <= 1e-12, k


def test_matrix_powers_rejects_bad_shift_order(case):
    sg, c, A, S, Fo, plan = case
    v0 = torch.zeros(c.N, dtype=torch.float64, device="cuda")
    with pytest.raises(sg.SpandError) as ei:
        sg.matrix_powers(A, None, v0, [0.5 - 0.4j, 0.5 + 0.4j])   # second shift of a pair first
    assert ei.value.status == -1
