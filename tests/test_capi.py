"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and its host-side nested-dissection tables are bit-exact
against the oracle (Sec. 2.2.1, Sec. 3.3)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2101_01763_gb300 import _lib
    return _lib.lib()


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "spand_gb300.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|double|size_t|uint64_t|const char\*)\s+(\w+)\s*\(", txt, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = _header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for st in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib.spand_status_string(st)


@pytest.mark.parametrize("nt,nr,D", [(16, 8, 2), (12, 6, 2), (64, 32, 6), (24, 20, 4), (10, 3, 3), (128, 64, 8)])
def test_plan_tables_bit_exact(lib, nt, nr, D):
    from oracle.nd import build_hierarchy
    from paper_2101_01763_gb300.api import Plan, parse_table
    t, levels = build_hierarchy(nt, nr, D)
    P = Plan(nt, nr, 16, D)
    ex = P.export()
    assert ex["D"] == D
    assert np.array_equal(ex["owner"], t.owner.astype(np.int32))
    assert list(ex["node_level"]) == list(t.level)
    got = parse_table(ex["table"], D)
    for l in range(D + 1):
        assert len(got[l]) == len(levels[l])
        for a, b in zip(got[l], levels[l]):
            assert a["node"] == b["node"] and a["key"] == list(b["key"])
            assert a["interior"] == b["interior"] and a["elems"] == b["elems"]
            assert a["children"] == (b["children"] or [])


def test_default_depth(lib):
    from paper_2101_01763_gb300.api import Plan
    from synth import get_config
    for name in ("C1", "C2", "C3", "C4"):
        c = get_config(name)
        assert Plan(c.n_theta, c.n_r, c.B).export()["D"] == c.nd_depth


def test_analyze_rejects_bad_args(lib):
    h = C.c_void_p()
    assert lib.spand_analyze(3, 4, 16, 2, C.byref(h)) == -1
    assert lib.spand_analyze(16, 0, 16, 2, C.byref(h)) == -1
    assert lib.spand_analyze(16, 8, 16, 2, None) == -1


def test_cfl_ramp_matches_oracle(lib):
    """dg_cfl_ramp (host) against the oracle's Eq. 9, bit for bit."""
    from oracle.march import cfl_ramp
    from paper_2101_01763_gb300.api import cfl_ramp as ramp
    rng = np.random.default_rng(9)
    for _ in range(200):
        c0 = 10 ** rng.uniform(-2, 4)
        cinf = c0 * 10 ** rng.uniform(0, 6)
        r0 = 10 ** rng.uniform(-8, 2)
        rp = r0 * 10 ** rng.uniform(-12, 1)
        assert ramp(c0, cinf, r0, rp) == cfl_ramp(c0, cinf, r0, rp)
    assert ramp(10.0, 1e6, 1.0, 0.0) == 1e6 == cfl_ramp(10.0, 1e6, 1.0, 0.0)


def test_march_rejects_bad_args(lib):
    """Argument checks of dg_pseudo_time_march return before any device work
    (the pointers below are never dereferenced)."""
    from paper_2101_01763_gb300 import _lib as L
    from paper_2101_01763_gb300.api import Plan
    P = Plan(16, 8, 16, 2)
    mesh = L.DgMesh(16, 8, 16)
    go = L.GmresOpts(4, 40, 1e-10, 400, 0, 0)

    def call(p=1, flow_cfl=10.0, cfl_inf=1e6, steps=5, plan=P, m=mesh):
        flow = L.DgFlow(1.4, 0.5, 2.0, flow_cfl, 0)
        opts = L.DgMarchOpts(steps, cfl_inf, 1e-10, 1e-3, 0, go)
        return lib.dg_pseudo_time_march(C.byref(m) if m is not None else None, p, C.c_void_p(16),
                                        C.byref(flow), plan.h, C.byref(opts), None, None)

    assert call(p=2) == -1                       # plan built for B = 16, not 36
    assert call(m=L.DgMesh(16, 4, 16)) == -1     # plan of another grid
    assert call(flow_cfl=0.0) == -1
    assert call(cfl_inf=5.0) == -1               # CFL^inf below CFL^0
    assert call(steps=-1) == -1
    assert call(m=None) == -1
    assert call(p=4) == -8
