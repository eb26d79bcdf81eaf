"""The no-allocation GMRES entry point against the regular one.

sstep_gmres_solve_noalloc serves callers that may not allocate device memory
while they run (a program that gives all device memory to its own pool at
start-up, or one with a fixed device-memory budget).  Its scratch is one fixed
device array; these tests check, through the C ABI, that two calls in a row
return the same solution as sstep_gmres_solve, that a call on a factor never
applied before (forward and transposed) takes no device memory (free device
memory and the stream-ordered pool's usage are unchanged, and the pool's usage
never rose during the calls), and that a problem too large for the array is
refused with SPAND_ERR_SCRATCH.  Kept in a file of its own, collected last, so
a failure here comes after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__ as g
    g.build()
    import paper_2101_01763_gb300 as sg
    from paper_2101_01763_gb300 import _lib as L
    from oracle import dg
    from synth import get_config, modal_state, naca_ogrid
    c = get_config("C1")
    X = naca_ogrid(c.n_theta, c.n_r, c.seed)
    u = modal_state(X, c.p, c.mach, c.alpha_deg, c.amp, c.seed)
    rhs_o, bsr, _ = dg.assemble(X, c.p, u, c.mach, c.alpha_deg, c.cfl)
    A = sg.BSR.from_host(*bsr)
    b = torch.as_tensor(rhs_o, device="cuda")
    F = sg.Factor(sg.Plan(c.n_theta, c.n_r, c.B, c.nd_depth), A, c.eps, "fp64")
    return sg, L, c, A, b, F


def _noalloc(L, A, F, b, s, restart, tol, max_iters, transpose=0, x=None):
    x = torch.zeros_like(b) if x is None else x
    opts = L.GmresOpts(s, restart, tol, max_iters, L.BASIS_NEWTON, transpose)
    st = L.GmresStats()
    Ast = A.struct()
    status = L.lib().sstep_gmres_solve_noalloc(C.byref(Ast), F.h, C.c_void_p(b.data_ptr()),
                                                C.c_void_p(x.data_ptr()), C.byref(opts), C.byref(st),
                                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return status, x, st


def test_noalloc_matches_regular_twice(setup):
    sg, L, c, A, b, F = setup
    ref, st_ref = sg.sstep_gmres(A, F, b, s=c.s, restart=c.restart, tol=c.tol, max_iters=c.max_iters)
    assert st_ref["converged"]
    ref = ref.cpu().numpy()
    for call in range(2):                 # the array keeps the previous call's contents
        status, x, st = _noalloc(L, A, F, b, c.s, c.restart, c.tol, c.max_iters)
        assert status == 0, L.STATUS.get(status)
        xn = x.cpu().numpy()
        assert np.linalg.norm(xn - ref) / np.linalg.norm(ref) <= 1e-10, call
        assert st.iters == st_ref["iters"] and st.true_relres <= c.tol


def test_noalloc_rejects_oversize(setup):
    sg, L, c, A, b, F = setup
    cap = L.lib().sstep_gmres_noalloc_capacity()
    assert cap == 8 << 20
    status, x, st = _noalloc(L, A, F, b, 4, 480, c.tol, 480)   # needs ~50 MB of scratch
    assert status == -9
    assert b"no-allocation" in L.lib().spand_status_string(status)


class _Pool:
    """The device's default stream-ordered memory pool, read through the driver
    API: bytes in use now, and the most in use since the last reset."""
    USED_CURRENT, USED_HIGH = 7, 8          # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH

    def __init__(self):
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int()
        assert self.cu.cuDeviceGet(C.byref(dev), torch.cuda.current_device()) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def get(self, attr):
        v = C.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, C.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = C.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_HIGH, C.byref(zero)) == 0


def test_noalloc_fresh_factor_allocates_nothing(setup):
    sg, L, c, A, b, F = setup
    # the first call in a process loads the library's kernels and looks up the
    # scratch array's address; the calls measured below come after it
    status, _, _ = _noalloc(L, A, F, b, c.s, c.restart, c.tol, c.max_iters)
    assert status == 0
    F2 = sg.Factor(sg.Plan(c.n_theta, c.n_r, c.B, c.nd_depth), A, c.eps, "fp64")   # never applied yet
    xs = [torch.zeros_like(b), torch.zeros_like(b)]
    pool = _Pool()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    used0 = pool.get(_Pool.USED_CURRENT)
    pool.reset_high()
    sts = []
    for tr in (0, 1):
        status, _, st = _noalloc(L, A, F2, b, c.s, c.restart, 1e-10, c.max_iters, transpose=tr, x=xs[tr])
        assert status == 0, L.STATUS.get(status)
        sts.append(st)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0           # nothing taken (the pool may only have given memory back)
    assert pool.get(_Pool.USED_CURRENT) == used0
    assert pool.get(_Pool.USED_HIGH) <= used0
    # and the answers are the regular solver's
    for tr in (0, 1):
        ref, st_ref = sg.sstep_gmres(A, F2, b, s=c.s, restart=c.restart, tol=1e-10, max_iters=c.max_iters,
                                     transpose=bool(tr))
        assert st_ref["converged"] and sts[tr].iters == st_ref["iters"]
        r = ref.cpu().numpy()
        assert np.linalg.norm(xs[tr].cpu().numpy() - r) / np.linalg.norm(r) <= 1e-10
    F2.close()
