"""Thin Python layer over the C ABI.  PyTorch provides device memory and
streams; every computation runs in the library's CUDA kernels."""
import ctypes as C

import numpy as np
import torch

from . import _lib as L


def kernel_launches():
    """spand_kernel_launches: kernels the library has launched in this process."""
    return int(L.lib().spand_kernel_launches())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _need(t, dtype, name):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")


class BSR:
    """Device block-CSR matrix (blocks column-major, see the C header)."""

    def __init__(self, K, B, row_ptr, col, val):
        self.K, self.B = K, B
        self.row_ptr, self.col, self.val = row_ptr, col, val
        self.nnzb = col.numel()

    def struct(self):
        return L.BsrMatrix(self.K, self.B, self.nnzb, self.row_ptr.data_ptr(), self.col.data_ptr(),
                           self.val.data_ptr())

    @staticmethod
    def empty(K, B, nnzb, device="cuda"):
        return BSR(K, B, torch.empty(K + 1, dtype=torch.int32, device=device),
                   torch.empty(nnzb, dtype=torch.int32, device=device),
                   torch.empty(nnzb * B * B, dtype=torch.float64, device=device))

    @staticmethod
    def from_host(row_ptr, col, val_rowmajor, device="cuda"):
        """From (row_ptr, col, val[nnzb, B, B] row-major blocks) numpy arrays."""
        nnzb, B, _ = val_rowmajor.shape
        v = np.ascontiguousarray(np.transpose(val_rowmajor, (0, 2, 1))).reshape(-1)
        return BSR(len(row_ptr) - 1, B, torch.as_tensor(np.asarray(row_ptr, np.int32), device=device),
                   torch.as_tensor(np.asarray(col, np.int32), device=device),
                   torch.as_tensor(v, dtype=torch.float64, device=device))

    def blocks_rowmajor(self):
        """val as a host [nnzb, B, B] row-major array."""
        v = self.val.detach().cpu().numpy().reshape(self.nnzb, self.B, self.B)
        return np.transpose(v, (0, 2, 1))


def assemble(nodes, p, u_hat, mach, alpha_deg, cfl, gamma=1.4, bc="wall", stream=None):
    """dg_assemble_jacobian: returns (rhs, A, dtau).  nodes: cuda f64 [n_r+1, n_theta, 2]."""
    _need(nodes, torch.float64, "nodes")
    _need(u_hat, torch.float64, "u_hat")
    n_r, n_theta = nodes.shape[0] - 1, nodes.shape[1]
    K = n_r * n_theta
    B = 4 * (p + 1) ** 2
    nnzb = 5 * K - 2 * n_theta if n_r > 1 else 3 * K
    A = BSR.empty(K, B, nnzb, device=nodes.device)
    rhs = torch.empty(K * B, dtype=torch.float64, device=nodes.device)
    mesh = L.DgMesh(n_theta, n_r, nodes.data_ptr())
    flow = L.DgFlow(gamma, mach, alpha_deg, cfl, L.BC_WALL if bc == "wall" else L.BC_FARFIELD)
    Ast = A.struct()
    dt = C.c_double(0.0)
    L.check(L.lib().dg_assemble_jacobian(C.byref(mesh), p, _ptr(u_hat), C.byref(flow), _ptr(rhs),
                                         C.byref(Ast), C.byref(dt), _stream(stream)), "dg_assemble_jacobian")
    A.nnzb = Ast.nnzb
    return rhs, A, dt.value


def spmv(A, x, transpose=False, out=None, stream=None):
    _need(x, torch.float64, "x")
    y = torch.empty_like(x) if out is None else out
    st = A.struct()
    L.check(L.lib().bsr_spmv(C.byref(st), _ptr(x), _ptr(y), int(transpose), _stream(stream)), "bsr_spmv")
    return y


class Plan:
    """spand_analyze: nested-dissection plan of an n_theta x n_r grid."""

    def __init__(self, n_theta, n_r, B, depth=0):
        h = C.c_void_p()
        L.check(L.lib().spand_analyze(n_theta, n_r, B, depth, C.byref(h)), "spand_analyze")
        self.h = h
        self.n_theta, self.n_r, self.B = n_theta, n_r, B

    def export(self):
        K, D, nn, tl = C.c_int(), C.c_int(), C.c_int(), C.c_int64()
        L.check(L.lib().spand_plan_sizes(self.h, C.byref(K), C.byref(D), C.byref(nn), C.byref(tl)), "sizes")
        owner = np.zeros(K.value, np.int32)
        lev = np.zeros(nn.value, np.int32)
        tab = np.zeros(tl.value, np.int32)
        L.check(L.lib().spand_plan_export(self.h, owner.ctypes.data_as(C.c_void_p),
                                          lev.ctypes.data_as(C.c_void_p), tab.ctypes.data_as(C.c_void_p)),
                "export")
        return dict(K=K.value, D=D.value, owner=owner, node_level=lev, table=tab)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                L.lib().spand_plan_destroy(self.h)
                self.h = None
        except Exception:
            pass


def parse_table(table, D):
    """Cluster table of spand_plan_export -> list over levels of cluster dicts."""
    levels, k = [], 0
    for _ in range(D + 1):
        nc = int(table[k]); k += 1
        cl = []
        for _ in range(nc):
            node, inter = int(table[k]), bool(table[k + 1]); k += 2
            nk = int(table[k]); k += 1
            key = [int(v) for v in table[k:k + nk]]; k += nk
            ne = int(table[k]); k += 1
            el = [int(v) for v in table[k:k + ne]]; k += ne
            nch = int(table[k]); k += 1
            ch = [int(v) for v in table[k:k + nch]]; k += nch
            cl.append(dict(node=node, interior=inter, key=key, elems=el, children=ch))
        levels.append(cl)
    return levels


class Factor:
    """spand_factor: spaND preconditioner of A with tolerance eps."""

    def __init__(self, plan, A, eps, precision="fp64", stream=None):
        prec = L.SPAND_FP64 if precision == "fp64" else L.SPAND_MIXED
        h = C.c_void_p()
        st = A.struct()
        L.check(L.lib().spand_factor(plan.h, C.byref(st), float(eps), prec, C.byref(h), _stream(stream)),
                "spand_factor")
        self.h = h
        self.N = A.K * A.B
        self.precision = precision

    @classmethod
    def _wrap(cls, h, N, precision):
        f = cls.__new__(cls)
        f.h, f.N, f.precision = h, N, precision
        return f

    def apply(self, r, transpose=False, out=None, stream=None):
        _need(r, torch.float64, "r")
        z = torch.empty_like(r) if out is None else out
        L.check(L.lib().spand_apply(self.h, _ptr(r), _ptr(z), int(transpose), _stream(stream)), "spand_apply")
        return z

    def stats(self):
        s = L.SpandStats()
        L.check(L.lib().spand_factor_stats(self.h, C.byref(s)), "spand_factor_stats")
        n = s.levels
        return dict(levels=n, n_sparsified=list(s.n_sparsified[:n]), sum_n=list(s.sum_n[:n]),
                    sum_r=list(s.sum_r[:n]), max_r=list(s.max_r[:n]), top_size=s.top_size,
                    factor_bytes=s.factor_bytes, factor_flops=s.factor_flops,
                    t_rrqr_ms=s.t_rrqr_ms, rrqr_bytes=s.rrqr_bytes, rrqr_launches=s.rrqr_launches,
                    t_elim_gemm_ms=s.t_elim_gemm_ms, elim_gemm_flops=s.elim_gemm_flops,
                    elim_gemm_launches=s.elim_gemm_launches, t_rrqr_level_ms=list(s.t_rrqr_level_ms[:n]),
                    rrqr_bytes_level=list(s.rrqr_bytes_level[:n]),
                    rrqr_form_count=[list(s.rrqr_form_count[l]) for l in range(n)],
                    t_host_ms=s.t_host_ms, t_wait_ms=s.t_wait_ms, t_host_phase_ms=list(s.t_host_phase_ms),
                    rrqr_stream_bytes=s.rrqr_stream_bytes,
                    rrqr_stream_bytes_level=list(s.rrqr_stream_bytes_level[:n]))

    def close(self):
        if getattr(self, "h", None):
            L.lib().spand_factor_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def factor_batched(plans, As, eps, precision="mixed", stream=None):
    """spand_factor_batched: one factorization of several systems; a Factor per system."""
    n = len(As)
    prec = L.SPAND_FP64 if precision == "fp64" else L.SPAND_MIXED
    ph = (C.c_void_p * n)(*[p.h.value for p in plans])
    mats = (L.BsrMatrix * n)(*[A.struct() for A in As])
    out = (C.c_void_p * n)()
    L.check(L.lib().spand_factor_batched(n, ph, mats, float(eps), prec, out, _stream(stream)),
            "spand_factor_batched")
    return [Factor._wrap(C.c_void_p(out[q]), As[q].K * As[q].B, precision) for q in range(n)]


def sstep_gmres_batched(As, Ms, bs, s=4, restart=60, tol=1e-8, max_iters=400, basis="newton", transpose=False,
                        stream=None):
    """sstep_gmres_solve_batched: returns (xs, stats list, statuses)."""
    n = len(As)
    for b in bs:
        _need(b, torch.float64, "b")
    xs = [torch.zeros_like(b) for b in bs]
    mats = (L.BsrMatrix * n)(*[A.struct() for A in As])
    mh = (C.c_void_p * n)(*[(M.h.value if M is not None else None) for M in Ms]) if Ms is not None else None
    bp = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    opt = L.GmresOpts(s, restart, tol, max_iters, L.BASIS_NEWTON if basis == "newton" else L.BASIS_MONOMIAL,
                      int(transpose))
    opts = (L.GmresOpts * n)(*[opt for _ in range(n)])
    stt = (L.GmresStats * n)()
    status = (C.c_int * n)()
    rc = L.lib().sstep_gmres_solve_batched(n, mats, mh, bp, xp, opts, stt, status, _stream(stream))
    if rc != L.OK and rc != -6:
        L.check(rc, "sstep_gmres_solve_batched")
    stats = [dict(iters=t.iters, restarts=t.restarts, true_relres=t.true_relres, converged=(status[q] == L.OK))
             for q, t in enumerate(stt)]
    return xs, stats, list(status)


def sstep_gmres(A, M, b, x0=None, s=4, restart=40, tol=1e-8, max_iters=400, basis="newton",
                transpose=False, stream=None, raise_on_nonconvergence=False):
    """sstep_gmres_solve: returns (x, stats dict)."""
    _need(b, torch.float64, "b")
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    opts = L.GmresOpts(s, restart, tol, max_iters, L.BASIS_NEWTON if basis == "newton" else L.BASIS_MONOMIAL,
                       int(transpose))
    stt = L.GmresStats()
    st = A.struct()
    status = L.lib().sstep_gmres_solve(C.byref(st), M.h if M is not None else None, _ptr(b), _ptr(x),
                                       C.byref(opts), C.byref(stt), _stream(stream))
    if status != L.OK and (status != -6 or raise_on_nonconvergence):
        L.check(status, "sstep_gmres_solve")
    stats = _gmres_stats(stt, status)
    stats["shifts"] = [complex(stt.shifts_re[k], stt.shifts_im[k]) for k in range(s)]
    return x, stats


def matrix_powers(A, M, v0, shifts, transpose=False, stream=None):
    """sstep_matrix_powers: the Newton basis [v_1 .. v_s] (N x s device tensor)
    from v0 with the preconditioner fused into the SpMV chain.  shifts: s
    complex numbers, conjugate pairs adjacent (+imag first)."""
    _need(v0, torch.float64, "v0")
    s = len(shifts)
    V = torch.empty((s, v0.numel()), dtype=torch.float64, device=v0.device)   # row k = column k of N x s
    re = (C.c_double * s)(*[complex(t).real for t in shifts])
    im = (C.c_double * s)(*[complex(t).imag for t in shifts])
    st = A.struct()
    L.check(L.lib().sstep_matrix_powers(C.byref(st), M.h if M is not None else None, _ptr(v0), s,
                                        C.cast(re, C.c_void_p), C.cast(im, C.c_void_p), _ptr(V), int(transpose),
                                        _stream(stream)), "sstep_matrix_powers")
    return V.T


def _gmres_stats(stt, status):
    return dict(iters=stt.iters, restarts=stt.restarts, reductions=stt.reductions,
                true_relres=stt.true_relres, est_relres=stt.est_relres, orth_err=stt.orth_err,
                t_spmv_ms=stt.t_spmv_ms, t_apply_ms=stt.t_apply_ms, t_orth_ms=stt.t_orth_ms,
                t_small_ms=stt.t_small_ms, t_gram_ms=stt.t_gram_ms, gram_bytes=stt.gram_bytes,
                gram_calls=stt.gram_calls, t_bupd_ms=stt.t_bupd_ms, bupd_bytes=stt.bupd_bytes,
                bupd_calls=stt.bupd_calls, converged=(status == L.OK))


def gmres(A, M, b, x0=None, restart=40, tol=1e-8, max_iters=400, transpose=False, stream=None,
          raise_on_nonconvergence=False):
    """gmres_solve (Algorithm 1, MGS): returns (x, stats dict)."""
    _need(b, torch.float64, "b")
    x = torch.zeros_like(b) if x0 is None else x0.clone()
    opts = L.GmresOpts(1, restart, tol, max_iters, L.BASIS_NEWTON, int(transpose))
    stt = L.GmresStats()
    st = A.struct()
    status = L.lib().gmres_solve(C.byref(st), M.h if M is not None else None, _ptr(b), _ptr(x),
                                 C.byref(opts), C.byref(stt), _stream(stream))
    if status != L.OK and (status != -6 or raise_on_nonconvergence):
        L.check(status, "gmres_solve")
    return x, _gmres_stats(stt, status)


def pattern_outer(A, u, v, alpha=1.0, out=None, stream=None):
    """bsr_pattern_outer: alpha * u v^T on A's block pattern (values in A's layout)."""
    _need(u, torch.float64, "u")
    _need(v, torch.float64, "v")
    o = torch.empty_like(A.val) if out is None else out
    st = A.struct()
    L.check(L.lib().bsr_pattern_outer(C.byref(st), _ptr(u), _ptr(v), float(alpha), _ptr(o), _stream(stream)),
            "bsr_pattern_outer")
    return o


def cfl_ramp(cfl0, cfl_inf, r0, r_prev):
    """dg_cfl_ramp: CFL^n = min(CFL^0 ||R^0|| / ||R^{n-1}||, CFL^inf) (Eq. 9)."""
    return float(L.lib().dg_cfl_ramp(float(cfl0), float(cfl_inf), float(r0), float(r_prev)))


def march(nodes, p, u_hat, mach, alpha_deg, plan, cfl0=10.0, cfl_inf=1e6, max_steps=20, rtol=1e-10, eps=1e-3,
          precision="mixed", s=4, restart=60, tol=1e-10, max_iters=400, basis="newton", gamma=1.4, bc="wall",
          stream=None):
    """dg_pseudo_time_march from u_hat (not modified): returns (u, history dict).

    history: res (||R^n||, n = 0..steps), cfl, dtau, gmres_iters (per solve), steps.
    """
    _need(nodes, torch.float64, "nodes")
    _need(u_hat, torch.float64, "u_hat")
    n_r, n_theta = nodes.shape[0] - 1, nodes.shape[1]
    u = u_hat.clone()
    mesh = L.DgMesh(n_theta, n_r, nodes.data_ptr())
    flow = L.DgFlow(gamma, mach, alpha_deg, cfl0, L.BC_WALL if bc == "wall" else L.BC_FARFIELD)
    go = L.GmresOpts(s, restart, tol, max_iters, L.BASIS_NEWTON if basis == "newton" else L.BASIS_MONOMIAL, 0)
    opts = L.DgMarchOpts(int(max_steps), float(cfl_inf), float(rtol), float(eps),
                         L.SPAND_FP64 if precision == "fp64" else L.SPAND_MIXED, go)
    res = np.zeros(max_steps + 1)
    cfl = np.zeros(max_steps + 1)
    dts = np.zeros(max_steps + 1)
    its = np.zeros(max(max_steps, 1), np.int32)
    hist = L.DgMarchHistory(0, res.ctypes.data, cfl.ctypes.data, dts.ctypes.data, its.ctypes.data)
    L.check(L.lib().dg_pseudo_time_march(C.byref(mesh), p, _ptr(u), C.byref(flow), plan.h, C.byref(opts),
                                         C.byref(hist), _stream(stream)), "dg_pseudo_time_march")
    n = hist.steps
    return u, dict(steps=n, res=res[:n + 1].copy(), cfl=cfl[:n + 1].copy(), dtau=dts[:n + 1].copy(),
                   gmres_iters=its[:n].copy())


class SpandSolve(torch.autograd.Function):
    """x = A^-1 b by spaND-preconditioned s-step GMRES, differentiable in (A values, b).

    backward: lambda = A^-T g by s-step GMRES with the transposed spaND apply
    (the factor of the forward solve is reused), dL/db = lambda and
    dL/dA = -lambda x^T on A's block pattern (bsr_pattern_outer).
    Call as SpandSolve.apply(val, b, A, plan, eps, precision, s, restart, tol).
    """

    @staticmethod
    def forward(ctx, val, b, A, plan, eps=1e-3, precision="fp64", s=4, restart=60, tol=1e-10):
        A2 = BSR(A.K, A.B, A.row_ptr, A.col, val.detach().contiguous())
        F = Factor(plan, A2, eps, precision)
        x, st = sstep_gmres(A2, F, b.detach().contiguous(), s=s, restart=restart, tol=tol)
        if not st["converged"]:
            raise L.SpandError(-6, "SpandSolve.forward")
        ctx.A, ctx.F, ctx.opts = A2, F, (s, restart, tol)
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        s, restart, tol = ctx.opts
        lam, st = sstep_gmres(ctx.A, ctx.F, g.contiguous(), s=s, restart=restart, tol=tol, transpose=True)
        if not st["converged"]:
            raise L.SpandError(-6, "SpandSolve.backward")
        dval = pattern_outer(ctx.A, lam, x, alpha=-1.0)
        return dval, lam, None, None, None, None, None, None, None
