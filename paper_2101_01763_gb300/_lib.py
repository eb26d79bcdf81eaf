"""ctypes view of include/spand_gb300.h (argument marshalling only).

Loading fails loudly when the compiled library is missing: there is no
fallback implementation.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspand_gb300.so")

OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "zero pivot", -4: "CholQR breakdown",
          -5: "non-finite value", -6: "not converged", -7: "CUDA error", -8: "unsupported",
          -9: "larger than the no-allocation scratch"}
SPAND_FP64, SPAND_MIXED = 0, 1
BASIS_NEWTON, BASIS_MONOMIAL = 0, 1
BC_WALL, BC_FARFIELD = 0, 1


class SpandError(RuntimeError):
    def __init__(self, status, where):
        super().__init__(f"{where}: status {status} ({STATUS.get(status, '?')})")
        self.status = status


class DgMesh(C.Structure):
    _fields_ = [("n_theta", C.c_int), ("n_r", C.c_int), ("nodes", C.c_void_p)]


class DgFlow(C.Structure):
    _fields_ = [("gamma", C.c_double), ("mach", C.c_double), ("alpha_deg", C.c_double),
                ("cfl", C.c_double), ("bc_mode", C.c_int)]


class BsrMatrix(C.Structure):
    _fields_ = [("K", C.c_int), ("B", C.c_int), ("nnzb", C.c_int), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class SpandStats(C.Structure):
    _fields_ = [("levels", C.c_int), ("n_sparsified", C.c_int64 * 32), ("sum_n", C.c_int64 * 32),
                ("sum_r", C.c_int64 * 32), ("max_r", C.c_int64 * 32), ("top_size", C.c_int64),
                ("factor_bytes", C.c_int64), ("factor_flops", C.c_double),
                ("t_rrqr_ms", C.c_double), ("rrqr_bytes", C.c_double), ("rrqr_launches", C.c_int),
                ("t_elim_gemm_ms", C.c_double), ("elim_gemm_flops", C.c_double), ("elim_gemm_launches", C.c_int),
                ("t_rrqr_level_ms", C.c_double * 32), ("rrqr_bytes_level", C.c_double * 32),
                ("rrqr_form_count", (C.c_int * 4) * 32), ("t_host_ms", C.c_double), ("t_wait_ms", C.c_double),
                ("t_host_phase_ms", C.c_double * 8), ("rrqr_stream_bytes", C.c_double),
                ("rrqr_stream_bytes_level", C.c_double * 32)]


class GmresOpts(C.Structure):
    _fields_ = [("s", C.c_int), ("restart", C.c_int), ("tol", C.c_double), ("max_iters", C.c_int),
                ("basis", C.c_int), ("transpose", C.c_int)]


class GmresStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("reductions", C.c_int),
                ("true_relres", C.c_double), ("est_relres", C.c_double), ("orth_err", C.c_double),
                ("shifts_re", C.c_double * 16), ("shifts_im", C.c_double * 16),
                ("t_spmv_ms", C.c_double), ("t_apply_ms", C.c_double), ("t_orth_ms", C.c_double),
                ("t_small_ms", C.c_double), ("t_gram_ms", C.c_double), ("gram_bytes", C.c_double),
                ("gram_calls", C.c_int), ("t_bupd_ms", C.c_double), ("bupd_bytes", C.c_double),
                ("bupd_calls", C.c_int)]


class DgMarchOpts(C.Structure):
    _fields_ = [("max_steps", C.c_int), ("cfl_inf", C.c_double), ("rtol", C.c_double), ("eps", C.c_double),
                ("precision", C.c_int), ("gmres", GmresOpts)]


class DgMarchHistory(C.Structure):
    _fields_ = [("steps", C.c_int), ("res_norm", C.c_void_p), ("cfl", C.c_void_p), ("dtau", C.c_void_p),
                ("gmres_iters", C.c_void_p)]


EXPORTS = {
    "dg_assemble_jacobian": ([C.POINTER(DgMesh), C.c_int, C.c_void_p, C.POINTER(DgFlow), C.c_void_p,
                              C.POINTER(BsrMatrix), C.POINTER(C.c_double), C.c_void_p], C.c_int),
    "bsr_spmv": ([C.POINTER(BsrMatrix), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "bsr_pattern_outer": ([C.POINTER(BsrMatrix), C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p],
                          C.c_int),
    "spand_analyze": ([C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_void_p)], C.c_int),
    "spand_plan_destroy": ([C.c_void_p], C.c_int),
    "spand_plan_sizes": ([C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                          C.POINTER(C.c_int64)], C.c_int),
    "spand_plan_export": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "spand_factor": ([C.c_void_p, C.POINTER(BsrMatrix), C.c_double, C.c_int, C.POINTER(C.c_void_p),
                      C.c_void_p], C.c_int),
    "spand_factor_batched": ([C.c_int, C.POINTER(C.c_void_p), C.POINTER(BsrMatrix), C.c_double, C.c_int,
                              C.POINTER(C.c_void_p), C.c_void_p], C.c_int),
    "spand_factor_destroy": ([C.c_void_p], C.c_int),
    "spand_factor_stats": ([C.c_void_p, C.POINTER(SpandStats)], C.c_int),
    "spand_apply": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "sstep_gmres_solve": ([C.POINTER(BsrMatrix), C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(GmresOpts),
                           C.POINTER(GmresStats), C.c_void_p], C.c_int),
    "gmres_solve": ([C.POINTER(BsrMatrix), C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(GmresOpts),
                     C.POINTER(GmresStats), C.c_void_p], C.c_int),
    "sstep_matrix_powers": ([C.POINTER(BsrMatrix), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "sstep_gmres_solve_batched": ([C.c_int, C.POINTER(BsrMatrix), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_void_p), C.POINTER(GmresOpts), C.POINTER(GmresStats),
                                   C.POINTER(C.c_int), C.c_void_p], C.c_int),
    "sstep_gmres_solve_noalloc": ([C.POINTER(BsrMatrix), C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.POINTER(GmresOpts), C.POINTER(GmresStats), C.c_void_p], C.c_int),
    "sstep_gmres_noalloc_capacity": ([], C.c_size_t),
    "dg_pseudo_time_march": ([C.POINTER(DgMesh), C.c_int, C.c_void_p, C.POINTER(DgFlow), C.c_void_p,
                              C.POINTER(DgMarchOpts), C.POINTER(DgMarchHistory), C.c_void_p], C.c_int),
    "dg_cfl_ramp": ([C.c_double, C.c_double, C.c_double, C.c_double], C.c_double),
    "spand_status_string": ([C.c_int], C.c_char_p),
    "spand_kernel_launches": ([], C.c_uint64),
}

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"compiled library not found at {LIB_PATH}; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in EXPORTS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def check(status, where):
    if status != OK:
        raise SpandError(status, where)
