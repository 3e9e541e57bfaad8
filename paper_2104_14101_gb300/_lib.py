"""ctypes view of the C ABI declared in include/sks.h (argument marshalling only).

The library is loaded from ``libsks.so`` next to this file; importing the
product API without it raises immediately -- there is no fallback path.
"""
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsks.so")

# sks_status
OK, ERR_INVALID_ARG, ERR_NOT_PD, ERR_NO_CONVERGENCE, ERR_NUMERIC, ERR_TIMEOUT, ERR_CUDA, ERR_WORKSPACE, ERR_UNSUPPORTED = range(9)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NOT_PD", 3: "NO_CONVERGENCE", 4: "NUMERIC", 5: "TIMEOUT", 6: "CUDA",
                7: "WORKSPACE", 8: "UNSUPPORTED"}
# sks_kind
SRHT, GAUSSIAN, SJLT, RADEMACHER = 0, 1, 2, 3
KINDS = {"srht": SRHT, "gaussian": GAUSSIAN, "sjlt": SJLT, "rademacher": RADEMACHER, "gaussian-e4m3": 4}
# stop rules
STOP_RULES = {"estimate": 0, "certified": 1}
# sks_fixed_method
FIXED_METHODS = {"fixed-pcg": 0, "fixed-ihs": 1, "polyak-ihs": 2, "cg": 3}
# sks_dtype
F64, F32 = 0, 1
# sks_precision
PLAIN_F64, MIXED_REFINED = 0, 1


class Problem(C.Structure):
    _fields_ = [("dtype", C.c_int), ("n", C.c_int64), ("d", C.c_int64), ("lda", C.c_int64), ("k", C.c_int64),
                ("A", C.c_void_p), ("b", C.c_void_p), ("nu", C.c_double), ("lambda_diag", C.c_void_p)]


class TraceEvent(C.Structure):
    _fields_ = [("t", C.c_int64), ("m", C.c_int64), ("ratio", C.c_double), ("threshold", C.c_double),
                ("accepted", C.c_int32), ("outer", C.c_int32), ("column", C.c_int32), ("reserved", C.c_int32),
                ("delta", C.c_double), ("delta0", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("rho", C.c_double), ("m_init", C.c_int64), ("m_max", C.c_int64), ("kind", C.c_int),
                ("sjlt_s", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int64), ("precision", C.c_int),
                ("reuse_residual", C.c_int), ("seed", C.c_uint64), ("max_outer", C.c_int64),
                ("inner_tol", C.c_double), ("trace", C.POINTER(TraceEvent)), ("trace_cap", C.c_int64),
                ("stop_rule", C.c_int), ("cert_delta", C.c_double), ("cert_de", C.c_double),
                ("x_star", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int64), ("rejections", C.c_int64), ("final_m", C.c_int64), ("a_passes", C.c_int64),
                ("sketch_passes", C.c_int64), ("factorizations", C.c_int64), ("outer_iters", C.c_int64),
                ("final_delta_tilde", C.c_double), ("est_rel_err", C.c_double), ("trace_len", C.c_int64),
                ("ms_total", C.c_float), ("ms_sketch", C.c_float), ("ms_factor", C.c_float),
                ("ms_iter", C.c_float), ("ms_apass", C.c_float), ("apass_timed", C.c_int64),
                ("status", C.c_int), ("sketch_e4m3", C.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class BatchInfo(C.Structure):
    _fields_ = [("rounds", C.c_int64), ("kernels_per_round", C.c_int64), ("rows_per_unit", C.c_int64),
                ("ms_setup", C.c_float), ("ms_autotune", C.c_float), ("ms_solve", C.c_float),
                ("ms_apass", C.c_float), ("apass_flops", C.c_double), ("ms_gram", C.c_float),
                ("gram_flops", C.c_double), ("ms_factor", C.c_float), ("ms_apply", C.c_float),
                ("ms_rounds", C.c_float)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


P = C.POINTER
_SIGS = {
    "sks_opts_default": (None, [P(Opts)]),
    "sks_version": (C.c_char_p, []),
    "sks_last_error": (C.c_char_p, []),
    "sks_kernel_launch_count": (C.c_uint64, []),
    "sks_hess_apply_workspace_size": (C.c_int, [P(Problem), P(C.c_size_t)]),
    "sks_hess_apply": (C.c_int, [P(Problem), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p]),
    "sks_hess_apply_noalloc": (C.c_int, [P(Problem), C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "sks_sketch_workspace_size": (C.c_int, [P(Problem), C.c_int, C.c_int64, C.c_int, P(C.c_size_t)]),
    "sks_sketch_create": (C.c_int, [P(C.c_void_p), P(Problem), C.c_int, C.c_int64, C.c_int64, C.c_int, C.c_uint64,
                                    C.c_void_p, C.c_size_t, C.c_void_p]),
    "sks_sketch_grow": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "sks_sketch_rows": (C.c_int, [C.c_void_p, P(C.c_int64)]),
    "sks_sketch_copy_out": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sks_sketch_destroy": (None, [C.c_void_p]),
    "sks_precond_workspace_size": (C.c_int, [P(Problem), C.c_int64, P(C.c_size_t)]),
    "sks_precond_build": (C.c_int, [P(C.c_void_p), C.c_void_p, P(Problem), C.c_void_p, C.c_size_t, C.c_void_p]),
    "sks_precond_build_ex": (C.c_int, [P(C.c_void_p), C.c_void_p, P(Problem), C.c_int, C.c_void_p, C.c_size_t,
                                       C.c_void_p]),
    "sks_precond_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "sks_precond_destroy": (None, [C.c_void_p]),
    "sks_solve_workspace_size": (C.c_int, [P(Problem), P(Opts), P(C.c_size_t)]),
    "sks_adaptive_pcg_solve": (C.c_int, [P(Problem), P(Opts), C.c_void_p, P(Stats), C.c_void_p, C.c_size_t,
                                         C.c_void_p]),
    "sks_adaptive_ihs_solve": (C.c_int, [P(Problem), P(Opts), C.c_void_p, P(Stats), C.c_void_p, C.c_size_t,
                                         C.c_void_p]),
    "sks_dual_workspace_size": (C.c_int, [P(Problem), P(Opts), P(C.c_size_t)]),
    "sks_dual_pcg_solve": (C.c_int, [P(Problem), P(Opts), C.c_void_p, P(Stats), C.c_void_p, C.c_size_t,
                                     C.c_void_p]),
    "sks_dual_ihs_solve": (C.c_int, [P(Problem), P(Opts), C.c_void_p, P(Stats), C.c_void_p, C.c_size_t,
                                     C.c_void_p]),
    "sks_fixed_solve": (C.c_int, [C.c_int, P(Problem), P(Opts), C.c_void_p, P(Stats), C.c_void_p, C.c_size_t,
                                  C.c_void_p]),
    "sks_adjoint": (C.c_int, [P(Problem), P(Opts), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                              P(C.c_double), C.c_void_p, P(Stats), C.c_void_p, C.c_size_t, C.c_void_p]),
    "sks_selftest_wait_timeout": (C.c_int, [C.c_int64, C.c_void_p]),
    "sks_batch_workspace_size": (C.c_int, [P(Problem), C.c_int, P(Opts), P(C.c_size_t)]),
    "sks_solve_batched": (C.c_int, [P(Problem), C.c_int, P(Opts), P(C.c_void_p), P(Stats), P(BatchInfo), C.c_int,
                                    C.c_void_p, C.c_size_t, C.c_void_p]),
    "sks_batch_create": (C.c_int, [P(C.c_void_p), P(Problem), C.c_int, P(Opts), C.c_int, C.c_void_p, C.c_size_t,
                                    C.c_void_p]),
    "sks_batch_solve": (C.c_int, [C.c_void_p, P(C.c_void_p), P(Stats), P(BatchInfo), C.c_void_p]),
    "sks_batch_destroy": (None, [C.c_void_p]),
}

EXPORTED = tuple(_SIGS)

_lib = None


class SksError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def load(path=LIB_PATH):
    """Load libsks.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libsks.so not built (%s); run paper_2104_14101_gb300.build.build()" % path)
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status):
    if status != OK:
        raise SksError(status, load().sks_last_error().decode())
    return status
