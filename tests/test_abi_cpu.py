"""The C-ABI library builds and exports every entry point include/*.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(sks_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2104_14101_gb300 import build
    try:
        return build.build()
    except RuntimeError as e:  # no nvcc in this environment
        pytest.skip(str(e))


def test_header_declares_entry_points():
    names = declared_functions()
    for expected in ("sks_adaptive_pcg_solve", "sks_adaptive_ihs_solve", "sks_sketch_create", "sks_precond_build",
                     "sks_hess_apply"):
        assert expected in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(lib_path):
    from paper_2104_14101_gb300 import _lib
    lib = _lib.load(lib_path)
    assert set(declared_functions()) <= set(_lib.EXPORTED)
    assert lib.sks_version().decode().startswith("sks")


def test_opts_default_and_validation_without_gpu(lib_path):
    # Host-side argument checks return a status without touching the GPU.
    from paper_2104_14101_gb300 import _lib
    lib = _lib.load(lib_path)
    o = _lib.Opts()
    lib.sks_opts_default(ctypes.byref(o))
    assert o.rho == 0.125 and o.m_init == 1 and o.reuse_residual == 1 and o.max_outer == 20
    assert o.stop_rule == 0 and o.cert_delta == 0.01 and o.cert_de == 0.0
    p = _lib.Problem()
    p.dtype, p.n, p.d, p.lda, p.k = _lib.F64, 10, 4, 2, 1  # lda < d
    nb = ctypes.c_size_t()
    assert lib.sks_solve_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(nb)) == _lib.ERR_INVALID_ARG
    assert b"lda" in lib.sks_last_error()
    p.lda, p.nu = 4, -1.0
    p.A, p.b, p.lambda_diag = 16, 16, 16  # never dereferenced: rejected first
    assert lib.sks_solve_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(nb)) == _lib.ERR_INVALID_ARG
    p.nu = 1e-2
    p.lda = 5  # 40 bytes: not a multiple of 16
    assert lib.sks_solve_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(nb)) == _lib.ERR_INVALID_ARG
    p.lda = 4
    assert lib.sks_solve_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(nb)) == _lib.OK
    assert nb.value > 0


def test_batched_validation_without_gpu(lib_path):
    # The batched entry point rejects what it does not implement before any
    # device work: no problems, float32 A in the plain form (float64 A in the
    # mixed form), another embedding, d > 1024.
    from paper_2104_14101_gb300 import _lib
    lib = _lib.load(lib_path)
    o = _lib.Opts()
    lib.sks_opts_default(ctypes.byref(o))
    arr = (_lib.Problem * 2)()
    for p in arr:
        p.dtype, p.n, p.d, p.lda, p.k, p.nu = _lib.F64, 64, 8, 8, 1, 1e-2
        p.A, p.b, p.lambda_diag = 16, 16, 16  # never dereferenced
    nb = ctypes.c_size_t()
    assert lib.sks_batch_workspace_size(arr, 0, ctypes.byref(o), ctypes.byref(nb)) == _lib.ERR_INVALID_ARG
    assert lib.sks_batch_workspace_size(arr, 2, ctypes.byref(o), ctypes.byref(nb)) == _lib.OK
    # H E A_pad (64 x 8), factor (8 x 8), perm and vectors of both problems at least
    assert nb.value > 2 * 8 * (64 * 8 + 8 * 8 + 10 * 8)
    arr[1].dtype = _lib.F32
    assert lib.sks_batch_workspace_size(arr, 2, ctypes.byref(o), ctypes.byref(nb)) == _lib.ERR_INVALID_ARG
    assert b"problem 1" in lib.sks_last_error()
    arr[1].dtype = _lib.F64
    arr[0].d, arr[0].lda = 1032, 1032
    assert lib.sks_batch_workspace_size(arr, 2, ctypes.byref(o), ctypes.byref(nb)) == _lib.ERR_UNSUPPORTED
    arr[0].d, arr[0].lda = 8, 8
    o.kind = _lib.KINDS["gaussian"]
    assert lib.sks_batch_workspace_size(arr, 2, ctypes.byref(o), ctypes.byref(nb)) == _lib.ERR_UNSUPPORTED
    o.kind = _lib.KINDS["srht"]
    arr[1].k = 2
    assert lib.sks_batch_workspace_size(arr, 2, ctypes.byref(o), ctypes.byref(nb)) == _lib.ERR_UNSUPPORTED
    arr[1].k = 1
    # the mixed form: float32 A only; its layout holds the float32 H E A_pad,
    # the factor as float pairs and the block inverses instead of float64 copies
    o.precision = _lib.MIXED_REFINED
    assert lib.sks_batch_workspace_size(arr, 2, ctypes.byref(o), ctypes.byref(nb)) == _lib.ERR_INVALID_ARG
    assert b"mixed form needs float32 A" in lib.sks_last_error()
    arr[0].dtype = arr[1].dtype = _lib.F32
    assert lib.sks_batch_workspace_size(arr, 2, ctypes.byref(o), ctypes.byref(nb)) == _lib.OK
    assert nb.value > 2 * (64 * 8 * 4 + 8 * 8 * 8 + 64 * 64 * 8)
    o.max_outer = 0
    assert lib.sks_batch_workspace_size(arr, 2, ctypes.byref(o), ctypes.byref(nb)) == _lib.ERR_INVALID_ARG


def test_new_entry_points_validation_without_gpu(lib_path):
    # Host-side checks of the non-adaptive solvers, the certified stop rule and
    # the dual formulation return a status before any device work.
    from paper_2104_14101_gb300 import _lib
    lib = _lib.load(lib_path)
    o = _lib.Opts()
    lib.sks_opts_default(ctypes.byref(o))
    p = _lib.Problem()
    p.dtype, p.n, p.d, p.lda, p.k, p.nu = _lib.F64, 100, 300, 300, 1, 1e-2
    p.A, p.b, p.lambda_diag = 16, 16, 16  # never dereferenced
    x = ctypes.c_void_p(16)
    st = _lib.Stats()
    # an unknown fixed-sketch method
    assert lib.sks_fixed_solve(9, ctypes.byref(p), ctypes.byref(o), x, ctypes.byref(st), None, 0, None) == \
        _lib.ERR_INVALID_ARG
    # CG has no preconditioner: no mixed form, no certified stop
    o.precision = _lib.MIXED_REFINED
    p.dtype = _lib.F32
    assert lib.sks_fixed_solve(3, ctypes.byref(p), ctypes.byref(o), x, ctypes.byref(st), None, 0, None) == \
        _lib.ERR_UNSUPPORTED
    o.precision, p.dtype = _lib.PLAIN_F64, _lib.F64
    o.stop_rule = _lib.STOP_RULES["certified"]
    assert lib.sks_fixed_solve(3, ctypes.byref(p), ctypes.byref(o), x, ctypes.byref(st), None, 0, None) == \
        _lib.ERR_UNSUPPORTED
    # certified rule: delta in (0, 1), d_e >= 0; unknown rules rejected
    o.cert_delta = 1.5
    assert lib.sks_adaptive_pcg_solve(ctypes.byref(p), ctypes.byref(o), x, ctypes.byref(st), None, 0, None) == \
        _lib.ERR_INVALID_ARG
    o.cert_delta, o.stop_rule = 0.01, 7
    assert lib.sks_adaptive_pcg_solve(ctypes.byref(p), ctypes.byref(o), x, ctypes.byref(st), None, 0, None) == \
        _lib.ERR_INVALID_ARG
    o.stop_rule = 0
    # dual formulation of this 100 x 300 problem: the workspace holds the 300 x 100 dual matrix
    nb = ctypes.c_size_t()
    assert lib.sks_dual_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(nb)) == _lib.OK
    assert nb.value > 300 * 100 * 8
    assert lib.sks_dual_pcg_solve(ctypes.byref(p), ctypes.byref(o), x, ctypes.byref(st), None, 0, None) == \
        _lib.ERR_WORKSPACE
    # the batch stops by the estimate rule only
    o.stop_rule = _lib.STOP_RULES["certified"]
    arr = (_lib.Problem * 1)(p)
    arr[0].n, arr[0].d, arr[0].lda = 64, 8, 8
    assert lib.sks_batch_workspace_size(arr, 1, ctypes.byref(o), ctypes.byref(nb)) == _lib.ERR_UNSUPPORTED
