"""The allocation-free Hessian pass (sks_hess_apply_noalloc).

It serves callers that may not allocate device memory when they need H x, so
they cannot pass the workspace the regular entry point asks for; its scratch
is a library-owned static device array.  This file is collected last so that
a failure here leaves every other test already run.  It must pass both alone
in a fresh process and after the rest of the suite.
"""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


def _call_both(A, x, nu, lam, extended):
    from paper_2104_14101_gb300 import _lib as L
    from paper_2104_14101_gb300.api import make_problem
    lib = L.load()
    tA = A
    p, keep = make_problem(tA, x, nu, lam)
    xcm = x.t().contiguous() if x.dim() == 2 else x[None, :].contiguous()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the existing entry point, with a caller workspace
    nb = C.c_size_t()
    L.check(lib.sks_hess_apply_workspace_size(C.byref(p), C.byref(nb)))
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    y_ref = torch.empty_like(xcm)
    L.check(lib.sks_hess_apply(C.byref(p), C.c_void_p(xcm.data_ptr()), C.c_void_p(y_ref.data_ptr()), extended,
                               C.c_void_p(ws.data_ptr()), nb.value, stream))
    # the allocation-free variant, twice in a row
    outs = []
    for _ in range(2):
        y = torch.full_like(xcm, float("nan"))
        L.check(lib.sks_hess_apply_noalloc(C.byref(p), C.c_void_p(xcm.data_ptr()), C.c_void_p(y.data_ptr()),
                                           extended, stream))
        outs.append(y)
    torch.cuda.synchronize()
    return host(y_ref), [host(o) for o in outs]


@pytest.mark.parametrize("n,d,dtype,extended", [
    (5000, 2048, torch.float64, 0), (3001, 256, torch.float64, 0), (4000, 4096, torch.float32, 0),
    (1000, 33, torch.float32, 1), (0, 17, torch.float64, 0),
    # wide rows (d > 4096) and rows whose byte length is not a 16-byte multiple (tiled copies)
    (333, 9000, torch.float32, 0), (700, 4100, torch.float64, 0), (501, 4099, torch.float32, 0)])
def test_noalloc_matches_workspace_entry_point(n, d, dtype, extended):
    require_gpu()
    rng = np.random.default_rng(n + d)
    A = dev(rng.standard_normal((n, d)), dtype)
    x = dev(rng.standard_normal(d))
    lam = dev(1 + rng.random(d))
    y_ref, (y1, y2) = _call_both(A, x, 0.3, lam, extended)
    An = host(A).astype(np.float64)
    scale = np.abs(An).T @ (np.abs(An) @ np.abs(host(x))) + 0.09 * host(lam) * np.abs(host(x)) + 1e-300
    tol = 1e-5 if (dtype == torch.float32 and not extended) else 1e-13
    for y in (y1, y2):
        assert np.all(np.isfinite(y))
        assert float(np.max(np.abs(y[0] - y_ref[0]) / scale)) < tol


def test_noalloc_rejects_oversized_problem():
    require_gpu()
    from paper_2104_14101_gb300 import _lib as L
    from paper_2104_14101_gb300.api import make_problem
    lib = L.load()
    rng = np.random.default_rng(0)
    d = 1024
    A = dev(rng.standard_normal((4096, d)))  # enough rows for a full grid of 152 blocks
    X = dev(rng.standard_normal((d, 8)))  # 8 float64 right-hand sides: ~10 MB of partial sums
    p, keep = make_problem(A, X, 0.3, dev(1 + rng.random(d)))
    xcm = X.t().contiguous()
    y = torch.empty_like(xcm)
    st = lib.sks_hess_apply_noalloc(C.byref(p), C.c_void_p(xcm.data_ptr()), C.c_void_p(y.data_ptr()), 0,
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == L.ERR_INVALID_ARG
    assert b"at most" in lib.sks_last_error()
