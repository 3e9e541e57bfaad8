"""Shared helpers of the GPU parity tests: move seeded synthetic problems to
the device and compare against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_14101_gb300 import build
    build.build()


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_err_vec(got, ref, scale):
    """max_i |got_i - ref_i| / scale_i."""
    return float(np.max(np.abs(got - ref) / scale))
