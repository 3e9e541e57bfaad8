"""GPU parity of the dual formulation (eq. 2) through the C ABI: problems with
more columns than rows solved through their n x n dual, the primal solution
recovered on the device, against the oracle's direct primal solve."""
import numpy as np
import pytest

from oracle import solvers as O
from tests.gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def api():
    import paper_2104_14101_gb300 as sks
    return sks


def wide_problem(n, d, nu, seed, k=1):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, d)) * (1.0 / (1.0 + np.arange(d)))[None, :]
    lam = 1 + 9 * rng.random(d)
    b = rng.standard_normal((d, k)) if k > 1 else rng.standard_normal(d)
    return A, b, nu, lam


@pytest.mark.parametrize("method,kind", [("pcg", "srht"), ("pcg", "gaussian"), ("pcg", "sjlt"), ("ihs", "srht")])
def test_dual_solve_matches_primal_oracle(method, kind):
    # n = 600 < d = 2000 (ragged: the dual data matrix is 2000 x 600, its rows padded to 16 bytes)
    A, b, nu, lam = wide_problem(600, 2000, 1e-2, 1)
    xs = O.direct_solve(A, b, nu, lam)
    x, st = api().dual_solve(dev(A), dev(b), nu, dev(lam), method=method, kind=kind, m_init=1, tol=1e-12,
                             sjlt_s=2, seed=3)
    assert st["status_name"] == "OK"
    assert O.rel_err_H(A, nu, lam, host(x), xs) <= 1e-8


def test_dual_error_bound_and_multiple_rhs():
    # ||x - x*||_H <= ||H_dual (w - w*)|| / nu^2, with w recovered from x on the host
    # (w solves A^T w = b - nu^2 Lambda x; A has full row rank)
    A, b, nu, lam = wide_problem(300, 1100, 3e-2, 2, k=2)
    xs = O.direct_solve(A, b, nu, lam)
    x, st = api().dual_solve(dev(A), dev(b), nu, dev(lam), kind="gaussian", tol=1e-6, seed=1)
    x = host(x)
    D, bd, _, lamd = O.dual_problem(A, b, nu, lam)
    ws = O.direct_solve(D, bd, nu, lamd)
    Hd = D.T @ D + nu ** 2 * np.eye(A.shape[0])
    for c in range(2):
        w = np.linalg.lstsq(A.T, b[:, c] - nu ** 2 * lam * x[:, c], rcond=None)[0]
        e = x[:, c] - xs[:, c]
        err_H = np.sqrt(e @ O.hess_apply(A, nu, lam, e))
        assert err_H <= np.linalg.norm(Hd @ (w - ws[:, c])) / nu ** 2 * (1 + 1e-6) + 1e-12
        assert O.rel_err_H(A, nu, lam, x[:, c], xs[:, c]) <= 1e-3


def test_dual_mixed_form():
    # float32 A through the dual (mixed form, refined).  With Lambda = I the
    # dual matrix A^T is exact in float32 and the primal error follows the
    # dual tolerance; with Lambda != I the float32 Lambda^{-1/2} A^T is rounded
    # (2^-24 per entry), which the oracle reproduces: the float64 solve of that
    # rounded dual, mapped back, is as far from x* as the GPU result.
    A, b, nu, lam = wide_problem(800, 3000, 1e-2, 4)
    A = A.astype(np.float32).astype(np.float64)
    one = np.ones_like(lam)
    xs = O.direct_solve(A, b, nu, one)
    x, st = api().dual_solve(dev(A, torch.float32), dev(b), nu, dev(one), kind="srht", tol=1e-10,
                             precision="mixed", seed=2)
    assert O.rel_err_H(A, nu, one, host(x), xs) <= 1e-8
    xs = O.direct_solve(A, b, nu, lam)
    x, st = api().dual_solve(dev(A, torch.float32), dev(b), nu, dev(lam), kind="srht", tol=1e-10,
                             precision="mixed", seed=2)
    D32 = (A / np.sqrt(lam)[None, :]).T.astype(np.float32).astype(np.float64)
    w = np.linalg.solve(D32.T @ D32 + nu ** 2 * np.eye(A.shape[0]), A @ (b / lam))
    x_rounded = (b - np.sqrt(lam) * (D32 @ w)) / (nu ** 2 * lam)
    e_ref = O.rel_err_H(A, nu, lam, x_rounded, xs)
    assert O.rel_err_H(A, nu, lam, host(x), xs) <= 1.5 * e_ref + 1e-8


def test_dual_ihs_at_the_sketch_cap_diverges_like_the_oracle():
    # Adaptive IHS with the Gaussian embedding on this dual (2000 rows) reaches
    # the cap m = 2000 while the step mu = 1 - rho still overshoots; at the cap
    # a failing test accepts the step (reading R10), the iterates blow up, and
    # the oracle's float64 run ends in non-finite values too.  The GPU reports
    # NUMERIC instead of returning garbage.
    from paper_2104_14101_gb300._lib import SksError
    A, b, nu, lam = wide_problem(600, 2000, 1e-2, 1)
    D, bd, _, lamd = O.dual_problem(A, b, nu, lam)
    with pytest.raises((ValueError, FloatingPointError)):
        with np.errstate(all="ignore"):
            O.adaptive_ihs(D, bd, nu, lamd, kind="gaussian", seed=3, m_init=1, tol=1e-12)
    with pytest.raises(SksError) as e:
        api().dual_solve(dev(A), dev(b), nu, dev(lam), method="ihs", kind="gaussian", m_init=1, tol=1e-12, seed=3)
    assert "NUMERIC" in str(e.value)
