"""GPU parity of the non-adaptive solvers (the baselines of Section 6 and the
Polyak-IHS of Appendix A) through the C ABI: the T-th iterate of each method
against the oracle's iteration with the same sketch, and solves to tolerance."""
import numpy as np
import pytest

import synthetic
from oracle import sketch as OS
from oracle import solvers as O
from tests.gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def api():
    import paper_2104_14101_gb300 as sks
    return sks


def _h_rel(p, x, ref):
    return O.rel_err_H(p.A, p.nu, p.lam, x, ref)


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
@pytest.mark.parametrize("method", ["fixed-pcg", "fixed-ihs", "polyak-ihs"])
@pytest.mark.parametrize("m_factor", [2.0, 0.5])  # m = 2d (Cholesky form), m = d/2 (Woodbury form)
def test_fixed_iterates_match_oracle(method, kind, m_factor):
    p = synthetic.make_problem("C1", 3, n=2048, d=96, nu=1e-2, decay="harmonic", lam="one_plus_9u")
    m = int(m_factor * p.d)
    SA = OS.sketch(kind, p.A, m, 7)
    rho = 0.125
    if method == "polyak-ihs":
        # the step size and momentum of Corollary A.2 assume the event E_rho: take rho from C_S
        ev = O.cs_eigenvalues(p.A, SA, p.nu, p.lam)
        rho = min(0.95, 1.05 * float(np.max(np.abs(ev - 1.0))) ** 2)
    P = O.Preconditioner(SA, p.nu, p.lam)
    T = 6
    x0 = np.zeros(p.d)
    if method == "fixed-pcg":
        ref = O.pcg(p.A, p.b, p.nu, p.lam, P, x0, T)[-1]
    elif method == "fixed-ihs":
        ref = O.ihs(p.A, p.b, p.nu, p.lam, P, x0, T, 1.0 - rho)[-1]
    else:
        ref = O.polyak_ihs(p.A, p.b, p.nu, p.lam, P, x0, T, rho)[-1]
    x, st, _ = api().fixed_solve(dev(p.A), dev(p.b), p.nu, dev(p.lam), method=method, kind=kind, m_init=m,
                                 rho=rho, tol=1e-30, max_iter=T, seed=7, check=False)
    assert st["status_name"] == "NO_CONVERGENCE" and st["iters"] == T
    assert st["final_m"] == m and st["rejections"] == 0 and st["factorizations"] == 1
    assert _h_rel(p, host(x), ref) <= 1e-10


def test_cg_iterates_match_oracle():
    p = synthetic.make_problem("C1", 4, n=1024, d=64, nu=1e-1)
    T = 12
    ref = O.cg(p.A, p.b, p.nu, p.lam, np.zeros(p.d), T)[-1]
    x, st, _ = api().fixed_solve(dev(p.A), dev(p.b), p.nu, dev(p.lam), method="cg", tol=1e-30, max_iter=T,
                                 check=False)
    assert st["iters"] == T and st["final_m"] == 0 and st["sketch_passes"] == 0
    assert _h_rel(p, host(x), ref) <= 1e-9


def test_fixed_pcg_2d_reaches_tolerance_plain():
    # the paper's PCG baseline: m = 2d, plain float64, to 1e-10
    p = synthetic.make_problem("C1", 0, n=4096, d=256, nu=1e-2)
    xs = O.direct_solve(p.A, p.b, p.nu, p.lam)
    x, st, _ = api().fixed_solve(dev(p.A), dev(p.b), p.nu, dev(p.lam), method="fixed-pcg", kind="srht",
                                 m_init=2 * p.d, tol=1e-10)
    assert st["status_name"] == "OK" and st["final_m"] == 2 * p.d
    assert _h_rel(p, host(x), xs) <= 1e-10


def test_cg_reaches_residual_tolerance():
    p = synthetic.make_problem("C1", 0, n=2048, d=128, nu=1e-1)
    x, st, _ = api().fixed_solve(dev(p.A), dev(p.b), p.nu, dev(p.lam), method="cg", tol=1e-10, max_iter=5000)
    r = p.b - O.hess_apply(p.A, p.nu, p.lam, host(x))
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(p.b) * 1.01
    assert st["est_rel_err"] <= 1e-10


@pytest.mark.parametrize("method,m_mult,rho", [("fixed-pcg", 2, 0.125), ("polyak-ihs", 8, 0.65)])
def test_fixed_mixed_form_reaches_1e8(method, m_mult, rho):
    # mixed form: float32 A, SJLT s = 4, float64 refinement.  Polyak-IHS needs
    # the event E_rho: at m = 8d the oracle's C_S spectrum is [0.43, 1.78], so rho = 0.65.
    p = synthetic.make_problem("C3", 0, n=8192, d=256, nu=1e-3)
    xs = O.direct_solve(p.A, p.b, p.nu, p.lam)
    x, st, _ = api().fixed_solve(dev(p.A, torch.float32), dev(p.b), p.nu, dev(p.lam), method=method, kind="sjlt",
                                 sjlt_s=4, m_init=m_mult * p.d, rho=rho, tol=1e-8, precision="mixed", max_iter=3000,
                                 seed=0)
    assert _h_rel(p, host(x), xs) <= 1e-8, st
    assert st["outer_iters"] >= 1 and st["rejections"] == 0


def test_cg_mixed_is_unsupported_and_zero_rhs():
    p = synthetic.make_problem("C3", 0, n=1024, d=64)
    from paper_2104_14101_gb300._lib import SksError
    with pytest.raises(SksError) as e:
        api().fixed_solve(dev(p.A, torch.float32), dev(p.b), p.nu, dev(p.lam), method="cg", precision="mixed")
    assert "UNSUPPORTED" in str(e.value)
    q = synthetic.make_problem("C1", 0, n=512, d=32)
    for method in ("cg", "fixed-pcg", "polyak-ihs"):
        x, st, _ = api().fixed_solve(dev(q.A), dev(np.zeros(32)), q.nu, dev(q.lam), method=method, m_init=64)
        assert float(torch.abs(x).max()) == 0.0 and st["iters"] == 0
