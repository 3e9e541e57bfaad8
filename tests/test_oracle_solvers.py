"""Pins of the oracle's solvers against closed forms and the paper's theorems.

Closed forms: x* = V diag(sigma/(sigma^2+nu^2)) U^T y for A = U diag(sigma) V^T,
Lambda = I, b = A^T y; the Woodbury identity; d_e from sigma.  Theorems:
Lemma 2.1 (delta vs delta~), Theorem 3.2 (IHS rate), eq. (11) (PCG rate),
Lemma 3.1 / Theorem 3.3 (PCG attains the polynomial lower bound, hence beats
IHS), Theorem 4.1 (adaptive sketch-size ceiling), Table 3 (Polyak-IHS bound).
"""
import math
import os

import numpy as np
import pytest

import synthetic
from oracle import sketch as SK
from oracle import solvers as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_problem(n=512, d=24, nu=1e-2, decay="geom0.9", seed=0, lam="identity"):
    return synthetic.make_problem("C1", seed, n=n, d=d, nu=nu, decay=decay, lam=lam)


def closed_form_xstar(p):
    return p.V @ ((p.sigma / (p.sigma ** 2 + p.nu ** 2)) * (p.U.T @ p.y))


def test_direct_solve_closed_form():
    p = synthetic.make_problem("C1", 0)
    xs = S.direct_solve(p.A, p.b, p.nu, p.lam)
    assert S.rel_err_H(p.A, p.nu, p.lam, xs, closed_form_xstar(p)) < 1e-12


def test_direct_solve_general_lambda():
    # H = V diag(sigma^2) V^T + nu^2 Lambda needs neither n nor U.
    p = synthetic.make_problem("C2", 1, n=1024, d=64)
    H = (p.V * p.sigma ** 2) @ p.V.T + p.nu ** 2 * np.diag(p.lam)
    xc = np.linalg.solve(H, p.b)
    xs = S.direct_solve(p.A, p.b, p.nu, p.lam)
    assert S.rel_err_H(p.A, p.nu, p.lam, xs, xc) < 1e-10


def test_h_norm_matches_quadratic_form():
    p = small_problem()
    e = np.random.default_rng(3).standard_normal(p.d)
    H = S.hessian(p.A, p.nu, p.lam)
    assert math.isclose(S.h_norm_sq(p.A, p.nu, p.lam, e), e @ H @ e, rel_tol=1e-12)


def test_objective_gap_is_delta():
    # f(x) - f(x*) = 1/2 ||x - x*||_H^2 = delta_x (Section 1.1)
    p = small_problem()
    xs = S.direct_solve(p.A, p.b, p.nu, p.lam)
    x = xs + np.random.default_rng(1).standard_normal(p.d) * 1e-2
    gap = S.objective(p.A, p.b, p.nu, p.lam, x) - S.objective(p.A, p.b, p.nu, p.lam, xs)
    assert math.isclose(gap, 0.5 * S.h_norm_sq(p.A, p.nu, p.lam, x - xs), rel_tol=1e-8)


@pytest.mark.parametrize("m", [1, 5, 23, 24, 40])
def test_preconditioner_solves_HS(m):
    p = small_problem(lam="one_plus_9u")
    SA = SK.sketch("gaussian", p.A, m, seed=2)
    P = S.Preconditioner(SA, p.nu, p.lam)
    assert P.woodbury == (m < p.d)
    HS = SA.T @ SA + p.nu ** 2 * np.diag(p.lam)
    z = np.random.default_rng(m).standard_normal((p.d, 2))
    v = P.apply(z)
    ref = np.linalg.inv(HS) @ z
    assert np.allclose(v, ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())


def test_effective_dimension_closed_form():
    p = synthetic.make_problem("C1", 0)
    w = p.sigma ** 2 / (p.sigma ** 2 + p.nu ** 2)
    assert math.isclose(S.effective_dimension(p.A, p.nu, p.lam), w.sum() / w.max(), rel_tol=1e-9)
    assert 90.0 < w.sum() / w.max() < 90.6


def _frac_solve(M, z):
    """Exact Gauss-Jordan elimination over the rationals."""
    from fractions import Fraction
    n = len(M)
    aug = [[Fraction(v) for v in row] + [Fraction(zi)] for row, zi in zip(M, z)]
    for c in range(n):
        piv = next(r for r in range(c, n) if aug[r][c] != 0)
        aug[c], aug[piv] = aug[piv], aug[c]
        for r in range(n):
            if r != c and aug[r][c] != 0:
                f = aug[r][c] / aug[c][c]
                aug[r] = [a - f * b for a, b in zip(aug[r], aug[c])]
    return [aug[i][n] / aug[i][i] for i in range(n)]


def test_pcg_exact_in_d_steps_rational():
    # In exact arithmetic PCG (eq. 5) reaches x* in at most d steps.  Run the
    # recursion over the rationals on a tiny instance (inputs rounded to
    # dyadic rationals) and compare the float64 oracle with it step by step.
    from fractions import Fraction
    rng = np.random.default_rng(4)
    n, d, m = 12, 5, 3
    A = np.round(rng.standard_normal((n, d)) * 64) / 64
    b = np.round(rng.standard_normal(d) * 64) / 64
    lam = 1 + np.round(rng.random(d) * 8) / 8
    nu = 0.5
    SA = np.round(rng.standard_normal((m, d)) * 64) / 64
    F = Fraction
    Af = [[F(v) for v in row] for row in A]
    H = [[sum(Af[k][i] * Af[k][j] for k in range(n)) + (F(nu) ** 2 * F(lam[i]) if i == j else 0)
          for j in range(d)] for i in range(d)]
    HS = [[sum(F(SA[k][i]) * F(SA[k][j]) for k in range(m)) + (F(nu) ** 2 * F(lam[i]) if i == j else 0)
           for j in range(d)] for i in range(d)]
    xstar = _frac_solve(H, [F(v) for v in b])
    mv = lambda M, v: [sum(M[i][j] * v[j] for j in range(d)) for i in range(d)]
    dot = lambda u, v: sum(a * c for a, c in zip(u, v))
    x = [F(0)] * d
    r = [F(v) for v in b]
    rt = _frac_solve(HS, r)
    pv = list(rt)
    dt = dot(r, rt)
    exact = [list(x)]
    for _ in range(d):
        Hp = mv(H, pv)
        al = dt / dot(pv, Hp)
        x = [a + al * c for a, c in zip(x, pv)]
        r = [a - al * c for a, c in zip(r, Hp)]
        rt = _frac_solve(HS, r)
        dn = dot(r, rt)
        pv = [a + (dn / dt) * c for a, c in zip(rt, pv)]
        dt = dn
        exact.append(list(x))
    assert exact[-1] == xstar  # exact termination in d steps
    P = S.Preconditioner(SA, nu, lam)
    it = S.pcg(A, b, nu, lam, P, np.zeros(d), d)
    for t in range(d + 1):
        ex = np.array([float(v) for v in exact[t]])
        assert np.allclose(it[t], ex, rtol=1e-9, atol=1e-12 * np.abs(ex).max() + 1e-300)


def test_exact_preconditioner_one_step():
    # SRHT with m = n_pad gives H_S = H: PCG and IHS(mu=1) converge in one step.
    p = small_problem(n=128, d=8)
    xs = S.direct_solve(p.A, p.b, p.nu, p.lam)
    SA = SK.sketch("srht", p.A, 128, seed=3)
    P = S.Preconditioner(SA, p.nu, p.lam)
    assert np.allclose(P.matrix(), S.hessian(p.A, p.nu, p.lam), atol=1e-12)
    x1 = S.pcg(p.A, p.b, p.nu, p.lam, P, np.zeros(p.d), 1)[1]
    assert S.rel_err_H(p.A, p.nu, p.lam, x1, xs) < 1e-10
    x1 = S.ihs(p.A, p.b, p.nu, p.lam, P, np.zeros(p.d), 1, mu=1.0)[1]
    assert S.rel_err_H(p.A, p.nu, p.lam, x1, xs) < 1e-10


def _delta(p, x, xs):
    return 0.5 * S.h_norm_sq(p.A, p.nu, p.lam, x - xs)


def test_lemma_2_1_newton_decrement():
    p = small_problem()
    xs = S.direct_solve(p.A, p.b, p.nu, p.lam)
    SA = SK.sketch("gaussian", p.A, 400, seed=5)
    lam_cs = S.cs_eigenvalues(p.A, SA, p.nu, p.lam)
    rho = max(abs(lam_cs[0] - 1), abs(lam_cs[-1] - 1)) ** 2
    assert rho < 1
    P = S.Preconditioner(SA, p.nu, p.lam)
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = xs + rng.standard_normal(p.d)
        g = S.hess_apply(p.A, p.nu, p.lam, x) - p.b
        dtil = 0.5 * g @ P.apply(g)
        assert abs(_delta(p, x, xs) - dtil) <= math.sqrt(rho) * dtil * (1 + 1e-9)


def test_rate_constants_from_eigenvalue_interval():
    # On E_rho the eigenvalues of C_S lie in [1 - sqrt rho, 1 + sqrt rho].
    for rho in (0.01, 0.125, 0.2):
        lo, hi = 1 - math.sqrt(rho), 1 + math.sqrt(rho)
        # IHS with mu = 1 - rho contracts by max |1 - mu/lambda|^2 = rho (Thm 3.2)
        phi_ihs, c_ihs = S.ihs_constants(rho)
        mu = 1 - rho
        assert math.isclose(max((1 - mu / lo) ** 2, (1 - mu / hi) ** 2), phi_ihs, rel_tol=1e-12)
        # PCG: Chebyshev rate ((sqrt k - 1)/(sqrt k + 1))^2 with k = hi/lo (eq. 11)
        kap = hi / lo
        phi_pcg, c_pcg = S.pcg_constants(rho)
        assert math.isclose(((math.sqrt(kap) - 1) / (math.sqrt(kap) + 1)) ** 2, phi_pcg, rel_tol=1e-12)
        # c(alpha, rho) = alpha * (upper/lower Lemma 2.1 factors) = alpha * hi / lo
        assert math.isclose(c_ihs, 1 * hi / lo, rel_tol=1e-12)
        assert math.isclose(c_pcg, 4 * hi / lo, rel_tol=1e-12)


def test_theorem_3_2_and_eq_11_rates():
    p = small_problem(n=2048, d=32, nu=1e-3)
    xs = S.direct_solve(p.A, p.b, p.nu, p.lam)
    SA = SK.sketch("srht", p.A, 1024, seed=7)
    ev = S.cs_eigenvalues(p.A, SA, p.nu, p.lam)
    rho = max(abs(ev[0] - 1), abs(ev[-1] - 1)) ** 2
    assert rho < 0.25
    P = S.Preconditioner(SA, p.nu, p.lam)
    x0 = np.zeros(p.d)
    d0 = _delta(p, x0, xs)
    it = S.ihs(p.A, p.b, p.nu, p.lam, P, x0, 8, mu=1 - rho)
    for t, x in enumerate(it):
        assert _delta(p, x, xs) <= rho ** t * d0 * (1 + 1e-6) + 1e-28
    phi, _ = S.pcg_constants(rho)
    it = S.pcg(p.A, p.b, p.nu, p.lam, P, x0, 6)
    for t, x in enumerate(it):
        assert _delta(p, x, xs) <= 4 * phi ** t * d0 * (1 + 1e-6) + 1e-28


def _ell_star(p, SA, x0, xs, t):
    """Lemma 3.1 lower bound by least squares over Q(z) = 1 + sum_k c_k z^k."""
    Hm = S.inv_sqrt_psd(S.hessian(p.A, p.nu, p.lam))
    Hh = np.linalg.inv(Hm)
    HS = SA.T @ SA + p.nu ** 2 * np.diag(p.lam)
    lam_i, vecs = np.linalg.eigh(Hm @ HS @ Hm)
    xi = vecs.T @ (Hh @ (x0 - xs))
    z = 1.0 / lam_i
    Vm = np.stack([xi * z ** k for k in range(1, t + 1)], axis=1)
    c, *_ = np.linalg.lstsq(Vm, -xi, rcond=None)
    return 0.5 * float(np.sum((xi + Vm @ c) ** 2))


def test_pcg_attains_lower_bound_and_beats_ihs():
    # Theorem 3.3: delta_t(PCG) = ell*_t, and by Lemma 3.1 every preconditioned
    # first-order method (IHS for any step size) has delta_t >= ell*_t.
    p = small_problem(n=400, d=10, nu=1e-1, decay="geom0.95")
    xs = S.direct_solve(p.A, p.b, p.nu, p.lam)
    SA = SK.sketch("gaussian", p.A, 6, seed=1)
    P = S.Preconditioner(SA, p.nu, p.lam)
    x0 = np.zeros(p.d)
    pc = S.pcg(p.A, p.b, p.nu, p.lam, P, x0, 4)
    for mu in (0.3, 0.7, 1.0):
        ih = S.ihs(p.A, p.b, p.nu, p.lam, P, x0, 4, mu=mu)
        for t in range(5):
            assert _delta(p, pc[t], xs) <= _delta(p, ih[t], xs) * (1 + 1e-8)
    for t in range(1, 5):
        ls = _ell_star(p, SA, x0, xs, t)
        assert math.isclose(_delta(p, pc[t], xs), ls, rel_tol=1e-5)


def test_table3_polyak_bound():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table3_polyak.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 28
    for row in rows:
        rho = float(row[0])
        t = math.inf if row[1] == "inf" else int(row[1])
        printed = float(row[2])
        bold = "*" in row[3:]
        expect = float(row[row.index("typo") + 1]) if "typo" in row else printed
        val = S.polyak_bound_root(t, rho)
        # the table prints one to three significant digits, sometimes rounded
        # and sometimes truncated: accept either reading of the digits shown
        digits = row[row.index("typo") + 1] if "typo" in row else row[2]
        sig = len(digits.split("e")[0].replace(".", "").lstrip("0"))
        e10 = math.floor(math.log10(val)) - sig + 1
        candidates = {round(val / 10 ** e10) * 10 ** e10, math.floor(val / 10 ** e10) * 10 ** e10}
        assert any(math.isclose(c, expect, rel_tol=1e-9) for c in candidates), (rho, t, val, expect)
        if t != math.inf:
            assert (val ** t <= rho ** t) == bold, (rho, t)
        else:
            assert bold


def test_polyak_ihs_asymptotic_rate():
    p = small_problem(n=2048, d=16, nu=1e-2)
    xs = S.direct_solve(p.A, p.b, p.nu, p.lam)
    SA = SK.sketch("srht", p.A, 1024, seed=2)
    ev = S.cs_eigenvalues(p.A, SA, p.nu, p.lam)
    # C_S^{-1} eigenvalues must sit in [1-sqrt? ...]: use the exact interval for mu, beta
    rho = 1 - (min(1 / ev) / max(1 / ev))  # a valid rho for the heavy-ball tuning below
    P = S.Preconditioner(SA, p.nu, p.lam)
    it = S.polyak_ihs(p.A, p.b, p.nu, p.lam, P, np.zeros(p.d), 60, rho=min(rho, 0.9))
    assert S.rel_err_H(p.A, p.nu, p.lam, it[-1], xs) < 1e-8


@pytest.mark.parametrize("kind", ["gaussian", "srht", "sjlt"])
@pytest.mark.parametrize("method", ["pcg", "ihs"])
def test_adaptive_reaches_tolerance(kind, method):
    p = small_problem(n=1024, d=48, nu=1e-3, decay="harmonic")
    xs = S.direct_solve(p.A, p.b, p.nu, p.lam)
    fn = S.adaptive_pcg if method == "pcg" else S.adaptive_ihs
    x, st, trace = fn(p.A, p.b, p.nu, p.lam, kind=kind, seed=3, m_init=1, tol=1e-10, sjlt_s=2)
    assert S.rel_err_H(p.A, p.nu, p.lam, x, xs) <= 1e-10
    # every decision is consistent with the test of Algorithm 1 / 2
    for ev in trace:
        assert ev["accepted"] == (ev["ratio"] <= ev["thr"] or ev["m"] >= S.default_m_max(kind, p.n))


def test_adaptive_without_rejection_is_plain_pcg():
    # Large initial sketch: E_rho holds, the test never fails (Corollary 2.5),
    # and Algorithm 2 reduces to PCG (eq. 5) with that sketch.
    p = small_problem(n=2048, d=16, nu=1e-2)
    x, st, trace = S.adaptive_pcg(p.A, p.b, p.nu, p.lam, kind="srht", seed=1, m_init=1024, tol=1e-12)
    assert st["rejections"] == 0
    P = S.Preconditioner(SK.sketch("srht", p.A, 1024, seed=1), p.nu, p.lam)
    it = S.pcg(p.A, p.b, p.nu, p.lam, P, np.zeros(p.d), st["iters"])
    assert np.allclose(x, it[-1], rtol=1e-10, atol=1e-14)


def test_theorem_4_1_sketch_size_ceiling():
    # m_t <= max(m_init, 2 m_delta / rho) with probability >= 1 - (1 + K_max) delta.
    p = synthetic.make_problem("C1", 0, n=2048, d=128)
    de = S.effective_dimension(p.A, p.nu, p.lam)
    rho, delta = 0.125, 0.05
    bound = max(1, 2 * S.m_delta_gaussian(de, delta) / rho)
    for seed in range(3):
        _, st, _ = S.adaptive_pcg(p.A, p.b, p.nu, p.lam, kind="gaussian", seed=seed, m_init=1, rho=rho, tol=1e-10)
        assert st["final_m"] <= bound
        _, st, _ = S.adaptive_ihs(p.A, p.b, p.nu, p.lam, kind="gaussian", seed=seed, m_init=1, rho=rho, tol=1e-10)
        assert st["final_m"] <= bound


def test_m_delta_formulas_monotone():
    assert S.m_delta_srht(10, 1000, 0.1) < S.m_delta_srht(20, 1000, 0.1)
    assert S.m_delta_gaussian(10, 0.1) < S.m_delta_gaussian(10, 0.01)
    # Theorem 5.2 with d_e -> 0 leaves the log term squared.
    assert math.isclose(S.m_delta_gaussian(0.0, 0.5), 8 * math.log(32), rel_tol=1e-12)


def test_polyak_ihs_exact_preconditioner_scalar_recurrence():
    # With H_S = H (SRHT at m = n_pad, where S^T S = I) the heavy-ball error obeys
    # e_{t+1} = (1 - mu + beta) e_t - beta e_{t-1}, e_{-1} = e_0: a scalar
    # recurrence in mu_rho, beta_rho of Corollary A.2, independent of the data.
    p = small_problem(n=256, d=12, nu=1e-2)
    xs = S.direct_solve(p.A, p.b, p.nu, p.lam)
    P = S.Preconditioner(SK.sketch("srht", p.A, 256, seed=3), p.nu, p.lam)
    rho = 0.3
    mu = 2 * (1 - rho) / (1 + math.sqrt(1 - rho))
    beta = (1 - math.sqrt(1 - rho)) / (1 + math.sqrt(1 - rho))
    it = S.polyak_ihs(p.A, p.b, p.nu, p.lam, P, np.zeros(p.d), 8, rho)
    e0 = -xs
    c_prev, c = 1.0, 1.0
    for t in range(1, 9):
        c_prev, c = c, (1 - mu + beta) * c - beta * c_prev
        assert np.linalg.norm(it[t] - xs - c * e0) <= 1e-9 * np.linalg.norm(e0), t


def test_cg_matches_scipy_cg_iterates():
    # The unpreconditioned CG baseline (Section 6) is the textbook method:
    # its iterates equal scipy.sparse.linalg.cg's on the same system.
    import scipy.sparse.linalg as spla
    p = small_problem(n=400, d=20, nu=1e-1)
    H = S.hessian(p.A, p.nu, p.lam)
    seen = []
    spla.cg(H, p.b, x0=np.zeros(p.d), rtol=1e-300, atol=0.0, maxiter=8, callback=lambda xk: seen.append(xk.copy()))
    ours = S.cg(p.A, p.b, p.nu, p.lam, np.zeros(p.d), 8)
    assert len(seen) == 8
    for t in range(8):
        assert np.linalg.norm(ours[t + 1] - seen[t]) <= 1e-10 * np.linalg.norm(seen[t]), t


def test_dual_formulation_recovers_primal_solution():
    # n < d: solving eq. (2) directly and mapping back with x = Lambda^{-1}(b - A^T w)/nu^2
    # gives the primal optimum of eq. (1) (the same x as the d x d Cholesky solve).
    rng = np.random.default_rng(8)
    n, d, nu = 40, 120, 3e-2
    A = rng.standard_normal((n, d)) * (0.9 ** np.arange(d))[None, :]
    lam = 1 + 9 * rng.random(d)
    b = rng.standard_normal((d, 2))
    D, bd, nud, lamd = S.dual_problem(A, b, nu, lam)
    assert D.shape == (d, n)
    w = S.direct_solve(D, bd, nud, lamd)
    x = S.primal_from_dual(A, b, nu, lam, w)
    xs = S.direct_solve(A, b, nu, lam)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    # the dual Hessian is A Lambda^{-1} A^T + nu^2 I
    assert np.allclose(D.T @ D + nu ** 2 * np.eye(n), (A / lam[None, :]) @ A.T + nu ** 2 * np.eye(n))


@pytest.mark.parametrize("kind,m", [("srht", 64), ("gaussian", 48)])
def test_remark_4_2_certified_termination(kind, m):
    # Remark 4.2: once delta~_t <= eps / (m_delta + 1), delta_t <= eps (with
    # probability >= 1 - delta over S; fixed seeds here).  delta = 1/2 ||x_t - x*||_H^2
    # from the exact x*, delta~_t = 1/2 r_t^T H_S^{-1} r_t along fixed-sketch PCG,
    # m_delta from Theorem 5.1 / 5.2 with d_e := d (the replacement the remark suggests).
    p = small_problem(n=1024, d=24, nu=1e-2, seed=2)
    xs = S.direct_solve(p.A, p.b, p.nu, p.lam)
    P = S.Preconditioner(SK.sketch(kind, p.A, m, seed=4), p.nu, p.lam)
    delta = 0.05
    md = S.m_delta_srht(p.d, p.A.shape[0], delta) if kind == "srht" else S.m_delta_gaussian(p.d, delta)
    eps = 1e-14 * S.h_norm_sq(p.A, p.nu, p.lam, xs)
    hit = False
    for x in S.pcg(p.A, p.b, p.nu, p.lam, P, np.zeros(p.d), 40):
        r = p.b - S.hess_apply(p.A, p.nu, p.lam, x)
        dtil = 0.5 * float(r @ P.apply(r))
        if dtil <= S.termination_threshold(eps, md):
            hit = True
            assert 0.5 * S.h_norm_sq(p.A, p.nu, p.lam, x - xs) <= eps
    assert hit


def test_dual_error_bound():
    # ||x - x*||_H <= ||H_dual (w - w*)|| / nu^2 for any w, with x the primal map of w
    rng = np.random.default_rng(9)
    n, d, nu = 30, 90, 5e-2
    A = rng.standard_normal((n, d)) / np.sqrt(d)
    lam = 1 + rng.random(d)
    b = rng.standard_normal(d)
    D, bd, _, lamd = S.dual_problem(A, b, nu, lam)
    ws = S.direct_solve(D, bd, nu, lamd)
    xs = S.direct_solve(A, b, nu, lam)
    Hd = D.T @ D + nu ** 2 * np.eye(n)
    for scale in (1e-1, 1e-4, 1e-8):
        w = ws + scale * rng.standard_normal(n)
        x = S.primal_from_dual(A, b, nu, lam, w)
        assert np.sqrt(S.h_norm_sq(A, nu, lam, x - xs)) <= np.linalg.norm(Hd @ (w - ws)) / nu ** 2 * (1 + 1e-9)


# ----------------------------------------------------------------------------
# Corollary 2.5: under E_rho the improvement test of Algorithms 1 / 2 passes
# ----------------------------------------------------------------------------

def _e_rho_events(p, method, kind, m_init, rho, seed=3, s=2, **kw):
    """Run the adaptive method and return [(event, ||C_S - I||_2 <= sqrt(rho),
    event follows a re-sketch)] with C_S = H^{-1/2} H_S H^{-1/2} of the
    sketch each event used (nested sketches: the one of size m)."""
    fn = S.adaptive_pcg if method == "pcg" else S.adaptive_ihs
    _, _, trace = fn(p.A, p.b, p.nu, p.lam, kind=kind, seed=seed, m_init=m_init, rho=rho, tol=1e-10,
                     sjlt_s=s, **kw)
    sk = S._Sketcher(p.A, kind, seed, s)
    dev = {}
    out = []
    after = True  # the first event follows the first sketch
    for ev in trace:
        m = ev["m"]
        if m not in dev:
            e = S.cs_eigenvalues(p.A, sk(m), p.nu, p.lam)
            dev[m] = max(abs(e[0] - 1.0), abs(e[-1] - 1.0))
        out.append((ev, dev[m] <= math.sqrt(rho), after))
        after = not ev["accepted"]
    return out


@pytest.mark.parametrize("kind", ["gaussian", "srht", "sjlt"])
@pytest.mark.parametrize("method", ["pcg", "ihs"])
def test_corollary_2_5_no_rejection_under_E_rho(kind, method):
    # Conditional on E_rho (||C_S - I|| <= sqrt(rho), rho < 1), delta~_t <=
    # c(alpha, rho) phi(rho)^t delta~_0 for the method restarted with that
    # sketch (Corollary 2.5 with Theorem 3.2 / eq. 11).  Algorithm 2 / 1 test
    # delta~+/delta~_I against c phi^(t+1-I), so every step taken with a
    # sketch in E_rho is accepted -- also the first step after a restart
    # (exponent 1).  A threshold exponent one too large, or delta~_I not
    # reset to the restart's decrement, rejects some of these steps.
    rho = 0.125
    p = small_problem(n=8192, d=32, nu=0.1)
    events = []
    for m_init in (1, 64, 2048):
        events += _e_rho_events(p, method, kind, m_init, rho)
    held = [(ev, after) for ev, ok, after in events if ok]
    assert len(held) >= 5  # m_init = 2048 lies in E_rho for every embedding here
    assert any(after for _, after in held)
    for ev, _ in held:
        assert ev["accepted"], ev


def test_corollary_2_5_after_a_rejection():
    # A run whose doubling lands on a sketch in E_rho: the step right after
    # the re-sketch (first step of the restarted method) is accepted.
    p = small_problem(n=8192, d=32, nu=0.1)
    seen = 0
    for method in ("pcg", "ihs"):
        ev = _e_rho_events(p, method, "sjlt", 64, 0.125)
        rejected_before = False
        for e, ok, after in ev:
            if ok and after and rejected_before:
                seen += 1
                assert e["accepted"]
            rejected_before = rejected_before or not e["accepted"]
    assert seen >= 2


@pytest.mark.parametrize("kind", ["gaussian", "srht"])
def test_adaptive_ihs_decisions_recomputed(kind):
    # Algorithm 1 with the IHS: every test event recomputed from its inputs by
    # the definitions -- the proposal x+ = x_t - (1 - rho) H_S^{-1} grad f(x_t)
    # (eq. 4 with Theorem 3.2's step), delta~ = 1/2 grad f^T H_S^{-1} grad f
    # (Section 2.3) with the CURRENT sketch, I = the time of the last re-sketch
    # (0 at the start), delta~_I the decrement at x_I with the current sketch
    # (reset at every re-sketch: the method restarts at x_t), the threshold
    # c(1, rho) rho^(t+1-I), and the verdict.
    rho = 0.125
    p = small_problem(n=2048, d=24, nu=1e-2)
    _, _, trace = S.adaptive_ihs(p.A, p.b, p.nu, p.lam, kind=kind, seed=4, m_init=1, rho=rho, tol=1e-10,
                                 record_states=True)
    sk = S._Sketcher(p.A, kind, 4, 1)
    c = (1 + math.sqrt(rho)) / (1 - math.sqrt(rho))
    H = S.hessian(p.A, p.nu, p.lam)
    I, xI = 0, np.zeros(p.d)
    assert sum(not e["accepted"] for e in trace) >= 3
    floor = 1e-12 * trace[0]["dI"]  # decrements below this are rounding noise of the residual
    for ev in trace:
        SA = sk(ev["m"])
        HS = SA.T @ SA + p.nu ** 2 * np.diag(p.lam)
        x = ev["x"]
        g = H @ x - p.b
        xp = x - (1 - rho) * np.linalg.solve(HS, g)
        gp = H @ xp - p.b
        dp = 0.5 * gp @ np.linalg.solve(HS, gp)
        gI = H @ xI - p.b
        dI = 0.5 * gI @ np.linalg.solve(HS, gI)
        thr = c * rho ** (ev["t"] + 1 - I)
        assert ev["I"] == I
        assert math.isclose(ev["dp"], dp, rel_tol=1e-7, abs_tol=floor)
        assert math.isclose(ev["dI"], dI, rel_tol=1e-7, abs_tol=floor)
        assert math.isclose(ev["thr"], thr, rel_tol=1e-12)
        if dp > floor and abs(dp / dI / thr - 1) > 1e-6:
            assert ev["accepted"] == (dp / dI <= thr)
        if not ev["accepted"]:
            I, xI = ev["t"], x.copy()
