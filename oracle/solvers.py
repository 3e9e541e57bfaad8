"""Problem (1), the sketched preconditioner and the (adaptive) iterative
solvers of Lacotte & Pilanci (arXiv 2104.14101), oracle side, float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation follows the paper: H = A^T A + nu^2 Lambda (eq. 1), H_S = (SA)^T SA +
nu^2 Lambda (eq. 3), delta_x = 1/2 ||x - x*||_H^2 (Section 1.1), the
approximate Newton decrement delta~_x = 1/2 grad f(x)^T H_S^{-1} grad f(x)
(Section 2.3), IHS (eq. 4), PCG (eq. 5), Algorithm 1 (prototype adaptive
method, instantiated with the IHS and mu = 1 - rho as in Theorem 3.2),
Algorithm 2 (adaptive PCG).
"""
import math

import numpy as np
import scipy.linalg

from . import sketch as SK


# ----------------------------------------------------------------------------
# Problem (1)
# ----------------------------------------------------------------------------

def _col(v, like):
    return v.reshape((-1,) + (1,) * (like.ndim - 1))


def hess_apply(A, nu, lam, x):
    """H x = A^T (A x) + nu^2 Lambda x (eq. 1); x may be d or d x k."""
    return A.T @ (A @ x) + nu ** 2 * _col(lam, x) * x


def hessian(A, nu, lam):
    return A.T @ A + nu ** 2 * np.diag(lam)


def objective(A, b, nu, lam, x):
    """f(x) = 1/2 <x, H x> - b^T x (eq. 1)."""
    return 0.5 * float(np.sum(x * hess_apply(A, nu, lam, x))) - float(np.sum(b * x))


def direct_solve(A, b, nu, lam, refine=3):
    """x* = H^{-1} b by Cholesky of H (the paper's direct baseline, Section 6),
    followed by ``refine`` steps of iterative refinement whose residual
    b - A^T(A x) - nu^2 Lambda x is formed from A itself (not from the Gram
    matrix), so that the result is accurate to ~kappa(H)^(1/2) u in H-norm.
    Pinned to the closed form x* = V diag(sigma/(sigma^2+nu^2)) U^T y in the
    tests."""
    c = scipy.linalg.cho_factor(hessian(A, nu, lam), lower=True)
    x = scipy.linalg.cho_solve(c, b)
    for _ in range(refine):
        r = b - hess_apply(A, nu, lam, x)
        x = x + scipy.linalg.cho_solve(c, r)
    return x


def h_norm_sq(A, nu, lam, e):
    """||e||_H^2 = ||A e||^2 + nu^2 e^T Lambda e, from A (summed over RHS)."""
    Ae = A @ e
    return float(np.sum(Ae * Ae) + nu ** 2 * np.sum(_col(lam, e) * e * e))


def rel_err_H(A, nu, lam, x, xstar):
    """||x - x*||_H / ||x*||_H: the accuracy measure of every result
    (delta_x = 1/2 ||x - x*||_H^2, Section 1.1)."""
    return math.sqrt(h_norm_sq(A, nu, lam, x - xstar) / h_norm_sq(A, nu, lam, xstar))


# ----------------------------------------------------------------------------
# Sketched preconditioner H_S (Section 4.1.1)
# ----------------------------------------------------------------------------

class Preconditioner:
    """Solve H_S v = z with H_S = (SA)^T SA + nu^2 Lambda (Section 4.1.1).

    m >= d: Cholesky of the d x d matrix H_S.
    m <  d: Cholesky of W_S = SA Lambda^{-1} (SA)^T + nu^2 I_m and the Woodbury
            identity v = (Lambda^{-1}/nu^2)(I - (SA)^T W_S^{-1} SA Lambda^{-1}) z.
    """

    def __init__(self, SA, nu, lam):
        self.SA = np.asarray(SA, dtype=np.float64)
        self.nu = float(nu)
        self.lam = np.asarray(lam, dtype=np.float64)
        m, d = self.SA.shape
        self.woodbury = m < d
        if self.woodbury:
            W = (self.SA / self.lam[None, :]) @ self.SA.T + self.nu ** 2 * np.eye(m)
            self.fac = scipy.linalg.cho_factor(W, lower=True)
        else:
            HS = self.SA.T @ self.SA + self.nu ** 2 * np.diag(self.lam)
            self.fac = scipy.linalg.cho_factor(HS, lower=True)

    def apply(self, z):
        if not self.woodbury:
            return scipy.linalg.cho_solve(self.fac, z)
        lz = z / _col(self.lam, z)
        s = scipy.linalg.cho_solve(self.fac, self.SA @ lz)
        return (z - self.SA.T @ s) / (_col(self.lam, z) * self.nu ** 2)

    def matrix(self):
        """H_S itself (for tests)."""
        return self.SA.T @ self.SA + self.nu ** 2 * np.diag(self.lam)


# ----------------------------------------------------------------------------
# Fixed-sketch methods
# ----------------------------------------------------------------------------

def ihs(A, b, nu, lam, P, x0, T, mu):
    """IHS (eq. 4): x_{t+1} = x_t - mu H_S^{-1} grad f(x_t). Returns iterates."""
    xs = [np.array(x0, dtype=np.float64)]
    x = xs[0]
    for _ in range(T):
        g = hess_apply(A, nu, lam, x) - b
        x = x - mu * P.apply(g)
        xs.append(x)
    return xs


def pcg(A, b, nu, lam, P, x0, T):
    """PCG with preconditioner H_S (eq. 5). Returns the iterates x_0..x_T."""
    x = np.array(x0, dtype=np.float64)
    r = b - hess_apply(A, nu, lam, x)
    rt = P.apply(r)
    p = rt.copy()
    dt = float(np.sum(r * rt))
    xs = [x.copy()]
    for _ in range(T):
        if dt == 0.0:
            xs.append(x.copy())
            continue
        Hp = hess_apply(A, nu, lam, p)
        alpha = dt / float(np.sum(p * Hp))
        x = x + alpha * p
        r = r - alpha * Hp
        rt = P.apply(r)
        dn = float(np.sum(r * rt))
        p = rt + (dn / dt) * p
        dt = dn
        xs.append(x.copy())
    return xs


def cg(A, b, nu, lam, x0, T):
    """Unpreconditioned CG (the paper's CG baseline, Section 6) = PCG with P = I."""
    class _Id:
        @staticmethod
        def apply(z):
            return z
    return pcg(A, b, nu, lam, _Id, x0, T)


def polyak_ihs(A, b, nu, lam, P, x0, T, rho):
    """Polyak-IHS / heavy ball (eq. A.1) with the step size and momentum of
    Corollary A.2: mu = 2(1-rho)/(1+sqrt(1-rho)), beta = (1-sqrt(1-rho))/(1+sqrt(1-rho))."""
    mu = 2.0 * (1.0 - rho) / (1.0 + math.sqrt(1.0 - rho))
    beta = (1.0 - math.sqrt(1.0 - rho)) / (1.0 + math.sqrt(1.0 - rho))
    x_prev = np.array(x0, dtype=np.float64)
    x = x_prev.copy()
    xs = [x.copy()]
    for _ in range(T):
        g = hess_apply(A, nu, lam, x) - b
        x_new = x - mu * P.apply(g) + beta * (x - x_prev)
        x_prev, x = x, x_new
        xs.append(x.copy())
    return xs


# ----------------------------------------------------------------------------
# Constants of Condition 2.4 / Corollary 2.5
# ----------------------------------------------------------------------------

def pcg_constants(rho):
    """phi(rho) = (1-sqrt(1-rho))/(1+sqrt(1-rho)) and c(rho) = 4 (1+sqrt rho)/(1-sqrt rho)
    of Algorithm 2 (alpha = 4, eq. 11)."""
    phi = (1.0 - math.sqrt(1.0 - rho)) / (1.0 + math.sqrt(1.0 - rho))
    c = 4.0 * (1.0 + math.sqrt(rho)) / (1.0 - math.sqrt(rho))
    return phi, c


def ihs_constants(rho):
    """IHS with mu = 1 - rho: phi(rho) = rho, alpha = 1 (Theorem 3.2), so
    c(1, rho) = (1+sqrt rho)/(1-sqrt rho)."""
    return rho, (1.0 + math.sqrt(rho)) / (1.0 - math.sqrt(rho))


# ----------------------------------------------------------------------------
# Adaptive methods
# ----------------------------------------------------------------------------

class _Sketcher:
    """Nested sketches S_m A for growing m (reading: one seed, the SRHT keeps
    E and the permutation and takes more rows, the Gaussian embedding appends
    rows; the SJLT re-hashes)."""

    def __init__(self, A, kind, seed, sjlt_s):
        self.A, self.kind, self.seed, self.s = A, kind, seed, sjlt_s
        self.B = SK.srht_hda(A, seed) if kind == "srht" else None
        self.n_pad = SK.next_pow2(A.shape[0])

    def __call__(self, m):
        if self.kind == "srht":
            return self.B[SK.srht_rows(m, self.n_pad, self.seed)] / math.sqrt(m)
        return SK.sketch(self.kind, self.A, m, self.seed, self.s)


def default_m_max(kind, n):
    """Cap on the sketch size: n_pad for the SRHT (where S^T S = I), n otherwise."""
    return SK.next_pow2(n) if kind == "srht" else n


def adaptive_pcg(A, b, nu, lam, kind="gaussian", seed=0, m_init=1, m_max=None, rho=0.125,
                 x0=None, tol=1e-10, max_iter=1000, sjlt_s=1, literal_restart=True,
                 stop="estimate", xstar=None, record_states=False):
    """Algorithm 2 (adaptive PCG).

    phi(rho) and c(rho) as in ``pcg_constants``; the step at time t produces
    x+, r+, r~+ = H_S^{-1} r+, delta~+ = (r+)^T r~+ and is rejected when
    delta~+ / delta~_I > c(rho) phi(rho)^(t+1-I); a rejection sets I = t,
    doubles m (capped at m_max, where a failing test accepts instead), draws the
    larger sketch, refactors H_S and restarts PCG at x_t with r_t = b - H x_t.

    Stop rule (the paper prescribes none): after each accepted step, stop when
    delta~_t <= (tol/2)^2 * b^T x_t, i.e. the estimate
    delta~_t / (b^T x_t) ~ ||x_t - x*||_H^2 / ||x*||_H^2 is below (tol/2)^2.
    With stop="exact" and ``xstar`` given, stop on the true relative H-error.
    With record_states, every trace event also holds the index I of the last
    re-sketch, delta~_I, delta~+ and a copy of x_t (the accepted iterate the
    step started from).
    Returns (x, stats, trace).
    """
    n, d = A.shape
    m_max = default_m_max(kind, n) if m_max is None else min(int(m_max), default_m_max(kind, n))
    phi, c = pcg_constants(rho)
    sk = _Sketcher(A, kind, seed, sjlt_s)
    m = min(int(m_init), m_max)
    P = Preconditioner(sk(m), nu, lam)
    stats = dict(iters=0, rejections=0, a_passes=0, sketches=1, factorizations=1, final_m=m)
    x = np.zeros(d) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - hess_apply(A, nu, lam, x)
    stats["a_passes"] += 1
    rt = P.apply(r)
    p = rt.copy()
    dt = float(r @ rt)
    dI = dt
    t, I = 0, 0
    trace = []

    def done(x, dt):
        if stop == "exact":
            return rel_err_H(A, nu, lam, x, xstar) <= tol
        return dt <= (tol / 2.0) ** 2 * float(b @ x)

    if dt == 0.0:
        stats.update(final_m=m, final_delta=dt)
        return x, stats, trace
    while t < max_iter:
        Hp = hess_apply(A, nu, lam, p)
        stats["a_passes"] += 1
        alpha = dt / float(p @ Hp)
        xp = x + alpha * p
        rp = r - alpha * Hp
        rtp = P.apply(rp)
        dp = float(rp @ rtp)
        thr = c * phi ** (t + 1 - I)
        ratio = dp / dI
        ev = dict(t=t, m=m, ratio=ratio, thr=thr)
        if record_states:
            ev.update(I=I, dI=dI, dp=dp, x=x.copy())
        if ratio > thr and m < m_max:
            trace.append(dict(ev, accepted=False))
            I = t
            m = min(2 * m, m_max)
            P = Preconditioner(sk(m), nu, lam)
            stats["rejections"] += 1
            stats["sketches"] += 1
            stats["factorizations"] += 1
            if literal_restart:
                r = b - hess_apply(A, nu, lam, x)
                stats["a_passes"] += 1
            rt = P.apply(r)
            p = rt.copy()
            dt = float(r @ rt)
            dI = dt
        else:
            trace.append(dict(ev, accepted=True))
            p = rtp + (dp / dt) * p
            x, r, rt, dt = xp, rp, rtp, dp
            t += 1
            if dt <= 0.0 or done(x, dt):
                break
    stats.update(iters=t, final_m=m, final_delta=dt)
    return x, stats, trace


def adaptive_ihs(A, b, nu, lam, kind="gaussian", seed=0, m_init=1, m_max=None, rho=0.125,
                 x0=None, tol=1e-10, max_iter=1000, sjlt_s=1, stop="estimate", xstar=None,
                 record_states=False):
    """Algorithm 1 instantiated with the IHS and step size mu = 1 - rho
    (Theorem 3.2: phi(rho) = rho, alpha = 1).

    The step at time t is x+ = x_t - mu H_S^{-1} grad f(x_t) with
    delta~+ = 1/2 grad f(x+)^T H_S^{-1} grad f(x+); it is rejected when
    delta~+ / delta~_I > c(1, rho) rho^(t+1-I), in which case I = t, m doubles
    (capped as in ``adaptive_pcg``), a larger sketch is drawn and
    delta~_I = 1/2 grad f(x_t)^T H_S^{-1} grad f(x_t).
    Stop rule: after an accepted step, 2 delta~_t <= (tol/2)^2 b^T x_t.
    record_states: as in ``adaptive_pcg``.
    """
    n, d = A.shape
    m_max = default_m_max(kind, n) if m_max is None else min(int(m_max), default_m_max(kind, n))
    mu = 1.0 - rho
    phi, c = ihs_constants(rho)
    sk = _Sketcher(A, kind, seed, sjlt_s)
    m = min(int(m_init), m_max)
    P = Preconditioner(sk(m), nu, lam)
    stats = dict(iters=0, rejections=0, a_passes=0, sketches=1, factorizations=1, final_m=m)
    x = np.zeros(d) if x0 is None else np.array(x0, dtype=np.float64)
    g = hess_apply(A, nu, lam, x) - b
    stats["a_passes"] += 1
    v = P.apply(g)
    dt = 0.5 * float(g @ v)
    dI = dt
    t, I = 0, 0
    trace = []

    def done(x, dt):
        if stop == "exact":
            return rel_err_H(A, nu, lam, x, xstar) <= tol
        return 2.0 * dt <= (tol / 2.0) ** 2 * float(b @ x)

    if dt == 0.0:
        stats.update(final_m=m, final_delta=dt)
        return x, stats, trace
    while t < max_iter:
        xp = x - mu * v
        gp = hess_apply(A, nu, lam, xp) - b
        stats["a_passes"] += 1
        vp = P.apply(gp)
        dp = 0.5 * float(gp @ vp)
        thr = c * phi ** (t + 1 - I)
        ratio = dp / dI
        ev = dict(t=t, m=m, ratio=ratio, thr=thr)
        if record_states:
            ev.update(I=I, dI=dI, dp=dp, x=x.copy())
        if ratio > thr and m < m_max:
            trace.append(dict(ev, accepted=False))
            I = t
            m = min(2 * m, m_max)
            P = Preconditioner(sk(m), nu, lam)
            stats["rejections"] += 1
            stats["sketches"] += 1
            stats["factorizations"] += 1
            v = P.apply(g)
            dt = 0.5 * float(g @ v)
            dI = dt
        else:
            trace.append(dict(ev, accepted=True))
            x, g, v, dt = xp, gp, vp, dp
            t += 1
            if dt <= 0.0 or done(x, dt):
                break
    stats.update(iters=t, final_m=m, final_delta=dt)
    return x, stats, trace


# ----------------------------------------------------------------------------
# Theory quantities (test tools)
# ----------------------------------------------------------------------------

# ----------------------------------------------------------------------------
# Dual formulation (eq. 2)
# ----------------------------------------------------------------------------

def dual_problem(A, b, nu, lam):
    """Eq. (2) as an instance of eq. (1): data matrix Lambda^{-1/2} A^T (d x n),
    Lambda = I_n, right-hand side A Lambda^{-1} b, the same nu."""
    lam = np.asarray(lam, dtype=np.float64)
    D = (A / np.sqrt(lam)[None, :]).T
    bd = A @ (b / _col(lam, b))
    return D, bd, nu, np.ones(A.shape[0])


def primal_from_dual(A, b, nu, lam, w):
    """x = Lambda^{-1} (b - A^T w) / nu^2: the primal optimum from the dual one
    (eq. 1's optimality condition H x = b with w = (A Lambda^{-1} A^T + nu^2
    I)^{-1} A Lambda^{-1} b, i.e. the Woodbury identity)."""
    lam = np.asarray(lam, dtype=np.float64)
    return (b - A.T @ w) / (_col(lam, b) * nu ** 2)


def inv_sqrt_psd(M):
    w, Q = np.linalg.eigh(M)
    return (Q / np.sqrt(w)[None, :]) @ Q.T


def effective_dimension(A, nu, lam):
    """d_e = tr(A_nu) / ||A_nu||_2 with A_nu = A^T A (A^T A + nu^2 Lambda)^{-1}
    (Section 1), computed as ||D||_F^2 / ||D||_2^2 from the singular values D of
    A (A^T A + nu^2 Lambda)^{-1/2} (Section 1.1)."""
    M = A @ inv_sqrt_psd(hessian(A, nu, lam))
    D = np.linalg.svd(M, compute_uv=False)
    return float(np.sum(D ** 2) / np.max(D) ** 2)


def cs_eigenvalues(A, SA, nu, lam):
    """Eigenvalues of C_S = H^{-1/2} H_S H^{-1/2} (Section 1.1), descending."""
    Hm = inv_sqrt_psd(hessian(A, nu, lam))
    HS = SA.T @ SA + nu ** 2 * np.diag(lam)
    return np.sort(np.linalg.eigvalsh(Hm @ HS @ Hm))[::-1]


def m_delta_srht(d_e, n, delta):
    """Theorem 5.1: m_delta = 16 log(16 d_e/delta) (sqrt(d_e) + sqrt(8 log(2n/delta)))^2."""
    return 16.0 * math.log(16.0 * d_e / delta) * (math.sqrt(d_e) + math.sqrt(8.0 * math.log(2.0 * n / delta))) ** 2


def m_delta_gaussian(d_e, delta):
    """Theorem 5.2 with omega(C)^2 <= d_e: m_delta = (sqrt(d_e) + sqrt(8 log(16/delta)))^2."""
    return (math.sqrt(d_e) + math.sqrt(8.0 * math.log(16.0 / delta))) ** 2


def polyak_bound_root(t, rho):
    """(alpha(t, rho) beta_rho^omega(t))^(1/t) of Corollary A.2 / Table 3 with
    alpha = 3^(nu(nu+1)) (1 + 4 beta + beta^2)^(2 nu), omega = t - 2 nu,
    nu(t) = log2(t) + 1, beta_rho = (1-sqrt(1-rho))/(1+sqrt(1-rho));
    t = inf gives the asymptotic rate beta_rho."""
    beta = (1.0 - math.sqrt(1.0 - rho)) / (1.0 + math.sqrt(1.0 - rho))
    if t == math.inf:
        return beta
    nu_t = math.log(t) / math.log(2.0) + 1.0
    log_alpha = nu_t * (nu_t + 1.0) * math.log(3.0) + 2.0 * nu_t * math.log(1.0 + 4.0 * beta + beta * beta)
    omega = t - 2.0 * nu_t
    return math.exp((log_alpha + omega * math.log(beta)) / t)


def termination_threshold(eps, m_delta):
    """Remark 4.2: delta~_t <= eps / (m_delta + 1) guarantees delta_t <= eps."""
    return eps / (m_delta + 1.0)
