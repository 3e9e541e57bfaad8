"""Seeded generators of the five workloads the solver is measured on.

All workloads follow the recipe of the paper's synthetic experiments
(Section 6): A = U diag(sigma) V^T with U (n x d) and V (d x d) orthonormal and
a prescribed decay of sigma.  U and V come from the QR factorisation of seeded
N(0, 1) matrices, with the sign convention diag(R) > 0 so that the factor is
unique.  ``make_problem`` does this in NumPy float64 (sizes the CPU handles in
seconds); ``make_problem_torch`` does the same recipe with the n x d work on a
torch device for the full benchmark sizes, orthonormalising by one CholeskyQR
pass.

Workloads (n rows, d columns):
  C1  n=4096,  d=256,  sigma_j = 0.95^j,        nu=1e-2, Lambda=I,   b=A^T y
  C2  n=2^17,  d=2048, sigma_j = 1/(1+j),       nu=1e-3, Lambda=1+9U, b=A^T y + 0.1 N(0,1)
  C3  n=2^20,  d=4096, sigma_j = 0.98^j + 1e-6, nu=1e-4, Lambda=I,   b=A^T y   (A stored fp32)
  C4  n=2^18,  d=1024, sigma_j = (1+j)^-1/2,    nu=1e-2, Lambda=1+U,  b=A^T N(0,1)^(n x 8)
  C5  256 problems, n in [2^11, 2^16], d in [32, 1024] log-uniform with n >= 4d,
      sigma_j = 0.9^j or 1/(1+j), nu log-uniform in [1e-4, 1e-1], Lambda=I.
with y ~ N(0, 1)^n and j = 0, ..., d-1.
"""
from dataclasses import dataclass, field
import math

import numpy as np

CONFIGS = {
    "C1": dict(n=4096, d=256, decay="geom0.95", nu=1e-2, lam="identity", rhs="Aty", k=1,
               dtype="f64", kind="gaussian", m_init=1, tol=1e-10),
    "C2": dict(n=1 << 17, d=2048, decay="harmonic", nu=1e-3, lam="one_plus_9u", rhs="Aty_noise", k=1,
               dtype="f64", kind="srht", m_init=16, m_max=4096, tol=1e-10),
    "C3": dict(n=1 << 20, d=4096, decay="geom0.98_floor", nu=1e-4, lam="identity", rhs="Aty", k=1,
               dtype="f32", kind="gaussian", m_init=1, tol=1e-8),
    "C4": dict(n=1 << 18, d=1024, decay="sqrt_harmonic", nu=1e-2, lam="one_plus_u", rhs="Aty_multi", k=8,
               dtype="f32", kind="gaussian", m_init=1, tol=1e-8),
    # the paper's synthetic experiments (Section 6): n up to 2^19, d 7000 / 14000, sigma_j = 0.995^j
    "P": dict(n=1 << 19, d=14000, decay="geom0.995", nu=1e-2, lam="identity", rhs="Aty", k=1,
              dtype="f32", kind="srht", m_init=1, tol=1e-8),
    # more columns than rows (solved through the dual, eq. 2): the shape of the paper's OVA-Lung
    # experiment (Section 6), sigma_j = 0.995^j over the n nonzero singular values
    "D": dict(n=1545, d=10936, decay="geom0.995", nu=1e-2, lam="identity", rhs="gauss", k=1,
              dtype="f64", kind="srht", m_init=1, tol=1e-10),
    # one member of the uneven batch; n, d, decay and nu come from batched_specs
    "C5": dict(n=4096, d=128, decay="geom0.9", nu=1e-2, lam="identity", rhs="Aty", k=1,
               dtype="f64", kind="srht", m_init=1, tol=1e-8),
}


def spectrum(decay, d):
    """Singular values sigma_j, j = 0..d-1, for the named decay."""
    j = np.arange(d, dtype=np.float64)
    if decay == "geom0.95":
        return 0.95 ** j
    if decay == "geom0.9":
        return 0.9 ** j
    if decay == "geom0.995":
        return 0.995 ** (j + 1)
    if decay == "harmonic":
        return 1.0 / (1.0 + j)
    if decay == "geom0.98_floor":
        return 0.98 ** j + 1e-6
    if decay == "sqrt_harmonic":
        return (1.0 + j) ** -0.5
    raise ValueError(decay)


@dataclass
class Problem:
    """One instance of problem (1).  A is n x d row-major; b is d x k."""
    A: np.ndarray
    b: np.ndarray
    nu: float
    lam: np.ndarray
    sigma: np.ndarray = None
    U: np.ndarray = None
    V: np.ndarray = None
    y: np.ndarray = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.A.shape[0]

    @property
    def d(self):
        return self.A.shape[1]


def _orthonormal(rng, rows, cols):
    Z = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(Z)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :]


def _lambda(kind, rng, d):
    if kind == "identity":
        return np.ones(d)
    if kind == "one_plus_9u":
        return 1.0 + 9.0 * rng.random(d)
    if kind == "one_plus_u":
        return 1.0 + rng.random(d)
    raise ValueError(kind)


def make_problem(config="C1", seed=0, n=None, d=None, nu=None, decay=None, lam=None,
                 rhs=None, k=None, dtype=None):
    """NumPy float64 generator (the stored matrix is rounded to float32 when the
    workload stores A in float32; the float64 problem is then the exact upcast
    of that float32 matrix, so both precisions solve the same problem)."""
    cfg = dict(CONFIGS[config])
    for key, val in dict(n=n, d=d, nu=nu, decay=decay, lam=lam, rhs=rhs, k=k, dtype=dtype).items():
        if val is not None:
            cfg[key] = val
    n, d = int(cfg["n"]), int(cfg["d"])
    rng = np.random.default_rng(seed)
    U = _orthonormal(rng, n, d)
    V = _orthonormal(rng, d, d)
    sigma = spectrum(cfg["decay"], d)
    A = (U * sigma[None, :]) @ V.T
    if cfg["dtype"] == "f32":
        A = A.astype(np.float32).astype(np.float64)
    lam_v = _lambda(cfg["lam"], rng, d)
    kk = int(cfg["k"])
    if cfg["rhs"] == "Aty":
        y = rng.standard_normal(n)
        b = A.T @ y
    elif cfg["rhs"] == "Aty_noise":
        y = rng.standard_normal(n)
        b = A.T @ y + 0.1 * rng.standard_normal(d)
    elif cfg["rhs"] == "Aty_multi":
        y = rng.standard_normal((n, kk))
        b = A.T @ y
    else:
        raise ValueError(cfg["rhs"])
    return Problem(A=np.ascontiguousarray(A), b=b, nu=float(cfg["nu"]), lam=lam_v, sigma=sigma,
                   U=U, V=V, y=y, meta=dict(config=config, seed=seed, **cfg))


def make_problem_torch(config="C2", seed=0, device="cuda", n=None, d=None, nu=None, decay=None):
    """Same recipe as ``make_problem`` on a torch device, for full sizes.

    The n x d Gaussian comes from a seeded ``torch.Generator`` on the device
    (so the values differ from the NumPy generator's); the d x d pieces (QR of
    the V Gaussian, Cholesky of Z^T Z, the triangular solve) are done in NumPy
    float64 on the host, and only the two n x d x d products run on the device
    (matmul).  U = Z L^{-T} is the CholeskyQR factor of Z.  Returns a dict of
    device tensors: A64 (float64) and, for float32-stored workloads, A32 with
    A64 its exact upcast; b (d x k); lam (d).
    """
    import scipy.linalg
    import torch

    cfg = dict(CONFIGS[config])
    for key, val in dict(n=n, d=d, nu=nu, decay=decay).items():
        if val is not None:
            cfg[key] = val
    n, d, kk = int(cfg["n"]), int(cfg["d"]), int(cfg["k"])
    rng = np.random.default_rng(seed)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = torch.float64
    sigma = spectrum(cfg["decay"], d)
    V = _orthonormal(rng, d, d)
    # float32-stored workloads do the two n x d x d products in float32 (U is
    # then orthonormal to ~1e-5, which only perturbs the spectrum by that
    # relative amount; the stored A defines the problem).
    wdt = torch.float32 if cfg["dtype"] == "f32" else f64
    Z = torch.randn(n, d, generator=g, device=device, dtype=wdt)
    C = (Z.T @ Z).to(f64).cpu().numpy()
    L = np.linalg.cholesky(C)
    # A = Z L^{-T} diag(sigma) V^T
    Mh = scipy.linalg.solve_triangular(L.T, np.diag(sigma) @ V.T, lower=False)
    M = torch.from_numpy(Mh).to(device=device, dtype=wdt)
    A = torch.empty(n, d, device=device, dtype=wdt)
    blk = 1 << 15
    for r0 in range(0, n, blk):
        A[r0:r0 + blk] = Z[r0:r0 + blk] @ M
    del Z
    lam = torch.from_numpy(_lambda(cfg["lam"], rng, d)).to(device=device, dtype=f64)
    out = dict(n=n, d=d, nu=float(cfg["nu"]), lam=lam, sigma=torch.from_numpy(sigma).to(device),
               meta=dict(config=config, seed=seed, **cfg))
    if cfg["dtype"] == "f32":
        out["A32"] = A
        A = A.to(f64)
    out["A64"] = A
    if cfg["rhs"] == "Aty":
        y = torch.randn(n, 1, generator=g, device=device, dtype=f64)
        b = A.T @ y
    elif cfg["rhs"] == "Aty_noise":
        y = torch.randn(n, 1, generator=g, device=device, dtype=f64)
        b = A.T @ y + 0.1 * torch.randn(d, 1, generator=g, device=device, dtype=f64)
    else:
        y = torch.randn(n, kk, generator=g, device=device, dtype=f64)
        b = A.T @ y
    out["b"] = b
    return out


def make_wide_problem_torch(config="D", seed=0, device="cuda", n=None, d=None, nu=None):
    """n < d: A = U diag(sigma) V^T with U (n x n) from the QR of a seeded
    Gaussian (host, float64) and V (d x n) the CholeskyQR factor of a seeded
    d x n Gaussian on the device; sigma has n entries; b ~ N(0, 1)^d.  Returns
    the dict of ``make_problem_torch`` (A64, b (d x 1), lam, nu)."""
    import torch

    cfg = dict(CONFIGS[config])
    for key, val in dict(n=n, d=d, nu=nu).items():
        if val is not None:
            cfg[key] = val
    n, d = int(cfg["n"]), int(cfg["d"])
    rng = np.random.default_rng(seed)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = torch.float64
    sigma = spectrum(cfg["decay"], n)
    U = _orthonormal(rng, n, n)
    Z = torch.randn(d, n, generator=g, device=device, dtype=f64)
    Lc = np.linalg.cholesky((Z.T @ Z).cpu().numpy())
    V = torch.linalg.solve_triangular(torch.from_numpy(Lc).to(device), Z.T, upper=False).T  # d x n, orthonormal
    A = (torch.from_numpy(U * sigma[None, :]).to(device) @ V.T).contiguous()
    lam = torch.from_numpy(_lambda(cfg["lam"], rng, d)).to(device=device, dtype=f64)
    b = torch.randn(d, 1, generator=g, device=device, dtype=f64)
    return dict(n=n, d=d, nu=float(cfg["nu"]), lam=lam, A64=A, b=b, sigma=torch.from_numpy(sigma).to(device),
                meta=dict(config=config, seed=seed, **cfg))


def batched_specs(count=256, seed=0):
    """Shapes of the uneven batch C5: n and d log-uniform (n in [2^11, 2^16],
    d in [32, 1024]) redrawn until n >= 4 d; decay 0.9^j or 1/(1+j) and nu
    log-uniform in [1e-4, 1e-1], one draw per problem from the seed."""
    rng = np.random.default_rng(seed)
    specs = []
    while len(specs) < count:
        n = int(round(math.exp(rng.uniform(math.log(2 ** 11), math.log(2 ** 16)))))
        d = int(round(math.exp(rng.uniform(math.log(32), math.log(1024)))))
        if n < 4 * d:
            continue
        decay = "geom0.9" if rng.random() < 0.5 else "harmonic"
        nu = float(math.exp(rng.uniform(math.log(1e-4), math.log(1e-1))))
        specs.append(dict(n=n, d=d, decay=decay, nu=nu, seed=int(rng.integers(0, 2 ** 31))))
    return specs


def make_batch_torch(count=256, seed=0, device="cuda"):
    """The uneven batch C5 on a torch device: one ``make_problem_torch("C5")``
    per entry of ``batched_specs(count, seed)``.  Returns (specs, problems)
    with problems a list of (A64, b, nu, lam) device tensors."""
    specs = batched_specs(count, seed)
    out = []
    for sp in specs:
        p = make_problem_torch("C5", seed=sp["seed"], device=device, n=sp["n"], d=sp["d"], nu=sp["nu"],
                               decay=sp["decay"])
        out.append((p["A64"], p["b"][:, 0].contiguous(), p["nu"], p["lam"]))
    return specs, out
