"""The three random embeddings of Section 2.1 (oracle side, float64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Every sketch is returned as the "unscaled" matrix Y with S A = scale * Y, where
scale = 1/sqrt(m) for the SRHT and the Gaussian embedding (whose rows are
then independent of m, so a larger sketch appends rows) and scale = 1 for the
SJLT.  ``*_matrix`` builds the m x n matrix S itself for small n, straight from
its definition, so that tests can compare the fast forms with S @ A.
"""
import numpy as np
import scipy.linalg

from . import rng as R


def next_pow2(n):
    """Smallest power of two >= n (the SRHT pads A with zero rows to it;
    footnote of Section 2.1)."""
    p = 1
    while p < n:
        p <<= 1
    return p


# ----------------------------------------------------------------------------
# SRHT  S = R H E  (Section 2.1; normalised H in the proof of Theorem 5.1)
# ----------------------------------------------------------------------------

def fwht(X):
    """Unnormalised Walsh-Hadamard transform along axis 0 in Sylvester order:
    returns H_{+-1} X with H_1 = [1], H_{2k} = [[H_k, H_k], [H_k, -H_k]].
    Pinned against ``scipy.linalg.hadamard`` and the explicit Sylvester
    recursion in the tests."""
    X = np.array(X, dtype=np.float64, copy=True)
    n = X.shape[0]
    assert n & (n - 1) == 0, "length must be a power of two"
    rest = X.shape[1:]
    h = 1
    while h < n:
        Y = X.reshape((n // (2 * h), 2, h) + rest)
        a = Y[:, 0].copy()
        b = Y[:, 1]
        Y[:, 0] = a + b
        Y[:, 1] = a - b
        X = Y.reshape((n,) + rest)
        h *= 2
    return X


def srht_rows(m, n_pad, seed):
    """Indices pi(0..m-1) of the rows kept by the subsampling R."""
    return R.feistel_permute(np.arange(m, dtype=np.uint64), n_pad, seed).astype(np.int64)


def srht_hda(A, seed):
    """B = H_{+-1} E A_pad, the n_pad x d matrix every SRHT of any size m
    subsamples (formed once; growing m only gathers more rows of it)."""
    n = A.shape[0]
    n_pad = next_pow2(n)
    Ap = np.zeros((n_pad,) + A.shape[1:])
    Ap[:n] = A
    E = R.srht_signs(n_pad, seed)
    return fwht(E.reshape((n_pad,) + (1,) * (A.ndim - 1)) * Ap)


def srht_sketch_unscaled(A, m, seed):
    """Y = R H_{+-1} E A_pad (m x d); the SRHT sketch is S A = Y / sqrt(m),
    i.e. S = sqrt(n_pad / m) R H_norm E with H_norm = H_{+-1} / sqrt(n_pad)."""
    n_pad = next_pow2(A.shape[0])
    B = srht_hda(A, seed)
    return B[srht_rows(m, n_pad, seed)]


def srht_matrix(n, m, seed):
    """Explicit m x n SRHT (small n only), from scipy's Sylvester Hadamard."""
    n_pad = next_pow2(n)
    H = scipy.linalg.hadamard(n_pad).astype(np.float64)
    E = R.srht_signs(n_pad, seed)
    rows = srht_rows(m, n_pad, seed)
    S = H[rows] * E[None, :] / np.sqrt(m)
    return S[:, :n]


# ----------------------------------------------------------------------------
# Gaussian embedding, entries N(0, 1/m)
# ----------------------------------------------------------------------------

def gaussian_sketch_unscaled(A, m, seed):
    """Y = G A with G[r, i] the Philox/Box-Muller normals; S A = Y / sqrt(m)."""
    G = R.gaussian_block(A.shape[0], m, seed)
    return G @ A


def gaussian_matrix(n, m, seed):
    return R.gaussian_block(n, m, seed) / np.sqrt(m)


# ----------------------------------------------------------------------------
# Rademacher (sub-Gaussian) embedding, entries +-1/sqrt(m)
# ----------------------------------------------------------------------------

def rademacher_sketch_unscaled(A, m, seed):
    """Y = R A with R[r, i] = +-1 from ``rng.rademacher_block``; S A = Y / sqrt(m)."""
    return R.rademacher_block(A.shape[0], m, seed) @ A


def rademacher_matrix(n, m, seed):
    return R.rademacher_block(n, m, seed) / np.sqrt(m)


# ----------------------------------------------------------------------------
# SJLT: s nonzeros per column, values +-1/sqrt(s)
# ----------------------------------------------------------------------------

def sjlt_matrix(n, m, s, seed):
    """Explicit m x n SJLT: column i has s_eff = min(s, m) nonzeros
    +-1/sqrt(s_eff) at distinct rows h_k(i)."""
    rows, signs = R.sjlt_rows_signs(n, m, s, seed)
    s_eff = rows.shape[1]
    S = np.zeros((m, n))
    for k in range(s_eff):
        S[rows[:, k], np.arange(n)] += signs[:, k] / np.sqrt(s_eff)
    return S


def sjlt_sketch(A, m, s, seed):
    """S A for the SJLT by scatter-add of the scaled data rows (scale = 1)."""
    rows, signs = R.sjlt_rows_signs(A.shape[0], m, s, seed)
    s_eff = rows.shape[1]
    Y = np.zeros((m,) + A.shape[1:])
    for k in range(s_eff):
        np.add.at(Y, rows[:, k], (signs[:, k] / np.sqrt(s_eff)).reshape((-1,) + (1,) * (A.ndim - 1)) * A)
    return Y


# ----------------------------------------------------------------------------

def sketch(kind, A, m, seed, sjlt_s=1):
    """S A (scaled) for kind in {'srht', 'gaussian', 'rademacher', 'sjlt'}."""
    if kind == "srht":
        return srht_sketch_unscaled(A, m, seed) / np.sqrt(m)
    if kind == "gaussian":
        return gaussian_sketch_unscaled(A, m, seed) / np.sqrt(m)
    if kind == "rademacher":
        return rademacher_sketch_unscaled(A, m, seed) / np.sqrt(m)
    if kind == "sjlt":
        return sjlt_sketch(A, m, sjlt_s, seed)
    raise ValueError(kind)


def sketch_matrix(kind, n, m, seed, sjlt_s=1):
    if kind == "srht":
        return srht_matrix(n, m, seed)
    if kind == "gaussian":
        return gaussian_matrix(n, m, seed)
    if kind == "rademacher":
        return rademacher_matrix(n, m, seed)
    if kind == "sjlt":
        return sjlt_matrix(n, m, sjlt_s, seed)
    raise ValueError(kind)
