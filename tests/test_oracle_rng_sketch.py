"""Pins of the oracle's random draws and embeddings (CPU only).

Each test ties the oracle to something other than itself: published known-
answer vectors, scipy's Hadamard matrix, the explicit Sylvester recursion,
brute-force bijectivity, and the moment identity E[S^T S] = I that the
scalings of Section 2.1 imply.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

from oracle import rng as R
from oracle import sketch as SK

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(t, 16) for t in row]
        out = R.philox4x32_10(v[0], v[1], v[2], v[3], v[4], v[5])
        assert [int(o) for o in out] == v[6:10]


def test_philox_vectorised_matches_scalar():
    c0 = np.arange(50, dtype=np.uint64)
    vec = R.philox4x32_10(c0, 7, 0, 3, 123, 456)
    for i in range(50):
        sc = R.philox4x32_10(i, 7, 0, 3, 123, 456)
        assert [int(v[i]) for v in vec] == [int(s) for s in sc]


def test_uniform_exact_open_interval():
    w = np.array([0, 1, 511, 512, 2 ** 31, 2 ** 32 - 1], dtype=np.uint64)
    u = R.uniform_open01(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)  # exact in fp32
    assert u[0] == 2.0 ** -24 and u[-1] == 1.0 - 2.0 ** -24


def test_gaussian_distribution():
    G = R.gaussian_block(4096, 64, seed=11)
    z = G.ravel()
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / z.size)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3
    # rows are independent of m (nested sketches append rows)
    assert np.array_equal(R.gaussian_block(100, 7, 3), R.gaussian_block(100, 12, 3)[:7])


def test_signs_balanced():
    E = R.srht_signs(1 << 16, seed=5)
    assert set(np.unique(E)) == {-1.0, 1.0}
    assert abs(E.sum()) < 5 * math.sqrt(E.size)


@pytest.mark.parametrize("n_pad", [1, 2, 4, 8, 32, 128, 1024, 4096])
def test_feistel_bijection(n_pad):
    for seed in (0, 1, 2 ** 40 + 17):
        p = R.feistel_permute(np.arange(n_pad, dtype=np.uint64), n_pad, seed)
        assert sorted(p.tolist()) == list(range(n_pad))


def test_feistel_first_index_uniform():
    n_pad = 16
    counts = np.zeros(n_pad)
    for seed in range(4000):
        counts[int(R.feistel_permute(np.array([0], dtype=np.uint64), n_pad, seed)[0])] += 1
    assert scipy.stats.chisquare(counts).pvalue > 1e-4


def test_fwht_matches_scipy_hadamard_and_sylvester():
    rng = np.random.default_rng(0)
    H = np.array([[1.0]])
    for k in range(1, 11):
        H = np.block([[H, H], [H, -H]])
        n = H.shape[0]
        X = rng.standard_normal((n, 3))
        assert np.allclose(SK.fwht(X), H @ X, rtol=0, atol=1e-10 * n)
        assert np.array_equal(H, scipy.linalg.hadamard(n))
    X = rng.standard_normal((256, 2))
    assert np.allclose(SK.fwht(SK.fwht(X)), 256 * X)  # H^2 = n I


@pytest.mark.parametrize("kind", ["srht", "gaussian", "rademacher", "sjlt"])
def test_fast_sketch_equals_explicit_matrix(kind):
    rng = np.random.default_rng(1)
    n, d, m = 300, 7, 24
    A = rng.standard_normal((n, d))
    S = SK.sketch_matrix(kind, n, m, seed=9, sjlt_s=3)
    assert S.shape == (m, n)
    assert np.allclose(SK.sketch(kind, A, m, seed=9, sjlt_s=3), S @ A, rtol=1e-12, atol=1e-12)


def test_srht_full_size_is_orthogonal():
    # m = n_pad: S^T S = (1/n_pad) E H^T H E = I exactly, so H_S = H.
    n = 64
    S = SK.srht_matrix(n, n, seed=4)
    assert np.allclose(S.T @ S, np.eye(n), atol=1e-12)


def test_srht_nested_rows():
    n_pad = 512
    a = SK.srht_rows(40, n_pad, 3)
    b = SK.srht_rows(80, n_pad, 3)
    assert np.array_equal(a, b[:40]) and len(set(b.tolist())) == 80


@pytest.mark.parametrize("kind", ["srht", "gaussian", "rademacher", "sjlt"])
def test_embedding_second_moment_is_identity(kind):
    # E[S^T S] = I for each embedding (the scalings of Section 2.1); Monte Carlo
    # over 3000 seeds, every entry within 5 standard errors.
    n, m, trials = 16, 8, 3000
    acc = np.zeros((n, n))
    acc2 = np.zeros((n, n))
    for seed in range(trials):
        S = SK.sketch_matrix(kind, n, m, seed=seed, sjlt_s=2)
        M = S.T @ S
        acc += M
        acc2 += M * M
    mean = acc / trials
    se = np.sqrt(np.maximum(acc2 / trials - mean ** 2, 1e-30) / trials)
    dev = np.abs(mean - np.eye(n))
    assert np.all(dev <= 5 * se + 1e-12), float(np.max(dev / (se + 1e-12)))


@pytest.mark.parametrize("m,s", [(1, 4), (2, 4), (3, 4), (16, 4), (64, 1), (5, 5)])
def test_sjlt_structure(m, s):
    n = 500
    rows, signs = R.sjlt_rows_signs(n, m, s, seed=21)
    s_eff = min(s, m)
    assert rows.shape == (n, s_eff)
    assert rows.min() >= 0 and rows.max() < m
    for i in range(n):
        assert len(set(rows[i].tolist())) == s_eff
    S = SK.sjlt_matrix(n, m, s, seed=21)
    nz = (S != 0).sum(axis=0)
    assert np.all(nz == s_eff)
    assert np.allclose(np.abs(S[S != 0]), 1 / math.sqrt(s_eff))


def test_sjlt_rows_uniform():
    rows, _ = R.sjlt_rows_signs(20000, 8, 1, seed=2)
    counts = np.bincount(rows[:, 0], minlength=8)
    assert scipy.stats.chisquare(counts).pvalue > 1e-4


def test_rademacher_entries_balanced_nested_and_independent_of_m():
    # +-1 entries, each sign with probability 1/2 (within 5 standard errors over
    # 2^20 entries), row r the same whatever m is, and no two rows of a block
    # of 128 (one Philox call per data row) equal.
    R200 = R.rademacher_block(4096, 256, 17)
    assert set(np.unique(R200).tolist()) == {-1.0, 1.0}
    frac = np.mean(R200 < 0)
    assert abs(frac - 0.5) <= 5 * 0.5 / np.sqrt(R200.size)
    assert np.array_equal(R.rademacher_block(4096, 130, 17), R200[:130])
    block = R200[:128]
    assert len({tuple(r) for r in block.astype(int)}) == 128
    # adjacent sketch rows are uncorrelated (the bits of one word are independent)
    corr = np.mean(R200[:-1] * R200[1:])
    assert abs(corr) <= 5 / np.sqrt(R200[:-1].size)
