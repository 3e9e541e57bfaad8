"""Pins of the oracle's gradient formulas (central finite differences) and of
the mixed-precision rounding rules (torch's bfloat16 conversion, exactness of
the hi/lo split)."""
import math

import numpy as np
import pytest
import torch

import synthetic
from oracle import adjoint as ADJ
from oracle import mixed as MX
from oracle import rng as R
from oracle import solvers as S


def _loss(A, B, nu, lam, C):
    return float(np.sum(C * S.direct_solve(A, B, nu, lam)))


def test_gradients_match_central_differences():
    p = synthetic.make_problem("C4", 0, n=96, d=12)
    A, B, nu, lam = p.A, p.b, p.nu, p.lam
    rng = np.random.default_rng(7)
    C = rng.standard_normal(B.shape)
    _, g = ADJ.solve_and_grads(A, B, nu, lam, C)
    h = 1e-3
    # b: coordinate directions
    for i in range(3):
        E = np.zeros_like(B)
        E[i, 1] = h
        fd = (_loss(A, B + E, nu, lam, C) - _loss(A, B - E, nu, lam, C)) / (2 * h)
        assert math.isclose(fd, g["b"][i, 1], rel_tol=1e-6, abs_tol=1e-9)
    # A: random directions (scaled so the step is h in Frobenius norm)
    for _ in range(4):
        D = rng.standard_normal(A.shape)
        D *= h / np.linalg.norm(D)
        fd = (_loss(A + D, B, nu, lam, C) - _loss(A - D, B, nu, lam, C)) / 2
        an = float(np.sum(g["A"] * D))
        assert math.isclose(fd, an, rel_tol=1e-4, abs_tol=1e-9 * h)
    # Lambda
    for i in range(3):
        E = np.zeros_like(lam)
        E[i] = h
        fd = (_loss(A, B, nu, lam + E, C) - _loss(A, B, nu, lam - E, C)) / (2 * h)
        assert math.isclose(fd, g["lam"][i], rel_tol=1e-5, abs_tol=1e-9)
    # nu, with a step relative to nu (a 1e-3 absolute step would be 10% of nu)
    hn = 1e-3 * nu
    fd = (_loss(A, B, nu + hn, lam, C) - _loss(A, B, nu - hn, lam, C)) / (2 * hn)
    assert math.isclose(fd, g["nu"], rel_tol=1e-5)


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(100000).astype(np.float32),
                        (rng.standard_normal(1000) * 1e-30).astype(np.float32),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0], dtype=np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(MX.bf16_round(x), ref)


def test_bf16_ties_to_even():
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert MX.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: ties to even -> 1 + 2^-6
    assert MX.bf16_round(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6


def test_split_hi_lo_accuracy():
    A = np.random.default_rng(1).standard_normal((200, 30)).astype(np.float32)
    hi, lo = MX.split_hi_lo(A)
    assert np.array_equal(MX.bf16_round(hi.astype(np.float32)), hi)
    assert np.array_equal(MX.bf16_round(lo.astype(np.float32)), lo)
    err = np.abs(A.astype(np.float64) - hi - lo)
    assert np.all(err <= np.abs(A) * 2.0 ** -16)


def test_refine_reaches_tolerance_with_inexact_inner():
    p = synthetic.make_problem("C1", 0, n=1024, d=64, nu=1e-4)
    xs = S.direct_solve(p.A, p.b, p.nu, p.lam)
    H32 = S.hessian(p.A, p.nu, p.lam).astype(np.float32)

    def inner(r):  # a float32 direct solve: relative accuracy ~1e-3 at this kappa
        return np.linalg.solve(H32, r.astype(np.float32)).astype(np.float64)

    x, outer = MX.refine(p.A, p.b, p.nu, p.lam, inner, tol=1e-10)
    assert outer > 1
    assert S.rel_err_H(p.A, p.nu, p.lam, x, xs) <= 1e-10


def test_split_rowscaled_exactness():
    # The slices are bfloat16-exact integers in their row units, the remainder
    # is below 2^(e-17), and every class of slice products sums exactly in
    # float32 over 256 terms (the property the tensor-core Gram relies on).
    rng = np.random.default_rng(3)
    X = (rng.standard_normal((40, 300)) * np.exp(rng.uniform(-20, 20, size=(40, 1)))).astype(np.float32)
    X[5] = 0
    hi, lo = MX.split_rowscaled(X)
    assert np.array_equal(MX.bf16_round(hi.astype(np.float32)), hi)
    assert np.array_equal(MX.bf16_round(lo.astype(np.float32)), lo)
    mx = np.max(np.abs(X), axis=1)
    _, e = np.frexp(mx)
    e = e[:, None]
    assert np.all(np.abs(np.ldexp(hi, 8 - e)) <= 256) and np.all(np.abs(np.ldexp(lo, 16 - e)) <= 128)
    assert np.all(np.abs(X.astype(np.float64) - hi - lo) <= np.ldexp(1.0, e - 17))
    assert np.all(hi[5] == 0) and np.all(lo[5] == 0)
    # exact float32 sums of 256 products of each class
    for a, b in ((hi, hi), (hi, lo), (lo, lo)):
        p32 = (a[0, :256].astype(np.float32) * b[1, :256].astype(np.float32))
        s32 = np.float32(0)
        for v in p32:
            s32 = np.float32(s32 + v)
        assert float(s32) == float(np.sum(a[0, :256] * b[1, :256]))


def test_gaussian_sketch_bf16_definition():
    # (a) every entry is the sum over data rows of bf16(G) times A: against a
    # correctly rounded sum (math.fsum) of the products, each of which is
    # exact in float64 (an 8-bit significand times a small integer);
    # (b) it is linear in A; (c) rows are nested:
    # rows [row0, m) of the m-row sketch are its tail, and the first rows do
    # not depend on m.
    rng = np.random.default_rng(11)
    A = rng.integers(-50, 50, size=(300, 7)).astype(np.float32)
    Gb = MX.gaussian_bf16(300, 12, 5)
    Y = MX.gaussian_sketch_bf16(A, 12, 5)
    ref = np.zeros((12, 7))
    for r in range(12):
        for c in range(7):
            ref[r, c] = math.fsum(float(Gb[r, i]) * float(A[i, c]) for i in range(300))
    # recursive summation bound: n u sum |products| (u = 2^-53)
    assert np.all(np.abs(Y - ref) <= 300 * 2.0 ** -53 * (np.abs(Gb) @ np.abs(A.astype(np.float64))))
    A = (rng.standard_normal((500, 9)) * np.exp(rng.uniform(-5, 5, size=(1, 9)))).astype(np.float32)
    B = rng.standard_normal((500, 9)).astype(np.float32)
    Ya, Yb = MX.gaussian_sketch_bf16(A, 16, 7), MX.gaussian_sketch_bf16(B, 16, 7)
    Yab = MX.gaussian_bf16(500, 16, 7) @ (A.astype(np.float64) + B.astype(np.float64))
    assert np.allclose(Ya + Yb, Yab, rtol=1e-12, atol=1e-12 * np.max(np.abs(Yab)))
    assert np.array_equal(MX.gaussian_sketch_bf16(A, 16, 7, row0=9), Ya[9:])
    assert np.array_equal(MX.gaussian_sketch_bf16(A, 10, 7), Ya[:10])


def test_bf16_midpoint_slack():
    # values far from a bfloat16 midpoint have slack 0 and round identically
    # under a small perturbation; values on a midpoint get one bfloat16 step
    g = np.array([1.0, 1.0 + 2 ** -8, 1.5, -3.0 - 2 ** -7], dtype=np.float32)
    sl = MX.bf16_midpoint_slack(g, ulps=2)
    assert sl[0] == 0 and sl[2] == 0
    assert sl[1] >= 2 ** -7 and sl[3] >= 2 ** -6  # at least one bfloat16 step
    rng = np.random.default_rng(2)
    x = rng.standard_normal(20000).astype(np.float32)
    sl = MX.bf16_midpoint_slack(x, ulps=2)
    y = (x + np.spacing(np.abs(x)) * rng.integers(-2, 3, size=x.shape)).astype(np.float32)
    same = MX.bf16_round(x) == MX.bf16_round(y)
    assert np.all(same | (sl > 0))


def test_e4m3_round_matches_torch_float8():
    # the e4m3 rounding written from the format definition against torch's
    # float8_e4m3fn conversion (round to nearest even; finite saturation is
    # applied before the cast, torch maps out-of-range values to NaN)
    rng = np.random.default_rng(8)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-4, 2.6, size=20000),
                        [0.0, 2 ** -9, 2 ** -10, 3 * 2 ** -10, 2 ** -6, 448.0, -448.0, 1.0625, 1.1875, 0.009]])
    x = x.astype(np.float32)
    xs = np.clip(x, -448.0, 448.0).astype(np.float32)
    ref = torch.from_numpy(xs).to(torch.float8_e4m3fn).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(MX.e4m3_round(x), ref)
    # saturation, and exactly representable values stay put
    assert MX.e4m3_round(np.float32(1000.0)) == 448.0
    for v in (1.0, 1.125, 240.0, 2.0 ** -6, 7 * 2.0 ** -9):
        assert MX.e4m3_round(np.float32(v)) == v


def test_gaussian_sketch_e4m3_definition():
    # (a) columns of powers of two times small integers that e4m3 holds after
    # scaling: the sketch is e4m3(G) A exactly; (b) two slices: each slice has
    # its own column scales and their products add; (c) nested rows
    rng = np.random.default_rng(12)
    A = (rng.integers(-7, 8, size=(300, 5)) * np.array([1.0, 2.0 ** 10, 2.0 ** -10, 4.0, 0.5])).astype(np.float32)
    G8 = MX.e4m3_round(R.gaussian_block(300, 6, 3).astype(np.float32))
    assert np.allclose(MX.gaussian_sketch_e4m3(A, 6, 3), G8 @ A.astype(np.float64), rtol=1e-14, atol=0)
    A = rng.standard_normal((700, 4)).astype(np.float32)
    A[400:] *= 1000.0
    sc = MX.e4m3_scales(A, slice_rows=256)
    assert sc.shape == (3, 4) and np.all(sc[2] > 100 * sc[0])
    assert np.all(np.max(np.abs(A[:256]), axis=0) / sc[0] <= 448.0)
    assert np.all(np.max(np.abs(A[:256]), axis=0) / sc[0] > 224.0)  # the least such power of two
    assert np.array_equal(sc[0], np.exp2(np.ceil(np.log2(np.max(np.abs(A[:256]).astype(np.float64), axis=0) / 448))))
    Y = MX.gaussian_sketch_e4m3(A, 9, 5, slice_rows=256)
    G8 = MX.e4m3_round(R.gaussian_block(700, 9, 5).astype(np.float32))
    # within e4m3 rounding of A (relative 2^-4 of each scaled entry)
    bound = (np.abs(G8) @ np.abs(A.astype(np.float64))) * 2.0 ** -4
    assert np.all(np.abs(Y - G8 @ A.astype(np.float64)) <= bound)
    assert np.array_equal(MX.gaussian_sketch_e4m3(A, 9, 5, row0=4, slice_rows=256), Y[4:])
