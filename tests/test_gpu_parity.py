"""GPU parity: every kernel of the hot path against the CPU oracle, through
the C ABI (sizes that span several tiles and ragged tails; edge cases)."""
import math

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


# ----------------------------------------------------------------------------- A-pass (K1)

HESS_SHAPES = [
    (1, 1), (7, 3), (1000, 33), (4096, 256), (5000, 512), (3001, 1000), (2049, 2048), (1500, 4096), (0, 17),
    (700, 4100), (333, 9000), (257, 14336),  # wide rows: x through L1, one CTA per SM
]


@pytest.mark.parametrize("n,d", HESS_SHAPES)
@pytest.mark.parametrize("dtype", ["f64", "f32", "f32ext"])
def test_hess_apply_matches_oracle(n, d, dtype):
    rng = np.random.default_rng(n * 7 + d)
    A = rng.standard_normal((n, d))
    if dtype != "f64":
        A = A.astype(np.float32).astype(np.float64)
    x = rng.standard_normal(d)
    lam = 1 + rng.random(d)
    nu = 0.3
    ref = O.hess_apply(A, nu, lam, x)
    # error scale: |A|^T |A| |x| + nu^2 lam |x|
    scale = np.abs(A).T @ (np.abs(A) @ np.abs(x)) + nu ** 2 * lam * np.abs(x) + 1e-300
    tA = dev(A, torch.float32 if dtype != "f64" else torch.float64)
    got = host(api().hess_apply(tA, dev(x), nu, dev(lam), extended=(dtype == "f32ext")))
    tol = 1e-5 if dtype == "f32" else 1e-13
    assert float(np.max(np.abs(got - ref) / scale)) < tol


def test_hess_apply_padded_leading_dimension():
    rng = np.random.default_rng(3)
    n, d, ld = 777, 250, 256
    buf = rng.standard_normal((n, ld))
    A = buf[:, :d]
    x, lam = rng.standard_normal(d), 1 + rng.random(d)
    ref = O.hess_apply(A, 0.1, lam, x)
    tA = dev(buf)[:, :d]
    got = host(api().hess_apply(tA, dev(x), 0.1, dev(lam)))
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_hess_apply_eight_rhs():
    rng = np.random.default_rng(4)
    n, d = 3000, 1024
    A = rng.standard_normal((n, d)).astype(np.float32).astype(np.float64)
    X = rng.standard_normal((d, 8))
    lam = 1 + rng.random(d)
    ref = O.hess_apply(A, 0.2, lam, X)
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        got = host(api().hess_apply(dev(A, dt), dev(X), 0.2, dev(lam)))
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < tol


# ----------------------------------------------------------------------------- sketches (K2-K5)

@pytest.mark.parametrize("kind", ["srht", "gaussian", "rademacher", "sjlt"])
@pytest.mark.parametrize("n,d,m", [(1000, 40, 24), (4096, 256, 300), (513, 7, 1), (64, 3, 64)])
def test_sketch_matches_oracle_fp64(kind, n, d, m):
    rng = np.random.default_rng(n + d + m)
    A = rng.standard_normal((n, d))
    lam = np.ones(d)
    sk = api().Sketch(dev(A), 0.1, dev(lam), kind=kind, m=m, sjlt_s=3, seed=12345)
    got = host(sk.matrix())
    ref = OS.sketch(kind, A, m, seed=12345, sjlt_s=3)
    scale = np.sqrt(np.sum(A * A, axis=0))[None, :] * (math.sqrt(OS.next_pow2(n) / m) if kind == "srht" else 1.0)
    assert got.shape == ref.shape
    assert float(np.max(np.abs(got - ref) / (scale + 1e-300))) < 1e-12


@pytest.mark.parametrize("kind", ["srht", "sjlt"])
def test_sketch_fp32_within_1e5(kind):
    rng = np.random.default_rng(9)
    n, d, m = 3000, 64, 96
    A = rng.standard_normal((n, d)).astype(np.float32).astype(np.float64)
    sk = api().Sketch(dev(A, torch.float32), 0.1, dev(np.ones(d)), kind=kind, m=m, sjlt_s=4, seed=77)
    got = host(sk.matrix())
    ref = OS.sketch(kind, A, m, seed=77, sjlt_s=4)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


@pytest.mark.parametrize("kind", ["srht", "gaussian", "rademacher", "sjlt"])
def test_sketch_growth_is_nested(kind):
    rng = np.random.default_rng(5)
    n, d = 2000, 30
    A = rng.standard_normal((n, d))
    sk = api().Sketch(dev(A), 0.1, dev(np.ones(d)), kind=kind, m=5, sjlt_s=2, seed=3)
    for m in (10, 20, 40, 80):
        sk.grow(m)
        ref = OS.sketch(kind, A, m, seed=3, sjlt_s=2)
        got = host(sk.matrix())
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("dt,tol", [(torch.float64, 1e-12), (torch.float32, 1e-7)])
def test_srht_multi_pass_transform(dt, tol):
    # n_pad = 2^19: the transform runs in three passes of 7, 6 and 6 levels;
    # d = 37 leaves a ragged column block of 5.
    rng = np.random.default_rng(19)
    n, d, m = 300001, 37, 200
    A = rng.standard_normal((n, d)).astype(np.float32).astype(np.float64)
    sk = api().Sketch(dev(A, dt), 0.1, dev(np.ones(d)), kind="srht", m=m, seed=21)
    got = host(sk.matrix())
    ref = OS.sketch("srht", A, m, seed=21)
    scale = np.sqrt(np.sum(A * A, axis=0))[None, :] * math.sqrt(OS.next_pow2(n) / m)
    assert float(np.max(np.abs(got - ref) / scale)) < tol


@pytest.mark.parametrize("dt,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
@pytest.mark.parametrize("n,d,m", [(5000, 1000, 1), (3001, 2052, 3), (4096, 64, 8), (777, 36, 13), (6000, 520, 40),
                                   (4100, 130, 100), (3000, 100, 300), (20000, 1028, 32), (9000, 130, 64),
                                   (7000, 258, 17)])
def test_sjlt_small_sketch_column_blocks(dt, tol, n, d, m):
    # small and medium m: float32 partial rows in registers (8, 16 rows of 4
    # columns, then eight warp groups), the column-block kernel (partial rows in
    # shared memory: float64, float32 with d not a multiple of 4); d = 2052
    # spans three column blocks of 1024 float32 columns, the last one ragged;
    # n = 20000 takes several 256-row hash batches per CTA; m = 300 is past
    # the shared-memory limit (the L2 scatter).
    rng = np.random.default_rng(n + d + m)
    A = rng.standard_normal((n, d)).astype(np.float32).astype(np.float64)
    sk = api().Sketch(dev(A, dt), 0.1, dev(np.ones(d)), kind="sjlt", m=m, sjlt_s=4, seed=99)
    got = host(sk.matrix())
    ref = OS.sketch("sjlt", A, m, seed=99, sjlt_s=4)
    scale = np.sqrt(np.sum(A * A, axis=0))[None, :]
    assert float(np.max(np.abs(got - ref) / scale)) < tol


@pytest.mark.parametrize("n,d,m,s", [(20000, 1100, 33, 4), (9001, 516, 128, 4), (40000, 260, 200, 4),
                                     (6000, 4096, 256, 4), (20011, 132, 511, 4), (3000, 1028, 512, 4),
                                     (12345, 100, 700, 4), (5000, 64, 1024, 4), (9000, 200, 96, 2),
                                     (9000, 200, 300, 3), (7000, 96, 64, 1)])
def test_sjlt_warp_group_kernel(n, d, m, s):
    # float32, 16 < m <= 512, s <= 4: the sketch rows live in the registers
    # (m <= 128) or per-warp shared-memory slabs (m <= 512) of warp groups
    # (rows g RPG .. (g+1) RPG - 1 of 128 or 64 columns per CTA) fed by a table
    # of the hashed rows sorted by group; m > 512 takes the L2 scatter.
    # Ragged cases: n not a multiple of the 32-row stage, d not a multiple of
    # the 128-column block, m below G RPG, s = 1, 2, 3.
    rng = np.random.default_rng(n + d + m + 7 * s)
    A = rng.standard_normal((n, d)).astype(np.float32).astype(np.float64)
    sk = api().Sketch(dev(A, torch.float32), 0.1, dev(np.ones(d)), kind="sjlt", m=m, sjlt_s=s, seed=123)
    got = host(sk.matrix())
    ref = OS.sketch("sjlt", A, m, seed=123, sjlt_s=s)
    scale = np.sqrt(np.sum(A * A, axis=0))[None, :]
    assert float(np.max(np.abs(got - ref) / scale)) < 1e-5


@pytest.mark.parametrize("dt,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
@pytest.mark.parametrize("n,d,m,s", [(3001, 1100, 257, 4), (5000, 600, 1024, 4), (9000, 64, 4096, 1),
                                     (1000, 2048, 300, 16),
                                     # ragged column blocks (d % 32 != 0), m not a power of two, s = 2, 3
                                     (20000, 100, 1536, 3), (7000, 132, 2000, 4), (30000, 260, 7000, 4),
                                     (8000, 36, 3001, 2)])
def test_sjlt_large_sketch(dt, tol, n, d, m, s):
    # larger m: float64 rows of 16 bytes gather per-sketch-row buckets of data
    # rows (warps over chunks of the bucket-ordered entries), float32 scatters
    # with vector atomics; d = 1100 (float32) and 600 (float64) leave a ragged
    # last column block, n = 9000 rows on m = 4096 and 8192 sketch rows leave
    # many buckets empty or with one row, s = 16 is the largest sparsity.
    rng = np.random.default_rng(n + d + m + s)
    A = rng.standard_normal((n, d)).astype(np.float32).astype(np.float64)
    sk = api().Sketch(dev(A, dt), 0.1, dev(np.ones(d)), kind="sjlt", m=m, sjlt_s=s, seed=31)
    got = host(sk.matrix())
    ref = OS.sketch("sjlt", A, m, seed=31, sjlt_s=s)
    scale = np.sqrt(np.sum(A * A, axis=0))[None, :]
    assert float(np.max(np.abs(got - ref) / scale)) < tol
    sk.grow(2 * m)  # re-hashed into 2m rows in one more pass
    ref2 = OS.sketch("sjlt", A, 2 * m, seed=31, sjlt_s=s)
    assert float(np.max(np.abs(host(sk.matrix()) - ref2) / scale)) < tol


def gpu_sketch_entries(n, m, seed, kind="gaussian", width=4096):
    """The m x n matrix of bfloat16 entries the tensor-core sketch applied
    (unscaled), read back through the same kernel: for a float32 A whose
    columns are unit vectors e_{i0}, ..., e_{i0+w-1}, every split slice is
    exact (hi = 1 or 0, lo = 0) and every output is one exact product, so
    Y = S_bf16[:, i0:i0+w].  The entries depend only on (data row, sketch
    row, seed), not on A."""
    out = np.empty((m, n))
    for i0 in range(0, n, width):
        w = min(width, n - i0)
        wp = (w + 3) // 4 * 4
        A = torch.zeros(n, wp, dtype=torch.float32, device="cuda")
        A[torch.arange(i0, i0 + w, device="cuda"), torch.arange(w, device="cuda")] = 1.0
        sk = api().Sketch(A, 0.1, torch.ones(wp, dtype=torch.float64, device="cuda"), kind=kind, m=m, seed=seed)
        out[:, i0:i0 + w] = host(sk.matrix())[:, :w] * math.sqrt(m)
        del sk, A
    from oracle import mixed as MX
    return MX.bf16_round(out.astype(np.float32))


def tc_sketch_bound(Gb, A32, Y):
    """Element-wise bound of |Y_gpu - bf16(G) A| for the tensor-core sketch
    (unscaled): the element-wise two-slice split of A leaves |a - hi - lo| <=
    2^-17 |a|; the float32 tensor-core accumulation over groups of 256 data
    rows and the float32 sum of the groups cost at most 2^-16 sum |g||a|
    (measured and asserted since the kernel's first parity test); the final
    rounding to float32 half an ulp of |Y|."""
    absGA = np.abs(Gb) @ np.abs(A32.astype(np.float64))
    return (2.0 ** -17 + 2.0 ** -16) * absGA + 2.0 ** -23 * np.abs(Y)


@pytest.mark.parametrize("n,d,m", [(3000, 64, 96), (20000, 300, 200), (777, 5, 130), (40000, 520, 257)])
def test_gaussian_tc_sketch_matches_plain_definition(n, d, m):
    # float32 A: bf16(G) A on tcgen05; n = 20000 and 40000 span two and three
    # K slices, d = 300 / 520 two and three column tiles, m = 257 three row
    # tiles with a ragged tail.  Reference: the plain definition (1/sqrt m)
    # bf16(G) A in float64 with G from the oracle's Philox / Box-Muller.
    from oracle import mixed as MX
    from oracle import rng as R
    rng = np.random.default_rng(n + d)
    A = (rng.standard_normal((n, d)) * rng.uniform(0.1, 10, size=(1, d))).astype(np.float32)
    sk = api().Sketch(dev(A.astype(np.float64), torch.float32), 0.1, dev(np.ones(d)), kind="gaussian", m=m, seed=31)
    got = host(sk.matrix()) * math.sqrt(m)
    # (1) the embedding's entries: bf16 of the oracle's float32 Gaussian draws,
    # bit for bit, except within 4 float32 ulps of a bfloat16 rounding
    # midpoint, where the GPU's float32 Box-Muller may round to the other
    # neighbour
    G32 = R.gaussian_block(n, m, 31).astype(np.float32)
    Gor = MX.bf16_round(G32)
    Ggpu = gpu_sketch_entries(n, m, 31)
    slack = MX.bf16_midpoint_slack(G32, ulps=4)
    assert np.array_equal(Ggpu[slack == 0], Gor[slack == 0])
    assert np.all(np.abs(Ggpu - Gor) <= slack)
    # (2) the product: against the plain definition with those entries,
    # element-wise within the split and accumulation bound, and S A within
    # 1e-5 relative (Frobenius) in float32
    ref = Ggpu @ A.astype(np.float64)
    assert np.all(np.abs(got - ref) <= tc_sketch_bound(Ggpu, A, ref)), \
        float(np.max(np.abs(got - ref) / tc_sketch_bound(Ggpu, A, ref)))
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    # and against the oracle's own sketch (its bf16 entries): the same, plus
    # one bfloat16 step at each ambiguous entry
    ref_or = MX.gaussian_sketch_bf16(A, m, 31)
    amb = slack @ np.abs(A.astype(np.float64))
    assert np.all(np.abs(got - ref_or) <= tc_sketch_bound(Gor, A, ref_or) + amb)


@pytest.mark.parametrize("n,d,m", [(3000, 64, 96), (20000, 300, 200), (40000, 520, 257)])
def test_rademacher_tc_sketch_matches_plain_definition(n, d, m):
    # +-1 entries are exact in bfloat16: the plain definition R A (float64)
    # and the split and accumulation bound
    from oracle import rng as R
    rng = np.random.default_rng(n + d + 1)
    A = (rng.standard_normal((n, d)) * rng.uniform(0.1, 10, size=(1, d))).astype(np.float32)
    sk = api().Sketch(dev(A.astype(np.float64), torch.float32), 0.1, dev(np.ones(d)), kind="rademacher", m=m,
                      seed=13)
    got = host(sk.matrix()) * math.sqrt(m)
    Rm = R.rademacher_block(n, m, 13)
    assert np.array_equal(gpu_sketch_entries(min(n, 3000), m, 13, kind="rademacher"), Rm[:, :min(n, 3000)])
    ref = Rm @ A.astype(np.float64)
    assert np.all(np.abs(got - ref) <= tc_sketch_bound(Rm, A, ref))
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("n,d,m", [(3000, 64, 96), (20000, 300, 200), (40000, 520, 257)])
def test_e4m3_tc_sketch_matches_definition(n, d, m):
    # the 8-bit Gaussian sketch: e4m3(G) times A quantised to e4m3 against one
    # power-of-two scale per column and slice of 16384 rows, each slice scaled
    # back; n = 20000 / 40000 span two / three slices with their own scales
    from oracle import mixed as MX
    from oracle import rng as R
    rng = np.random.default_rng(n + d + 7)
    A = (rng.standard_normal((n, d)) * rng.uniform(0.1, 10, size=(1, d))).astype(np.float32)
    A[n // 2:] *= 30.0  # slices with different scales
    sk = api().Sketch(dev(A.astype(np.float64), torch.float32), 0.1, dev(np.ones(d)), kind="gaussian-e4m3", m=m,
                      seed=17)
    got = host(sk.matrix()) * math.sqrt(m)
    G32 = R.gaussian_block(n, m, 17).astype(np.float32)
    Gor = MX.e4m3_round(G32)
    # unit columns make every scaled entry 256 = 2^8 against a scale 2^-8: exact
    Ggpu = gpu_sketch_entries(n, m, 17, kind="gaussian-e4m3")
    Ggpu = MX.e4m3_round(Ggpu.astype(np.float32))
    slack = MX.e4m3_midpoint_slack(G32, ulps=4)
    assert np.array_equal(Ggpu[slack == 0], Gor[slack == 0])
    assert np.all(np.abs(Ggpu - Gor) <= slack)
    sc = MX.e4m3_scales(A)
    ref = np.zeros((m, d))
    absref = np.zeros((m, d))
    for k in range(sc.shape[0]):
        blk = slice(k * 16384, (k + 1) * 16384)
        A8 = MX.e4m3_round((A[blk].astype(np.float64) / sc[k][None, :]).astype(np.float32)) * sc[k][None, :]
        ref += Ggpu[:, blk] @ A8
        absref += np.abs(Ggpu[:, blk]) @ np.abs(A8)
    bound = 2.0 ** -16 * absref + 2.0 ** -23 * np.abs(ref)  # float32 accumulation; the products are exact
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / (bound + 1e-300)))
    # and the oracle's own definition (its e4m3 entries), up to the midpoint entries
    ref_or = MX.gaussian_sketch_e4m3(A, m, 17)
    amb = slack @ np.abs(A.astype(np.float64))
    assert np.all(np.abs(got - ref_or) <= bound + 1.01 * amb)


@pytest.mark.parametrize("nu,expect_e4m3", [(3e-2, 1), (1e-4, 0)])
def test_e4m3_sketch_gate_and_mixed_solve(nu, expect_e4m3):
    # the adaptive solver takes 8 bits only when 2^-8/3 ||A||_F^2 / d <= 0.1 nu^2 min lambda
    # (C4's spectrum and Lambda; at nu = 1e-4 the estimate rules 8 bits out and the
    # bfloat16 split serves instead); either way the mixed form reaches 1e-8
    p = synthetic.make_problem("C4", 5, n=8192, d=256, k=1, nu=nu, dtype="f32")
    b = p.b[:, 0] if p.b.ndim == 2 else p.b
    xs = O.direct_solve(p.A, b, p.nu, p.lam)
    x, st, _ = api().adaptive_pcg(dev(p.A, torch.float32), dev(b), p.nu, dev(p.lam), kind="gaussian-e4m3", tol=1e-8,
                                  precision="mixed", seed=3)
    assert st["sketch_e4m3"] == expect_e4m3
    assert O.rel_err_H(p.A, p.nu, p.lam, host(x), xs) <= 1e-8
    noise = 2.0 ** -8 / 3 * np.sum(p.A.astype(np.float64) ** 2) / p.d
    assert (noise <= 0.1 * p.nu ** 2 * np.min(p.lam)) == bool(expect_e4m3)


def test_gaussian_tc_sketch_nested_growth():
    # m = 1, 2, 3, 6, 13: new rows start at offsets that are not multiples of
    # the four rows one Philox call gives
    from oracle import mixed as MX
    from oracle import rng as R
    rng = np.random.default_rng(4)
    n, d = 5000, 40
    A = rng.standard_normal((n, d)).astype(np.float32)
    sk = api().Sketch(dev(A.astype(np.float64), torch.float32), 0.1, dev(np.ones(d)), kind="gaussian", m=1, seed=8)
    for m in (2, 3, 6, 13):
        sk.grow(m)
        got = host(sk.matrix()) * math.sqrt(m)
        G32 = R.gaussian_block(n, m, 8).astype(np.float32)
        Gor = MX.bf16_round(G32)
        ref = MX.gaussian_sketch_bf16(A, m, 8)
        amb = MX.bf16_midpoint_slack(G32, ulps=4) @ np.abs(A.astype(np.float64))
        assert np.all(np.abs(got - ref) <= tc_sketch_bound(Gor, A, ref) + amb)


def test_srht_full_size_gives_exact_hessian():
    # m = n_pad: S^T S = I, so (SA)^T SA = A^T A exactly (up to rounding).
    rng = np.random.default_rng(1)
    A = rng.standard_normal((128, 16))
    sk = api().Sketch(dev(A), 0.1, dev(np.ones(16)), kind="srht", m=128, seed=8)
    SA = host(sk.matrix())
    assert np.allclose(SA.T @ SA, A.T @ A, rtol=1e-12, atol=1e-11)


# ----------------------------------------------------------------------------- preconditioner (a5, a6)

@pytest.mark.parametrize("m,d", [(1, 40), (17, 40), (39, 40), (40, 40), (100, 40), (300, 256), (64, 300)])
def test_preconditioner_apply_matches_oracle(m, d):
    rng = np.random.default_rng(m * 13 + d)
    n = 2000
    A = rng.standard_normal((n, d)) * (0.9 ** np.arange(d))[None, :]
    lam = 1 + 9 * rng.random(d)
    nu = 1e-2
    sk = api().Sketch(dev(A), nu, dev(lam), kind="gaussian", m=m, seed=4)
    P = api().Preconditioner(sk)
    Z = rng.standard_normal((d, 3))
    got = host(P.apply(dev(Z)))
    ref = O.Preconditioner(OS.sketch("gaussian", A, m, seed=4), nu, lam).apply(Z)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-9


def test_precond_rejects_lambda_below_one():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((100, 8))
    lam = np.ones(8)
    lam[3] = 0.5
    sk = api().Sketch(dev(A), 0.1, dev(lam), kind="gaussian", m=4, seed=1)
    from paper_2104_14101_gb300._lib import SksError
    with pytest.raises(SksError) as e:
        api().Preconditioner(sk)
    assert "lambda" in str(e.value)


# ----------------------------------------------------------------------------- adaptive solvers (a7-a11)

def _xstar(p):
    return O.direct_solve(p.A, p.b, p.nu, p.lam)


@pytest.mark.parametrize("method", ["pcg", "ihs"])
@pytest.mark.parametrize("kind", ["gaussian", "srht", "sjlt", "rademacher"])
def test_adaptive_solve_reaches_tolerance(method, kind):
    p = synthetic.make_problem("C1", 0, n=2048, d=96, nu=1e-3, decay="harmonic", lam="one_plus_9u")
    xs = _xstar(p)
    fn = api().adaptive_pcg if method == "pcg" else api().adaptive_ihs
    x, st, _ = fn(dev(p.A), dev(p.b), p.nu, dev(p.lam), kind=kind, m_init=1, tol=1e-10, sjlt_s=2, seed=11)
    err = O.rel_err_H(p.A, p.nu, p.lam, host(x), xs)
    assert err <= 1e-10, (err, st)
    assert st["status_name"] == "OK"


@pytest.mark.parametrize("method", ["pcg", "ihs"])
@pytest.mark.parametrize("kind", ["gaussian", "srht", "rademacher", "sjlt"])
def test_m_sequence_matches_oracle(method, kind):
    # Plain float64: the GPU takes the same accept/reject decisions as the
    # oracle (literal restart), except where the oracle's ratio sits within
    # 1e-9 of the threshold.
    p = synthetic.make_problem("C1", 1, n=1024, d=64, nu=1e-2)
    fo = O.adaptive_pcg if method == "pcg" else O.adaptive_ihs
    kw = dict(literal_restart=True) if method == "pcg" else {}
    xo, so, to = fo(p.A, p.b, p.nu, p.lam, kind=kind, seed=5, m_init=1, tol=1e-10, **kw)
    fg = api().adaptive_pcg if method == "pcg" else api().adaptive_ihs
    xg, sg, tg = fg(dev(p.A), dev(p.b), p.nu, dev(p.lam), kind=kind, m_init=1, tol=1e-10, seed=5,
                    reuse_residual=False, trace_cap=4096)
    for eo, eg in zip(to, tg):
        if abs(eo["ratio"] / eo["thr"] - 1) < 1e-9:
            break
        assert (eo["t"], eo["m"], eo["accepted"]) == (eg["t"], eg["m"], eg["accepted"])
        if eo["ratio"] > 1e-12:  # below that the decrements are rounding noise
            assert math.isclose(eo["ratio"], eg["ratio"], rel_tol=1e-6)
    else:
        assert len(to) == len(tg)
        assert so["final_m"] == sg["final_m"] and so["iters"] == sg["iters"]


@pytest.mark.parametrize("method", ["pcg", "ihs"])
@pytest.mark.parametrize("kind", ["gaussian", "srht", "sjlt"])
def test_corollary_2_5_no_rejection_under_E_rho(method, kind):
    # Every step the GPU takes with a sketch in E_rho (||C_S - I||_2 <=
    # sqrt(rho), C_S from the oracle's sketch of the same size and seed:
    # the integer streams are bit-identical) passes the improvement test
    # (Corollary 2.5), including the first step after a restart.
    rho = 0.125
    p = synthetic.make_problem("C1", 0, n=8192, d=32, nu=0.1)
    sk = O._Sketcher(p.A, kind, 3, 2)
    dev_of = {}
    held = 0
    fg = api().adaptive_pcg if method == "pcg" else api().adaptive_ihs
    for m_init in (1, 64, 2048):
        _, _, tg = fg(dev(p.A), dev(p.b), p.nu, dev(p.lam), kind=kind, m_init=m_init, tol=1e-10, seed=3, sjlt_s=2,
                      rho=rho, trace_cap=4096)
        for ev in tg:
            m = ev["m"]
            if m not in dev_of:
                e = O.cs_eigenvalues(p.A, sk(m), p.nu, p.lam)
                dev_of[m] = max(abs(e[0] - 1.0), abs(e[-1] - 1.0))
            if dev_of[m] <= math.sqrt(rho):
                held += 1
                assert ev["accepted"], ev
    assert held >= 5


@pytest.mark.parametrize("method", ["pcg", "ihs"])
@pytest.mark.parametrize("kind", ["srht", "gaussian", "sjlt"])
def test_certified_stop_rule(method, kind):
    # Remark 4.2: stop when delta~_t <= eps / (m_delta + 1), eps = 1/2 tol^2 ||x*||_H^2
    # (estimated by b^T x_t), with m_delta of Theorem 5.1 / 5.2 at d_e := d and
    # d_e^2/delta for the SJLT; then delta_t <= eps.
    p = synthetic.make_problem("C1", 2, n=2048, d=64, nu=1e-2)
    xs = _xstar(p)
    tol, delta = 1e-6, 0.05
    fn = api().adaptive_pcg if method == "pcg" else api().adaptive_ihs
    kw = dict(kind=kind, m_init=1, tol=tol, seed=3, sjlt_s=2)
    _, s0, _ = fn(dev(p.A), dev(p.b), p.nu, dev(p.lam), **kw)
    x1, s1, _ = fn(dev(p.A), dev(p.b), p.nu, dev(p.lam), stop_rule="certified", cert_delta=delta, **kw)
    md = {"srht": O.m_delta_srht(p.d, p.n, delta), "gaussian": O.m_delta_gaussian(p.d, delta),
          "sjlt": p.d ** 2 / delta}[kind]
    btx = float(p.b @ host(x1))
    dt_paper = s1["final_delta_tilde"] / (2.0 if method == "pcg" else 1.0)  # Algorithm 2's decrement has no 1/2
    assert dt_paper <= O.termination_threshold(0.5 * tol ** 2 * btx, md) * (1 + 1e-9)
    assert s1["iters"] > s0["iters"]
    assert O.rel_err_H(p.A, p.nu, p.lam, host(x1), xs) <= tol


def test_config1_full_size():
    # C1 at its stated size: Gaussian, m_init = 1, tol 1e-10, float64.
    p = synthetic.make_problem("C1", 0)
    xs = p.V @ ((p.sigma / (p.sigma ** 2 + p.nu ** 2)) * (p.U.T @ p.y))
    x, st, _ = api().adaptive_pcg(dev(p.A), dev(p.b), p.nu, dev(p.lam), kind="gaussian", m_init=1, tol=1e-10, seed=0)
    assert O.rel_err_H(p.A, p.nu, p.lam, host(x), xs) <= 1e-10
    assert st["final_m"] <= 4096


def test_config2_full_size():
    # C2 at its stated size: n = 2^17, d = 2048, sigma_j = 1/(1+j), nu = 1e-3,
    # Lambda = diag(1 + 9 U[0,1]), b = A^T y + 0.1 N(0,1)^d, SRHT, m 16 -> 4096,
    # adaptive PCG and adaptive IHS in float64 to tol 1e-10, each against the
    # oracle's direct solve on all of A (2 GiB, generated on the device).
    prob = synthetic.make_problem_torch("C2", seed=0, device="cuda")
    A, b, lam, nu = prob["A64"], prob["b"][:, 0].contiguous(), prob["lam"], prob["nu"]
    An, bn, ln = host(A), host(b), host(lam)
    xs = O.direct_solve(An, bn, nu, ln)
    for fn, name in ((api().adaptive_pcg, "pcg"), (api().adaptive_ihs, "ihs")):
        x, st, _ = fn(A, b, nu, lam, kind="srht", m_init=16, m_max=4096, tol=1e-10, seed=0, max_iter=2000)
        err = O.rel_err_H(An, nu, ln, host(x), xs)
        assert err <= 1e-10, (name, err, st)
        assert st["final_m"] <= 4096


def test_zero_rhs_returns_zero():
    p = synthetic.make_problem("C1", 0, n=512, d=32)
    x, st, _ = api().adaptive_pcg(dev(p.A), dev(np.zeros(32)), p.nu, dev(p.lam), kind="srht")
    assert float(torch.abs(x).max()) == 0.0 and st["iters"] == 0


def test_max_iter_reports_no_convergence():
    p = synthetic.make_problem("C1", 0, n=1024, d=64, nu=1e-4)
    from paper_2104_14101_gb300._lib import SksError
    with pytest.raises(SksError) as e:
        api().adaptive_pcg(dev(p.A), dev(p.b), p.nu, dev(p.lam), kind="srht", m_init=1, tol=1e-14, max_iter=2)
    assert "NO_CONVERGENCE" in str(e.value)


def test_multiple_rhs_solved_columnwise():
    p = synthetic.make_problem("C4", 0, n=2048, d=64, k=3, dtype="f64")
    xs = O.direct_solve(p.A, p.b, p.nu, p.lam)
    x, st, _ = api().adaptive_pcg(dev(p.A), dev(p.b), p.nu, dev(p.lam), kind="gaussian", tol=1e-10)
    for c in range(3):
        assert O.rel_err_H(p.A, p.nu, p.lam, host(x)[:, c], xs[:, c]) <= 1e-10


# ----------------------------------------------------------------------------- mixed form (a12)

@pytest.mark.parametrize("method", ["pcg", "ihs"])
@pytest.mark.parametrize("kind", ["gaussian", "sjlt", "srht", "rademacher"])
def test_mixed_refined_reaches_1e8(method, kind):
    # C3 recipe at a reduced size: float32 A, nu = 1e-4, kappa(H) ~ 1e8.
    p = synthetic.make_problem("C3", 0, n=8192, d=256)
    xs = O.direct_solve(p.A, p.b, p.nu, p.lam)  # A is the exact upcast of the float32 matrix
    fn = api().adaptive_pcg if method == "pcg" else api().adaptive_ihs
    x, st, tr = fn(dev(p.A, torch.float32), dev(p.b), p.nu, dev(p.lam), kind=kind, m_init=1, tol=1e-8, sjlt_s=4,
                   precision="mixed", seed=2, trace_cap=4096, max_iter=2000)
    err = O.rel_err_H(p.A, p.nu, p.lam, host(x), xs)
    assert err <= 1e-8, (err, st)
    assert st["outer_iters"] >= 2
    assert max(e["outer"] for e in tr) >= 1


@pytest.mark.parametrize("kind", ["gaussian", "sjlt"])
def test_mixed_refined_ill_conditioned_woodbury(kind):
    # d = 1024 with sigma down to ~1e-6 and nu = 1e-4: the Woodbury phases
    # (m < d) factor W_S with eigenvalues near nu^2, where the apply's
    # cancellation demands an accurate W^{-1}.
    p = synthetic.make_problem("C3", 1, n=16384, d=1024)
    xs = O.direct_solve(p.A, p.b, p.nu, p.lam)
    x, st, _ = api().adaptive_pcg(dev(p.A, torch.float32), dev(p.b), p.nu, dev(p.lam), kind=kind, m_init=1,
                                  tol=1e-8, sjlt_s=4, precision="mixed", seed=4, max_iter=3000)
    assert O.rel_err_H(p.A, p.nu, p.lam, host(x), xs) <= 1e-8, st
    assert st["iters"] > 0


def test_mixed_requires_float32_A():
    p = synthetic.make_problem("C1", 0, n=512, d=32)
    from paper_2104_14101_gb300._lib import SksError
    with pytest.raises(SksError):
        api().adaptive_pcg(dev(p.A), dev(p.b), p.nu, dev(p.lam), precision="mixed")


def test_gpu_generator_matches_spectrum():
    # make_problem_torch (used by the benchmark) follows the same recipe.
    prob = synthetic.make_problem_torch("C2", seed=0, device="cuda", n=4096, d=128)
    s = np.linalg.svd(host(prob["A64"]), compute_uv=False)
    assert np.allclose(s, synthetic.spectrum("harmonic", 128), rtol=1e-10)


# ----------------------------------------------------------------------------- tensor-core Gram (K6, float32 sketches)

def _inv_sqrt_spd(M):
    w, Q = np.linalg.eigh(M)
    return (Q / np.sqrt(w)[None, :]) @ Q.T


@pytest.mark.parametrize("m,d,nu,kind", [(300, 256, 1e-2, "rademacher"), (700, 520, 1e-2, "gaussian"),
                                         (64, 64, 1e-2, "srht"), (100, 300, 0.5, "rademacher"),
                                         (1, 64, 0.5, "gaussian"), (129, 200, 0.5, "srht")])
def test_tensor_core_preconditioner_spectrally_close_to_oracle(m, d, nu, kind):
    # A float32 sketch's H_S (m >= d) or W_S (m < d) is built on the tensor
    # cores.  Reference: the oracle's own sketch S A (float64, same seed) and
    # H_S = (SA)^T SA + nu^2 Lambda by definition.  The GPU's preconditioner
    # P must satisfy  eig(H_S^{1/2} P H_S^{1/2}) in [1/(1+eps), 1/(1-eps)]
    # (the event E_rho of Section 2.2 is a statement about exactly this
    # spectrum), with eps the sum of
    #   eps_s:  the GPU sketch's own deviation, ||H_S^{-1/2}(H(Y_gpu) - H_S)H_S^{-1/2}||,
    #           computed exactly from the GPU's float32 sketch (asserted <= 1e-3:
    #           a wrong sketch fails here);
    #   eps_sp: the Gram operand's two-slice bfloat16 split, |y - hi - lo| <=
    #           2^(e-17) against the maximum exponent e of the split row
    #           (a column of Y for H_S, a row of Z = Y Lambda^{-1/2}, itself
    #           rounded to float32, for W_S): with E bounded entry-wise by
    #           that, ||H_S^{-1/2} Delta H_S^{-1/2}|| <= 2 sqrt(1+eps_s) t + t^2,
    #           t = c ||E M|| bounded through the diagonal scaling M = D^{-1/2}
    #           (divided by sqrt(lambda_min(D^{-1/2} H_S D^{-1/2}))) or
    #           through M = Lambda^{-1/2}/nu (H_S >= nu^2 Lambda);
    #   1e-6:   float64 factorisation and the float64 inverse factor.
    from oracle import mixed as MX
    from oracle import sketch as OS
    rng = np.random.default_rng(m * 7 + d)
    n = 3000
    A = (rng.standard_normal((n, d)) * (0.9 ** np.arange(d))[None, :]).astype(np.float32).astype(np.float64)
    lam = 1 + 9 * rng.random(d)
    sk = api().Sketch(dev(A, torch.float32), nu, dev(lam), kind=kind, m=m, seed=6)
    if kind == "gaussian":  # the mixed form's embedding: bf16-rounded Gaussian entries
        SA_or = MX.gaussian_sketch_bf16(A.astype(np.float32), m, 6) / math.sqrt(m)
    else:
        SA_or = OS.sketch(kind, A, m, seed=6)
    c = 1.0 / math.sqrt(m)
    H_or = SA_or.T @ SA_or + nu ** 2 * np.diag(lam)
    Hi = _inv_sqrt_spd(H_or)
    Y = host(sk.matrix()) / c  # the GPU's float32 sketch (unscaled), used only to measure its deviation
    H_y = c * c * Y.T @ Y + nu ** 2 * np.diag(lam)
    eps_s = float(np.linalg.norm(Hi @ (H_y - H_or) @ Hi, 2))
    assert eps_s <= 1e-3
    Y32 = Y.astype(np.float32).astype(np.float64)
    if m >= d:
        _, e = np.frexp(np.max(np.abs(Y32), axis=0))
        E = np.ldexp(1.0, e - 17)[None, :] * np.ones((m, 1))
    else:
        Z = (Y32 / np.sqrt(lam)[None, :]).astype(np.float32).astype(np.float64)
        _, e = np.frexp(np.max(np.abs(Z), axis=1))
        E = (np.ldexp(1.0, e - 17)[:, None] + 2.0 ** -24 * np.abs(Z)) * np.sqrt(lam)[None, :]
    D = np.sqrt(np.diag(H_or))
    K = H_or / D[:, None] / D[None, :]
    t = min(c * np.linalg.norm(E / D[None, :]) / math.sqrt(np.linalg.eigvalsh(K)[0]),
            c * np.linalg.norm(E / np.sqrt(lam)[None, :]) / nu)
    eps = eps_s + 2 * math.sqrt(1 + eps_s) * t + t * t + 1e-6
    assert eps <= 0.05  # the check below is meaningful
    P = api().Preconditioner(sk)
    Pinv = host(P.apply(dev(np.eye(d))))
    Pinv = 0.5 * (Pinv + Pinv.T)
    Hs = np.linalg.cholesky(H_or)
    ev = np.linalg.eigvalsh(Hs.T @ Pinv @ Hs)  # similar to H_S^{1/2} P H_S^{1/2}
    assert ev[0] >= 1.0 / (1.0 + eps) and ev[-1] <= 1.0 / (1.0 - eps), (ev[0], ev[-1], eps)


@pytest.mark.parametrize("m,d,nu,kind", [(300, 256, 0.1, "gaussian"), (700, 520, 1e-2, "rademacher"),
                                         (64, 64, 1e-2, "srht"), (2000, 1100, 3e-2, "sjlt"),
                                         (100, 300, 1e-2, "rademacher"), (1, 64, 0.5, "gaussian"),
                                         (129, 200, 0.5, "srht"), (1000, 1500, 3e-2, "gaussian")])
def test_mixed_factorisation_matches_float64(m, d, nu, kind):
    # The mixed form factors the same tensor-core Gram matrix G (H_S for m >= d,
    # W_S for m < d) as the plain build, but in double-float arithmetic, with the
    # inverse factor merged in float32 (m >= d) or double-float (m < d).  With
    # P64 from the float64 build standing for G's exact preconditioner, the
    # eigenvalues of P64^{-1/2} P P64^{-1/2} must lie within 1 +- tol, tol a
    # first-order error estimate with a safety factor of 8 (u = 2^-44 for a
    # double-float operation chain, 2^-24 for float32, n the order of G):
    #   m >= d:  8 n u_df kappa(H_S) + 8 n u_32 sqrt(kappa(H_S))   (|X L - I| ~ n u kappa(L))
    #   m <  d:  8 m u_df kappa(W_S)^2  (an error E in W_S^{-1} moves the apply
    #            (Lambda^{-1}/nu^2)(I - Z^T W_S^{-1} Z) by ||E|| relative to its
    #            smallest eigenvalue 1/kappa(W_S))
    # plus 1e-9 for the float64 build.  Blocks of 64: several block columns, a
    # ragged last block and merges up to 512 are covered.
    rng = np.random.default_rng(m * 13 + d)
    n = 3000
    A = (rng.standard_normal((n, d)) * (0.97 ** np.arange(d))[None, :] / math.sqrt(n)).astype(np.float32)
    lam = 1 + 9 * rng.random(d)
    sk = api().Sketch(dev(A.astype(np.float64), torch.float32), nu, dev(lam), kind=kind, m=m, sjlt_s=4, seed=9)
    P64 = host(api().Preconditioner(sk).apply(dev(np.eye(d))))
    Pm = host(api().Preconditioner(sk, precision="mixed").apply(dev(np.eye(d))))
    P64 = 0.5 * (P64 + P64.T)
    Pm = 0.5 * (Pm + Pm.T)
    G = np.linalg.inv(P64)
    G = 0.5 * (G + G.T)
    Lg = np.linalg.cholesky(G)
    ev = np.linalg.eigvalsh(Lg.T @ Pm @ Lg)
    Y = host(sk.matrix())  # scaled S A
    if m >= d:
        kappa = np.linalg.cond(G)
        tol = 8 * d * 2.0 ** -44 * kappa + 8 * d * 2.0 ** -24 * math.sqrt(kappa) + 1e-9
    else:
        w = np.linalg.eigvalsh((Y / lam[None, :]) @ Y.T)
        kappa = (w[-1] + nu ** 2) / nu ** 2
        tol = 8 * m * 2.0 ** -44 * kappa ** 2 + 1e-9
    assert tol <= 0.05  # the check is meaningful
    assert np.all(np.abs(ev - 1.0) <= tol), (ev[0], ev[-1], tol, kappa)


# ----------------------------------------------------------------------------- adjoint (a13)

@pytest.mark.parametrize("precision", ["plain", "mixed"])
def test_adjoint_matches_oracle_gradient(precision):
    # C4 recipe at n=4096, d=256, 8 right-hand sides; loss L = sum_k c_k^T x_k.
    from oracle import adjoint as OA
    p = synthetic.make_problem("C4", 0, n=4096, d=256)
    rng = np.random.default_rng(1)
    Cw = rng.standard_normal(p.b.shape)
    Xo, go = OA.solve_and_grads(p.A, p.b, p.nu, p.lam, Cw)
    dt = torch.float64 if precision == "plain" else torch.float32
    tA = dev(p.A, dt).requires_grad_(True)
    tb = dev(p.b).requires_grad_(True)
    tlam = dev(p.lam).requires_grad_(True)
    tnu = torch.tensor(p.nu, dtype=torch.float64, device="cuda", requires_grad=True)
    tol = 1e-10 if precision == "plain" else 1e-8
    x = api().sketch_solve(tA, tb, tnu, tlam, kind="gaussian", m_init=1, tol=tol, precision=precision, seed=3)
    loss = (x * dev(Cw)).sum()
    loss.backward()
    gtol = 1e-7 if precision == "plain" else 1e-5
    assert np.max(np.abs(host(tb.grad) - go["b"])) / np.max(np.abs(go["b"])) < gtol
    assert np.max(np.abs(host(tA.grad).astype(np.float64) - go["A"])) / np.max(np.abs(go["A"])) < gtol
    assert np.max(np.abs(host(tlam.grad) - go["lam"])) / np.max(np.abs(go["lam"])) < gtol
    assert abs(float(tnu.grad) - go["nu"]) / abs(go["nu"]) < gtol


def test_adjoint_central_differences():
    # Directional central differences (h = 1e-3; for nu a step of 1e-3 * nu)
    # of L = c^T x(A, b, nu, Lambda) with the plain float64 solver.
    p = synthetic.make_problem("C4", 0, n=4096, d=256, k=1)
    rng = np.random.default_rng(2)
    cw = rng.standard_normal(256)
    opts = dict(kind="gaussian", m_init=1, tol=1e-12, seed=3)

    def L(A, b, nu, lam):
        x, _, _ = api().adaptive_pcg(dev(A), dev(b), nu, dev(lam), **opts)
        return float(np.dot(cw, host(x)))

    tA = dev(p.A).requires_grad_(True)
    tb = dev(p.b[:, 0]).requires_grad_(True)
    tlam = dev(p.lam).requires_grad_(True)
    tnu = torch.tensor(p.nu, dtype=torch.float64, device="cuda", requires_grad=True)
    x = api().sketch_solve(tA, tb, tnu, tlam, **opts)
    (x * dev(cw)).sum().backward()
    h = 1e-3
    D = rng.standard_normal(p.A.shape)
    D *= h / np.linalg.norm(D)
    fd = (L(p.A + D, p.b[:, 0], p.nu, p.lam) - L(p.A - D, p.b[:, 0], p.nu, p.lam)) / 2
    assert math.isclose(fd, float(np.sum(host(tA.grad) * D)), rel_tol=1e-4)
    e = np.zeros(256)
    e[7] = h
    fd = (L(p.A, p.b[:, 0] + e, p.nu, p.lam) - L(p.A, p.b[:, 0] - e, p.nu, p.lam)) / (2 * h)
    assert math.isclose(fd, float(host(tb.grad)[7]), rel_tol=1e-5)
    fd = (L(p.A, p.b[:, 0], p.nu, p.lam + e) - L(p.A, p.b[:, 0], p.nu, p.lam - e)) / (2 * h)
    assert math.isclose(fd, float(host(tlam.grad)[7]), rel_tol=1e-4)
    hn = 1e-3 * p.nu
    fd = (L(p.A, p.b[:, 0], p.nu + hn, p.lam) - L(p.A, p.b[:, 0], p.nu - hn, p.lam)) / (2 * hn)
    assert math.isclose(fd, float(tnu.grad), rel_tol=1e-4)


def test_adjoint_requires_a_solved_workspace():
    p = synthetic.make_problem("C1", 0, n=512, d=32)
    solver = api().Solver(dev(p.A), dev(p.b), p.nu, dev(p.lam), kind="srht")
    from paper_2104_14101_gb300._lib import SksError
    with pytest.raises(SksError):
        solver.adjoint(dev(np.zeros(32)), dev(np.ones(32)))


# ----------------------------------------------------------------------------- failure path

def test_bounded_wait_reports_timeout_and_context_survives():
    # a device wait that can never complete gives up after 20 ms with
    # SKS_ERR_TIMEOUT; the next call on the same context works
    from paper_2104_14101_gb300 import _lib
    lib = _lib.load()
    stream = api().api._stream()
    assert lib.sks_selftest_wait_timeout(20_000_000, stream) == _lib.ERR_TIMEOUT
    assert b"site 99" in lib.sks_last_error()
    assert lib.sks_selftest_wait_timeout(10, stream) == _lib.ERR_INVALID_ARG
    rng = np.random.default_rng(3)
    A = rng.standard_normal((300, 20))
    x = rng.standard_normal(20)
    got = host(api().hess_apply(dev(A), dev(x), 0.5, dev(np.ones(20))))
    assert np.allclose(got, O.hess_apply(A, 0.5, np.ones(20), x), rtol=1e-12)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_hess_apply_widest_rows(dtype):
    # the largest supported d of each precision
    d = 16384 if dtype == "f32" else 14336
    rng = np.random.default_rng(d)
    A = rng.standard_normal((129, d)).astype(np.float32).astype(np.float64)
    x = rng.standard_normal(d)
    lam = 1 + rng.random(d)
    ref = O.hess_apply(A, 0.3, lam, x)
    got = host(api().hess_apply(dev(A, torch.float32 if dtype == "f32" else torch.float64), dev(x), 0.3, dev(lam)))
    tol = 1e-5 if dtype == "f32" else 1e-12
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < tol


@pytest.mark.parametrize("precision", ["plain", "mixed"])
def test_adaptive_solve_wide_d(precision):
    # d = 5000 > 4096 (the paper's experiments use d = 7000 and 14000): the
    # wide A-pass, a 5000 x 5000 factorisation, SRHT
    p = synthetic.make_problem("C3" if precision == "mixed" else "C2", 3, n=12000, d=5000, nu=1e-3,
                               decay="geom0.995")
    xs = O.direct_solve(p.A, p.b, p.nu, p.lam)
    A = dev(p.A, torch.float32) if precision == "mixed" else dev(p.A)
    tol = 1e-8 if precision == "mixed" else 1e-10
    x, st, _ = api().adaptive_pcg(A, dev(p.b), p.nu, dev(p.lam), kind="srht", m_init=64, tol=tol,
                                  precision=precision, seed=4, max_iter=2000)
    assert O.rel_err_H(p.A, p.nu, p.lam, host(x), xs) <= tol, st
