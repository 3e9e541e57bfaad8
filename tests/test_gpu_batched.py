"""GPU parity of the batched solve (many uneven problems, one captured round
replayed): every problem against the oracle's direct solve and against the
single-problem adaptive PCG of the same options."""
import numpy as np
import pytest

import synthetic
from oracle import solvers as O
from tests.gpu_util import dev, host, require_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def api():
    import paper_2104_14101_gb300 as sks
    return sks


# (n, d, nu, decay, config for Lambda): d = 1, tails of 32 / 64, one
# d = 1024 problem (32 columns per lane, 16 Cholesky panels), n not a power of 2
SHAPES = [
    (300, 1, 1e-2, "geom0.9", "C1"),
    (1000, 33, 1e-3, "harmonic", "C2"),
    (2500, 64, 1e-1, "geom0.9", "C1"),
    (777, 65, 1e-4, "harmonic", "C1"),
    (4096, 130, 3e-3, "geom0.9", "C2"),
    (5000, 200, 1e-4, "harmonic", "C1"),
    (2049, 257, 2e-2, "harmonic", "C2"),
    (9000, 1024, 1e-3, "geom0.9", "C1"),
]


def batch_problems(shapes, seed0=0):
    out = []
    for i, (n, d, nu, decay, cfg) in enumerate(shapes):
        p = synthetic.make_problem(cfg, seed0 + i, n=n, d=d, nu=nu, decay=decay)
        out.append(p)
    return out


def to_dev(probs):
    return [(dev(p.A), dev(p.b), p.nu, dev(p.lam)) for p in probs]


def test_batched_matches_oracle_and_single_solves():
    probs = batch_problems(SHAPES)
    tol = 1e-8
    xs, stats, info = api().solve_batched(to_dev(probs), tol=tol, max_iter=500)
    assert info["rounds"] > 0 and info["rows_per_unit"] in (32, 64, 128, 256, 512)
    for p, x, st in zip(probs, xs, stats):
        assert st["status"] == 0, st
        xs_ref = O.direct_solve(p.A, p.b, p.nu, p.lam)
        err = O.rel_err_H(p.A, p.nu, p.lam, host(x), xs_ref)
        assert err <= tol, (p.A.shape, err, st)
        # the same Algorithm 2 run one problem at a time
        x1, st1, _ = api().adaptive_pcg(dev(p.A), dev(p.b), p.nu, dev(p.lam), kind="srht", tol=tol, max_iter=500)
        assert (st["final_m"], st["iters"], st["rejections"]) == (st1["final_m"], st1["iters"], st1["rejections"])
        assert O.rel_err_H(p.A, p.nu, p.lam, host(x), host(x1)) <= 1e-9


def test_batched_unit_height_does_not_change_the_result():
    probs = batch_problems(SHAPES[:5], seed0=10)
    res = []
    for rows in (32, 512):
        xs, stats, info = api().solve_batched(to_dev(probs), rows_per_unit=rows, tol=1e-8)
        assert info["rows_per_unit"] == rows
        res.append((xs, stats))
    for p, xa, xb, sa, sb in zip(probs, res[0][0], res[1][0], res[0][1], res[1][1]):
        assert sa["final_m"] == sb["final_m"] and sa["iters"] == sb["iters"]
        assert O.rel_err_H(p.A, p.nu, p.lam, host(xa), host(xb)) <= 1e-11


def test_batched_edge_cases_zero_rhs_and_warm_start():
    probs = batch_problems(SHAPES[1:4], seed0=20)
    items = to_dev(probs)
    # problem 0: b = 0 (the solution is 0: stops at the first restart)
    items[0] = (items[0][0], torch.zeros_like(items[0][1]), items[0][2], items[0][3])
    # problem 2: warm start at the solution plus a small perturbation
    x_star = O.direct_solve(probs[2].A, probs[2].b, probs[2].nu, probs[2].lam)
    x0s = [torch.zeros(p.A.shape[1], dtype=torch.float64, device="cuda") for p in probs]
    x0s[2] = dev(x_star * (1 + 1e-6))
    xs, stats, _ = api().solve_batched(items, x0s=x0s, tol=1e-8)
    assert np.all(host(xs[0]) == 0.0) and stats[0]["iters"] == 0 and stats[0]["status"] == 0
    for i in (1, 2):
        p = probs[i]
        ref = O.direct_solve(p.A, p.b, p.nu, p.lam)
        assert O.rel_err_H(p.A, p.nu, p.lam, host(xs[i]), ref) <= 1e-8
    assert stats[2]["iters"] <= stats[1]["iters"]


def test_batched_reports_per_problem_no_convergence():
    # m fixed at 1 (m_max = 1) and at most 2 accepted steps: the d = 1 problem
    # is solved exactly in one step, the d = 65 problem cannot be.
    probs = batch_problems([SHAPES[0], SHAPES[3]], seed0=30)
    solver = api().BatchSolver(to_dev(probs), m_max=1, max_iter=2, tol=1e-8)
    xs, stats, _ = solver.solve(check=False)
    assert stats[0]["status"] == 0 and stats[0]["final_m"] == 1
    assert stats[1]["status_name"] == "NO_CONVERGENCE" and stats[1]["iters"] == 2 and stats[1]["final_m"] == 1
    with pytest.raises(api()._lib.SksError, match="batch problem 1"):
        solver.solve()


def test_batched_solver_is_reusable():
    probs = batch_problems(SHAPES[:3], seed0=40)
    solver = api().BatchSolver(to_dev(probs), tol=1e-8)
    xa, sa, _ = solver.solve()
    xb, sb, _ = solver.solve()
    for a, b in zip(xa, xb):
        assert torch.equal(a, b)
    assert [s["iters"] for s in sa] == [s["iters"] for s in sb]


# ---- mixed form (float32 A, iterative refinement around Algorithm 2)

def to_dev32(probs):
    return [(dev(p.A.astype(np.float32)), dev(p.b), p.nu, dev(p.lam)) for p in probs]


def up32(p):
    """The problem the mixed form solves: A rounded to float32, upcast exactly."""
    return p.A.astype(np.float32).astype(np.float64)


def test_batched_mixed_matches_oracle():
    probs = batch_problems(SHAPES, seed0=50)
    tol = 1e-8
    xs, stats, info = api().solve_batched(to_dev32(probs), precision="mixed", tol=tol, max_iter=2000)
    assert info["rounds"] > 0
    for p, x, st in zip(probs, xs, stats):
        assert st["status"] == 0, st
        A = up32(p)
        ref = O.direct_solve(A, p.b, p.nu, p.lam)
        err = O.rel_err_H(A, p.nu, p.lam, host(x), ref)
        assert err <= tol, (p.A.shape, p.nu, err, st)
        assert st["outer_iters"] >= 1 and st["final_m"] >= 1
        # the estimate the stop rule used is the decrement at the returned x
        assert st["est_rel_err"] <= tol


def test_batched_mixed_edge_cases_and_reuse():
    probs = batch_problems(SHAPES[1:4], seed0=60)
    items = to_dev32(probs)
    items[0] = (items[0][0], torch.zeros_like(items[0][1]), items[0][2], items[0][3])
    solver = api().BatchSolver(items, precision="mixed", tol=1e-8)
    xa, sa, _ = solver.solve()
    xb, sb, _ = solver.solve()
    assert np.all(host(xa[0]) == 0.0) and sa[0]["iters"] == 0 and sa[0]["status"] == 0
    for a, b in zip(xa, xb):
        assert torch.equal(a, b)
    for i in (1, 2):
        p = probs[i]
        A = up32(p)
        assert O.rel_err_H(A, p.nu, p.lam, host(xa[i]), O.direct_solve(A, p.b, p.nu, p.lam)) <= 1e-8
    # a warm start near the solution: converged, and no more work than from 0
    x0s = [torch.zeros(p.A.shape[1], dtype=torch.float64, device="cuda") for p in probs]
    A2 = up32(probs[2])
    ref2 = O.direct_solve(A2, probs[2].b, probs[2].nu, probs[2].lam)
    x0s[2] = dev(ref2 * (1 + 1e-6))
    xw, sw, _ = solver.solve(x0s=x0s)
    assert sw[2]["status"] == 0 and sw[2]["iters"] <= sa[2]["iters"]
    assert O.rel_err_H(A2, probs[2].nu, probs[2].lam, host(xw[2]), ref2) <= 1e-8


def test_batched_mixed_reports_no_convergence_after_max_outer():
    # one refinement step with a loose inner solve cannot reach 1e-10
    probs = batch_problems([SHAPES[3], SHAPES[5]], seed0=70)
    solver = api().BatchSolver(to_dev32(probs), precision="mixed", tol=1e-10, max_outer=1, inner_tol=0.5)
    xs, stats, _ = solver.solve(check=False)
    for st in stats:
        assert st["status_name"] == "NO_CONVERGENCE" and st["outer_iters"] == 1


def test_batched_precision_must_match_the_dtype_of_A():
    probs = batch_problems(SHAPES[:2], seed0=80)
    with pytest.raises(api()._lib.SksError, match="mixed form needs float32 A"):
        api().BatchSolver(to_dev(probs), precision="mixed")
    with pytest.raises(api()._lib.SksError, match="plain form needs float64 A"):
        api().BatchSolver(to_dev32(probs), precision="plain")
