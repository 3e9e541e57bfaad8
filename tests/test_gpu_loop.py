"""The device-resident iteration (one cooperative launch per sketch size) with
several right-hand sides in lockstep: every column against the oracle's direct
solve, the passes over A shared by the columns, per-column traces consistent
with the test of Algorithm 1 / 2."""
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


@pytest.mark.parametrize("method", ["pcg", "ihs"])
@pytest.mark.parametrize("k", [2, 8, 11])
def test_lockstep_plain_matches_oracle(method, k):
    # k = 11 runs a batch of 8 and a batch of 3 (columns past 3 inert)
    p = synthetic.make_problem("C4", 1, n=4096, d=256, k=k, dtype="f64")
    xs = O.direct_solve(p.A, p.b, p.nu, p.lam)
    fn = api().adaptive_pcg if method == "pcg" else api().adaptive_ihs
    x, st, tr = fn(dev(p.A), dev(p.b), p.nu, dev(p.lam), kind="gaussian", tol=1e-10, seed=2, trace_cap=4096)
    assert st["status_name"] == "OK"
    for c in range(k):
        assert O.rel_err_H(p.A, p.nu, p.lam, host(x)[:, c], xs[:, c]) <= 1e-10, c
    # every column took part in the tests, and every verdict follows Algorithm 2 / 1
    cols = {e["column"] for e in tr}
    assert cols == set(range(k))
    m_max = p.n
    for e in tr:
        assert e["accepted"] == (e["ratio"] <= e["thr"] or e["m"] >= m_max)


@pytest.mark.parametrize("method", ["pcg", "ihs"])
@pytest.mark.parametrize("kind", ["gaussian", "sjlt"])
def test_lockstep_mixed_matches_oracle(method, kind):
    p = synthetic.make_problem("C4", 2, n=8192, d=256, k=8, dtype="f32")
    xs = O.direct_solve(p.A, p.b, p.nu, p.lam)
    fn = api().adaptive_pcg if method == "pcg" else api().adaptive_ihs
    x, st, _ = fn(dev(p.A, torch.float32), dev(p.b), p.nu, dev(p.lam), kind=kind, sjlt_s=2, tol=1e-8,
                  precision="mixed", seed=4)
    assert st["status_name"] == "OK"
    for c in range(8):
        assert O.rel_err_H(p.A, p.nu, p.lam, host(x)[:, c], xs[:, c]) <= 1e-8, c


def test_lockstep_shares_the_passes_over_A():
    # eight right-hand sides in lockstep make about as many passes as the
    # slowest single column, not the sum over the columns
    p = synthetic.make_problem("C4", 3, n=4096, d=256, k=8, dtype="f64")
    A, lam = dev(p.A), dev(p.lam)
    _, st8, _ = api().adaptive_pcg(A, dev(p.b), p.nu, lam, kind="srht", tol=1e-10, seed=1)
    single = []
    for c in range(8):
        _, s1, _ = api().adaptive_pcg(A, dev(np.ascontiguousarray(p.b[:, c])), p.nu, lam, kind="srht", tol=1e-10,
                                      seed=1)
        single.append(s1["a_passes"])
    assert st8["a_passes"] <= max(single) + 4
    assert st8["a_passes"] < sum(single) / 3


def test_lockstep_zero_and_nonzero_columns():
    # a zero right-hand side stops at once without holding the others back;
    # a warm start from the solution stops at the first test
    p = synthetic.make_problem("C4", 4, n=2048, d=128, k=3, dtype="f64")
    b = p.b.copy()
    b[:, 1] = 0.0
    xs = O.direct_solve(p.A, b, p.nu, p.lam)
    x0 = np.zeros_like(b)
    x0[:, 2] = xs[:, 2]
    x, st, _ = api().adaptive_pcg(dev(p.A), dev(b), p.nu, dev(p.lam), x0=dev(x0), kind="gaussian", tol=1e-10)
    assert np.all(host(x)[:, 1] == 0.0)
    for c in (0, 2):
        assert O.rel_err_H(p.A, p.nu, p.lam, host(x)[:, c], xs[:, c]) <= 1e-10


@pytest.mark.parametrize("method", ["pcg", "ihs", "fixed-pcg"])
def test_trace_delta_matches_oracle(method):
    # with x_star, every trace event carries delta_t = 1/2 ||x_t - x*||_H^2 of
    # the iterate kept after it; the device forms it as 1/2 (x* - x)^T r.
    # Fused loop (adaptive) and host-driven loop (fixed PCG) alike.
    p = synthetic.make_problem("C1", 1, n=1024, d=64, nu=1e-2)
    xs = O.direct_solve(p.A, p.b, p.nu, p.lam)
    kw = dict(kind="gaussian", m_init=1 if method != "fixed-pcg" else 128, tol=1e-10, seed=5, reuse_residual=False)
    solver = api().Solver(dev(p.A), dev(p.b), p.nu, dev(p.lam), method=method, trace_cap=4096, x_star=dev(xs), **kw)
    x, st, tr = solver.solve()
    d0 = 0.5 * O.h_norm_sq(p.A, p.nu, p.lam, xs)  # x_0 = 0
    assert len(tr) > 5
    for e in tr:
        assert np.isclose(e["delta0"], d0, rtol=1e-10)
    final = 0.5 * O.h_norm_sq(p.A, p.nu, p.lam, host(x) - xs)
    assert np.isclose(tr[-1]["delta"], final, rtol=1e-4, atol=1e-20 * d0)
    kept = [e["delta"] for e in tr]
    if method != "ihs":  # PCG minimises the H-norm error over a growing space: non-increasing
        assert all(b <= a * (1 + 1e-8) + 1e-22 * d0 for a, b in zip(kept, kept[1:]))
    if method == "pcg":
        # against the oracle's own iterates (same accept / reject sequence, literal restart)
        xo, so, to = O.adaptive_pcg(p.A, p.b, p.nu, p.lam, kind="gaussian", seed=5, m_init=1, tol=1e-10,
                                    literal_restart=True, record_states=True)
        xs_o = [e["x"] for e in to[1:]] + [xo]  # the iterate kept after each event
        for eo, eg, xk in zip(to, tr, xs_o):
            if abs(eo["ratio"] / eo["thr"] - 1) < 1e-9:
                break
            assert eo["accepted"] == eg["accepted"]
            do = 0.5 * O.h_norm_sq(p.A, p.nu, p.lam, xk - xs)
            if do > 1e-16 * d0:
                assert np.isclose(eg["delta"], do, rtol=1e-5), (eo["t"], eg["delta"], do)
