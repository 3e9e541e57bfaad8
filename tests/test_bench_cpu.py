"""The benchmark's workload table and generators, on CPU (no GPU): every
workload names a known configuration, its generator runs at a reduced size,
and the oracle legs it would time accept the generated problem."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synthetic  # noqa: E402


@pytest.mark.parametrize("name", sorted(bench.WORKLOADS))
def test_workload_generators_run_on_cpu(name):
    wl = dict(bench.WORKLOADS[name])
    assert wl["config"] in synthetic.CONFIGS
    assert wl["method"] in ("pcg", "ihs") and wl["kind"] in ("srht", "gaussian", "sjlt", "rademacher", "gaussian-e4m3")
    if wl.get("batched"):
        specs = synthetic.batched_specs(8, seed=0)
        assert all(s["n"] >= 4 * s["d"] for s in specs)
        return
    small = dict(wl, n=64 if wl.get("dual") else 512, d=200 if wl.get("dual") else 32)
    prob = bench.make_workload_problem(small, "cpu")
    A = prob["A64"]
    n, d = A.shape
    assert (n, d) == (small["n"], small["d"])
    if wl.get("dual"):
        assert n < d
    b = prob["b"][:, 0].numpy()
    x, st, _ = bench.oracle_solve(dict(wl, m_max=0), A.numpy(), b, prob["nu"], prob["lam"].numpy())
    from oracle import solvers as O
    xs = O.direct_solve(A.numpy(), b, prob["nu"], prob["lam"].numpy())
    assert O.rel_err_H(A.numpy(), prob["nu"], prob["lam"].numpy(), x, xs) <= max(10 * wl["tol"], 1e-7)


def test_sketch_phase_roofline_arithmetic():
    st = dict(ms_sketch=126.0, sketch_passes=14)
    r = bench.sketch_phase_roofline("sjlt", st, 1 << 20, 4096, 4, 6794.5)
    assert r["passes"] == 14 and r["bytes_per_pass"] == (1 << 20) * 4096 * 4
    assert abs(r["achieved"] - 14 * (1 << 20) * 4096 * 4 / 0.126 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / 6794.5) < 1e-12
    assert bench.sketch_phase_roofline("srht", st, 1, 1, 4, 1.0) is None
    assert bench.sketch_phase_roofline("sjlt", dict(ms_sketch=0.0, sketch_passes=1), 1, 1, 4, 1.0) is None
