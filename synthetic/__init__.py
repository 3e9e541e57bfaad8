"""Seeded synthetic problem generators for problem (1) of Lacotte & Pilanci
(arXiv 2104.14101): min 1/2 <x, H x> - b^T x with H = A^T A + nu^2 Lambda.

This package builds inputs only: matrices with a controlled singular-value
decay A = U diag(sigma) V^T (the synthetic workloads of Section 6), right-hand
sides and regularisation.  It holds none of the solvers' arithmetic, so both
the CPU oracle (``oracle/``) and the GPU path's tests and benchmark may use it.
"""
from .problems import (  # noqa: F401
    CONFIGS,
    Problem,
    make_problem,
    make_problem_torch,
    make_wide_problem_torch,
    spectrum,
    batched_specs,
    make_batch_torch,
)
