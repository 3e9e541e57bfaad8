"""GB300 (sm_103a) adaptive sketching-based solvers for
min 1/2 <x, H x> - b^T x, H = A^T A + nu^2 Lambda (Lacotte & Pilanci,
arXiv 2104.14101): SRHT / Gaussian / SJLT sketches, the sketched-Hessian
preconditioner, and adaptive PCG (Algorithm 2) / adaptive IHS (Algorithm 1),
all in hand-written CUDA behind the C ABI of include/sks.h.
"""
from . import _lib  # noqa: F401
from .api import (  # noqa: F401
    BatchSolver,
    DualSolver,
    Preconditioner,
    Sketch,
    SketchSolve,
    Solver,
    adaptive_ihs,
    adaptive_pcg,
    dual_solve,
    fixed_solve,
    hess_apply,
    make_problem,
    options,
    sketch_solve,
    solve_batched,
)
