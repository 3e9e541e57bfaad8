"""CPU FP64 oracle for the adaptive sketching-based solvers of Lacotte & Pilanci,
"Fast Convex Quadratic Optimization Solvers with Adaptive Sketching-based
Preconditioners" (arXiv 2104.14101).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The GPU product path
(``paper_2104_14101_gb300``) never imports, links or executes anything here,
and this package never imports the GPU path: the two share no code.  The only
module both sides use is the seeded input generator package ``synthetic``,
which holds none of the method's arithmetic.

Everything here is plain NumPy / SciPy in float64, written to be checked by
eye against the paper:

* ``rng``      -- Philox4x32-10 counter-based generator (Salmon et al., SC'11)
                  and the keyed draws every sketch takes from it (signs,
                  Gaussian variates, the Feistel row permutation, SJLT hashes).
* ``sketch``   -- the three embeddings of Section 2.1: SRHT, Gaussian, SJLT.
* ``solvers``  -- problem (1), the direct Cholesky solve, the sketched
                  preconditioner of Section 4.1.1 (Cholesky and Woodbury
                  forms), IHS (eq. 4), PCG (eq. 5), Algorithm 1 with the IHS,
                  Algorithm 2, the effective dimension, the critical sketch
                  sizes of Theorems 5.1 / 5.2 and the Polyak-IHS bound of
                  Corollary A.2 / Table 3.
* ``mixed``    -- the chosen mixed-precision form: BF16 rounding and the
                  hi/lo split, FP64 iterative refinement around an inner
                  adaptive PCG.
* ``adjoint``  -- gradients of x*(A, b, nu, Lambda) (implicit function
                  theorem applied to problem (1)).

Parity status of every function is stated in its docstring; functions whose
value is not pinned to anything but themselves say "parity unpinned".
"""
