"""The chosen mixed-precision form (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's preconditioner only has to be spectrally close to H (the event
E_rho of Section 2.2 bounds ||C_S - I||), so the sketch and the sketched
Gram matrix may be formed in low precision while the accuracy of the final
iterate is restored by iterative refinement on the exact residual
b - A^T A x - nu^2 Lambda x.  This module defines, in float64 arithmetic on
exactly represented values, the pieces whose rounding decisions the GPU must
reproduce bit for bit:

* ``bf16_round``: float32 -> bfloat16 with round-to-nearest-even.
* ``split_hi_lo``: A = hi + lo + tail with hi = bf16(A), lo = bf16(A - hi)
  (A - hi is exact in float32), so hi + lo carries ~16 significant bits.
* ``gaussian_sketch_bf16``: the mixed form's Gaussian sketch by its plain
  definition, Y = bf16(G) A in float64 (the embedding's entries are the
  Gaussian draws of ``rng.gaussian_block`` rounded to float32, then to
  bfloat16; A enters exactly).  How a kernel represents A to reach that
  product is not part of the definition: its error is bounded in the tests.
* ``split_rowscaled``: a secondary check of the tensor-core Gram matrix's
  operand split (every row cut against its own maximum exponent into two
  slices of integers, 8 + 8 bits, so that all slice products are exactly
  summable); the Gram's parity test compares with the plain definition.
* ``e4m3_round`` and ``gaussian_sketch_e4m3``: the optional 8-bit sketch --
  the Gaussian entries rounded to float32, then to e4m3 (1 sign, 4 exponent
  bits with bias 7, 3 mantissa bits; largest finite 448; subnormals down to
  2^-9), times A quantised to e4m3 against one power-of-two scale per column
  and per slice of 16384 data rows, 2^ceil(log2(max|a| / 448)); each slice's
  product is multiplied back by its scales.
* ``refine``: the outer refinement loop around any inner solver.
"""
import numpy as np

from . import rng as R
from .solvers import hess_apply, h_norm_sq


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even); returns
    float64 holding the exact bfloat16 values."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def split_hi_lo(A32):
    """hi = bf16(A), lo = bf16(A - hi) for float32 A."""
    A32 = np.asarray(A32, dtype=np.float32)
    hi = bf16_round(A32)
    rem = (A32.astype(np.float64) - hi).astype(np.float32)  # exact
    lo = bf16_round(rem)
    return hi, lo


def split_rowscaled(X32):
    """Row-scaled two-slice split of a float32 matrix (float32 arithmetic).

    For each row with maximum |x| = f 2^e (f in [0.5, 1), so |x| < 2^e):
        hi = rint(x 2^(8-e)) 2^(e-8),  lo = rint((x - hi) 2^(16-e)) 2^(e-16)
    (rint = round half to even).  hi holds integers of magnitude <= 256 and lo
    integers <= 128 in their units, both exact in bfloat16, and
    |x - hi - lo| <= 2^(e-17).  Returns float64 arrays (hi, lo)."""
    X = np.asarray(X32, dtype=np.float32)
    mx = np.max(np.abs(X), axis=1)
    _, ex = np.frexp(mx)
    ex = ex.astype(np.int32)[:, None]
    hi = np.ldexp(np.rint(np.ldexp(X, 8 - ex)), ex - 8).astype(np.float32)
    hi[mx == 0] = 0
    lo = np.ldexp(np.rint(np.ldexp((X - hi).astype(np.float32), 16 - ex)), ex - 16).astype(np.float32)
    lo[mx == 0] = 0
    return hi.astype(np.float64), lo.astype(np.float64)


def gaussian_bf16(n_rows_data, m_rows, seed):
    """bf16(float32(G)) with G from ``rng.gaussian_block`` (the GPU forms the
    Box-Muller values in float32; values within one float32 ulp of a bfloat16
    rounding midpoint may round the other way there, which the parity test's
    tolerance absorbs)."""
    G = R.gaussian_block(n_rows_data, m_rows, seed)
    return bf16_round(G.astype(np.float32))


def gaussian_sketch_bf16(A32, m, seed, row0=0):
    """Rows [row0, m) of the unscaled Gaussian sketch of a float32 A by its
    definition, Y = bf16(G) A (S A = Y / sqrt(m)), in float64: G from
    ``rng.gaussian_block`` rounded to float32, then to bfloat16; the float32
    values of A enter exactly."""
    Gb = gaussian_bf16(A32.shape[0], m, seed)[row0:]
    return Gb @ np.asarray(A32, dtype=np.float32).astype(np.float64)


def bf16_midpoint_slack(g32, ulps=4):
    """For float32 values g32: the size of one bfloat16 step at each entry
    where a perturbation of up to `ulps` float32 ulps can change the
    bfloat16 rounding (a rounding midpoint lies within reach), else 0.  Two
    implementations of the same float32 formula that agree to `ulps` ulps
    round to bfloat16 identically everywhere the slack is 0."""
    g = np.asarray(g32, dtype=np.float32)
    step = np.spacing(np.abs(g)).astype(np.float32) * np.float32(ulps)
    lo = bf16_round((g - step).astype(np.float32))
    hi = bf16_round((g + step).astype(np.float32))
    here = bf16_round(g)
    amb = (lo != here) | (hi != here)
    ulp_bf16 = np.abs(here) * 2.0 ** -7 + 1e-45
    return np.where(amb, np.maximum(np.abs(hi - lo), ulp_bf16), 0.0)


def refine(A, b, nu, lam, inner, tol, max_outer=20):
    """Iterative refinement: x <- x + inner(r) with r = b - H x formed from A in
    float64, until ||r||_{H^{-1}} estimate via the inner solve is below tol
    relative to ||x||_H.  ``inner(r)`` returns an approximate H^{-1} r.
    Returns (x, outer iterations)."""
    x = np.zeros_like(b, dtype=np.float64)
    for it in range(1, max_outer + 1):
        r = b - hess_apply(A, nu, lam, x)
        dx = inner(r)
        x = x + dx
        if h_norm_sq(A, nu, lam, dx) <= (tol / 2.0) ** 2 * max(h_norm_sq(A, nu, lam, x), 1e-300):
            return x, it
    return x, max_outer


E4M3_MAX = 448.0


def e4m3_round(x):
    """Round float32 values to the nearest e4m3 value (ties to even), as
    float64: normal values keep 3 fraction bits (spacing 2^(e-3) for |x| in
    [2^e, 2^(e+1)), e >= -6), subnormals are multiples of 2^-9 below 2^-6,
    magnitudes past 448 saturate to 448 (finite saturation)."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    a = np.abs(x)
    _, e = np.frexp(a)               # a = f 2^e, f in [0.5, 1): the binade is [2^(e-1), 2^e)
    e = np.maximum(e - 1, -6)         # exponent of the binade, clamped into the subnormal range
    step = np.ldexp(1.0, e - 3)
    q = np.rint(a / step) * step      # rint: round half to even on the exact quotient
    q = np.minimum(q, E4M3_MAX)
    return np.sign(x) * q


def e4m3_scales(A32, slice_rows=16384):
    """Per-(slice, column) power-of-two scales 2^e, e the least integer with
    max|a| <= 448 2^e, i.e. 2^ceil(log2(max|a| / 448)) (1 for an all-zero
    block).  Computed exactly: with max|a| = f 2^E (f in [0.5, 1)) and
    448 = 0.875 2^9, e = E - 9, plus 1 when f > 0.875."""
    A = np.asarray(A32, dtype=np.float32).astype(np.float64)
    n, d = A.shape
    ns = max(1, (n + slice_rows - 1) // slice_rows)
    sc = np.ones((ns, d))
    for k in range(ns):
        mx = np.max(np.abs(A[k * slice_rows:(k + 1) * slice_rows]), axis=0) if n else np.zeros(d)
        nz = mx > 0
        f, E = np.frexp(mx[nz])
        sc[k, nz] = np.ldexp(1.0, E - 9 + (f > 0.875))
    return sc


def gaussian_sketch_e4m3(A32, m, seed, row0=0, slice_rows=16384):
    """Rows [row0, m) of the unscaled 8-bit Gaussian sketch (S A = Y / sqrt(m)):
    Y = sum over slices k of e4m3(G_k) e4m3(A_k / s_k) diag(s_k), with G from
    ``rng.gaussian_block`` rounded to float32, then to e4m3, and s_k the
    slice's column scales (``e4m3_scales``), all in float64."""
    A = np.asarray(A32, dtype=np.float32)
    n, d = A.shape
    G8 = e4m3_round(R.gaussian_block(n, m, seed).astype(np.float32))[row0:]
    sc = e4m3_scales(A, slice_rows)
    Y = np.zeros((G8.shape[0], d))
    for k in range(sc.shape[0]):
        blk = A[k * slice_rows:(k + 1) * slice_rows].astype(np.float64) / sc[k][None, :]
        A8 = e4m3_round(blk.astype(np.float32))
        Y += (G8[:, k * slice_rows:(k + 1) * slice_rows] @ A8) * sc[k][None, :]
    return Y


def e4m3_midpoint_slack(g32, ulps=4):
    """As ``bf16_midpoint_slack`` for the e4m3 rounding: one e4m3 step where a
    perturbation of up to `ulps` float32 ulps can change the rounding, else 0."""
    g = np.asarray(g32, dtype=np.float32)
    step = np.spacing(np.abs(g)).astype(np.float32) * np.float32(ulps)
    lo = e4m3_round((g - step).astype(np.float32))
    hi = e4m3_round((g + step).astype(np.float32))
    here = e4m3_round(g)
    amb = (lo != here) | (hi != here)
    return np.where(amb, np.maximum(np.abs(hi - lo), 2.0 ** -9), 0.0)
