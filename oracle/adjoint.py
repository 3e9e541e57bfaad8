"""Gradients of the solution map of problem (1) (oracle side, float64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For X = H^{-1} B (B is d x k, H = A^T A + nu^2 Lambda, eq. 1) and a scalar
loss L(X) with upstream gradient G = dL/dX, the implicit function theorem
applied to H X = B gives U = H^{-1} G (H is symmetric) and

    dL/dB      =  U
    dL/dH      = -U X^T
    dL/dA      = -A (U X^T + X U^T)          (H depends on A through A^T A)
    dL/dnu     = -2 nu sum_k u_k^T Lambda x_k
    dL/dLambda_ii = -nu^2 sum_k u_ik x_ik.

Pinned against central finite differences of L in the tests.
"""
import numpy as np

from .solvers import direct_solve


def solve_and_grads(A, B, nu, lam, G):
    """Returns X and the gradients (dB, dA, dnu, dlam) for upstream G."""
    X = direct_solve(A, B, nu, lam)
    U = direct_solve(A, G, nu, lam)
    X2 = X.reshape(X.shape[0], -1)
    U2 = U.reshape(U.shape[0], -1)
    dB = U
    dA = -(A @ U2) @ X2.T - (A @ X2) @ U2.T
    dnu = -2.0 * nu * float(np.sum(U2 * lam[:, None] * X2))
    dlam = -(nu ** 2) * np.sum(U2 * X2, axis=1)
    return X, dict(b=dB, A=dA, nu=dnu, lam=dlam)
