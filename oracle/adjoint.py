"""Dense adjoint of the loss L = ||u - u_obs||^2, A(kappa) u = f (Section 2.2.1 operator).

TEST INFRASTRUCTURE ONLY.  The paper has no adjoint; this is the plain
derivation for the operator of ``oracle.operator``:

    lambda = A^{-T} 2 (u - u_obs),   dL/df = lambda,
    dL/dkappa_p = - lambda^T (dA/dkappa_p) u
                = - sum_{interior faces pq} dc_pq/dkappa_p (lambda_p - lambda_q)(u_p - u_q)
                  - (#boundary faces of p) lambda_p u_p / h^2,
    dc_pq/dkappa_p = 2 kappa_q^2 / ((kappa_p + kappa_q)^2 h^2),
    dL/dg_p = kappa_p dL/dkappa_p   (kappa = exp(g)).

Solves are dense LU (small grids).  Pinned against central finite differences
of dense solves in tests/test_oracle_adjoint.py.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import operator as op


def loss(n, g, f, u_obs, shift=0.0):
    A = op.assemble(n, g, shift).toarray()
    u = sla.solve(A, f)
    return float(np.sum((u - u_obs) ** 2)), u


def grad_from_fields(n, g, u, lam):
    """dL/dg from the state u and adjoint lam (either (N,) or (N, r), summed over columns)."""
    h = 1.0 / (n + 1)
    kap = op.kappa_from_log(n, g)
    U = u.reshape(n, n, n, -1)
    Lm = lam.reshape(n, n, n, -1)
    dk = np.zeros((n, n, n))
    for ax in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, n - 1)
        hi[ax] = slice(1, n)
        lo, hi = tuple(lo), tuple(hi)
        kp, kq = kap[lo], kap[hi]
        term = np.sum((Lm[lo] - Lm[hi]) * (U[lo] - U[hi]), axis=-1)
        dcp = 2.0 * kq ** 2 / ((kp + kq) ** 2 * h * h)
        dcq = 2.0 * kp ** 2 / ((kp + kq) ** 2 * h * h)
        dk[lo] -= dcp * term
        dk[hi] -= dcq * term
        # boundary faces on both ends of this axis
        first = [slice(None)] * 3
        last = [slice(None)] * 3
        first[ax] = 0
        last[ax] = n - 1
        for sl in (tuple(first), tuple(last)):
            dk[sl] -= np.sum(Lm[sl] * U[sl], axis=-1) / (h * h)
    return (kap * dk).reshape(-1)


def loss_and_grad(n, g, f, u_obs, shift=0.0):
    """Returns (L, dL/dg, dL/df) by dense solves."""
    A = op.assemble(n, g, shift).toarray()
    u = sla.solve(A, f)
    lam = sla.solve(A.T, 2.0 * (u - u_obs))
    return float(np.sum((u - u_obs) ** 2)), grad_from_fields(n, g, u, lam), lam
