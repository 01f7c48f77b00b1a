"""FP64 Krylov references on the sparse 7-point operator.

Used where dense cyclic reduction does not fit (n >= 64): the relative
residual ``||f - A u|| / ||f||`` of Section 5 (Poisson experiments) is exactly
computable at any size, and a CG (SPD) or GMRES (indefinite) solve to a tight
tolerance is the reference solution.  Plain textbook CG (Hestenes-Stiefel)
without preconditioning, written out; GMRES from SciPy.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import operator as op


def rel_residual(n: int, log_kappa, u: np.ndarray, f: np.ndarray, shift: float = 0.0) -> np.ndarray:
    """Per-column ``||f - A u||_2 / ||f||_2``."""
    r = f - op.apply(n, log_kappa, u, shift)
    if r.ndim == 1:
        return np.array([np.linalg.norm(r) / np.linalg.norm(f)])
    return np.linalg.norm(r, axis=0) / np.linalg.norm(f, axis=0)


def cg(A, f: np.ndarray, rtol: float = 1e-12, maxiter: int = 20000):
    """Conjugate gradients for SPD ``A`` (sparse matrix or LinearOperator); returns ``(u, iters)``."""
    u = np.zeros_like(f)
    r = f.copy()
    p = r.copy()
    rr = r @ r
    stop = (rtol * np.linalg.norm(f)) ** 2
    for it in range(1, maxiter + 1):
        Ap = A @ p
        alpha = rr / (p @ Ap)
        u += alpha * p
        r -= alpha * Ap
        rr_new = r @ r
        if rr_new <= stop:
            return u, it
        p = r + (rr_new / rr) * p
        rr = rr_new
    return u, maxiter


def gmres(A, f: np.ndarray, rtol: float = 1e-12, restart: int = 100, maxiter: int = 2000):
    u, info = spla.gmres(A, f, rtol=rtol, restart=restart, maxiter=maxiter)
    return u, info


def reference_solve(n: int, log_kappa, f: np.ndarray, shift: float = 0.0, rtol: float = 1e-12):
    """Tight FP64 reference solution, one column at a time: CG if ``shift >= 0`` else GMRES."""
    A = op.assemble(n, log_kappa, shift)
    cols = f[:, None] if f.ndim == 1 else f
    out = np.empty_like(cols)
    for c in range(cols.shape[1]):
        if shift >= 0.0:
            out[:, c], _ = cg(A, np.ascontiguousarray(cols[:, c]), rtol=rtol)
        else:
            out[:, c], _ = gmres(A, np.ascontiguousarray(cols[:, c]), rtol=rtol)
    return out[:, 0] if f.ndim == 1 else out
