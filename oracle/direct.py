"""Exact solutions: dense LU and the discrete-sine-transform closed form.

``dense_solve`` is the plain definition ``u = A^{-1} f`` by LAPACK LU (small
grids only, ``N <= ~5000``).  ``dst_solve`` is the closed form for constant
kappa: the 7-point Laplacian is diagonalised by the orthonormal 1D DST-I on
every axis, the Fourier route that FACR combines with cyclic reduction
(Section 1).  With ``S_ab = sqrt(2/(n+1)) sin(pi (a+1)(b+1)/(n+1))`` (symmetric,
orthogonal) and ``lambda_a = (4/h^2) sin^2(pi (a+1) h / 2)``,
``u = (S x S x S) diag(1/(lam_i + lam_j + lam_k + shift)) (S x S x S) f``.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import operator as op


def dense_solve(n: int, log_kappa, f: np.ndarray, shift: float = 0.0) -> np.ndarray:
    A = op.assemble(n, log_kappa, shift).toarray()
    return sla.solve(A, f)


def dst_matrix(n: int) -> np.ndarray:
    a = np.arange(1, n + 1, dtype=np.float64)
    return np.sqrt(2.0 / (n + 1)) * np.sin(np.pi * np.outer(a, a) / (n + 1))


def laplacian_eigs_1d(n: int) -> np.ndarray:
    h = 1.0 / (n + 1)
    return (4.0 / h ** 2) * np.sin(np.pi * np.arange(1, n + 1) * h / 2.0) ** 2


def dst_solve(n: int, f: np.ndarray, shift: float = 0.0) -> np.ndarray:
    """Constant-coefficient solve of ``(-Delta_h + shift) u = f``; ``f`` is ``(N,)`` or ``(N, r)``."""
    S = dst_matrix(n)
    lam = laplacian_eigs_1d(n)
    squeeze = f.ndim == 1
    F = f.reshape(n, n, n, -1)  # [k][j][i][r]
    fh = np.einsum("ak,bj,ci,kjir->abcr", S, S, S, F, optimize=True)
    denom = lam[:, None, None] + lam[None, :, None] + lam[None, None, :] + shift
    uh = fh / denom[..., None]
    u = np.einsum("ak,bj,ci,abcr->kjir", S, S, S, uh, optimize=True).reshape(n ** 3, -1)
    return u[:, 0] if squeeze else u
