"""7-point operator of the model problem (Section 2.2.1, Eq. probSta, Eq. originalMatrix).

The paper fixes only "-div(kappa grad u) = f, 7-point finite differences,
Dirichlet, unit cube" and the block-tridiagonal shape ``tridiag(E_i, D_i, F_i)``
with ``n`` blocks of size ``n^2``.  Where it is silent this module takes these
readings:

* vertex-centred grid, ``n`` interior nodes per axis, ``h = 1/(n+1)``;
* ``kappa_p = exp(g_p)`` is attached to node ``p`` (its control volume);
* interior face ``pq``: ``c_pq = 2 kappa_p kappa_q / (kappa_p + kappa_q) / h^2``
  (harmonic mean);
* boundary face of ``p`` (neighbour outside the cube, ``u = 0`` there):
  ``c = kappa_p / h^2``;
* ``(A u)_p = sum_faces c (u_p - u_q) + shift * u_p`` with ``u_q = 0`` outside.

With ``kappa = 1`` and ``shift = 0`` this is the textbook ``-Delta_h``.  The
Helmholtz workload uses ``shift = -omega^2``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def kappa_from_log(n: int, log_kappa) -> np.ndarray:
    """Node coefficients ``kappa = exp(g)`` shaped ``[k][j][i]``; ``None`` means kappa = 1."""
    if log_kappa is None:
        return np.ones((n, n, n))
    g = np.asarray(log_kappa, dtype=np.float64).reshape(n, n, n)
    return np.exp(g)


def _harmonic(a, b, h):
    return 2.0 * a * b / (a + b) / (h * h)


def face_coefficients(n: int, log_kappa=None):
    """Return ``(cx, cy, cz, bsum)``.

    ``cx[k,j,i]`` couples node ``(i,j,k)`` with ``(i+1,j,k)`` (``i < n-1``), and
    likewise ``cy`` (``j``) and ``cz`` (``k``).  ``bsum[k,j,i]`` is the sum of
    the boundary-face coefficients of the node.
    """
    h = 1.0 / (n + 1)
    kap = kappa_from_log(n, log_kappa)
    cx = _harmonic(kap[:, :, :-1], kap[:, :, 1:], h)
    cy = _harmonic(kap[:, :-1, :], kap[:, 1:, :], h)
    cz = _harmonic(kap[:-1, :, :], kap[1:, :, :], h)
    nb = np.zeros((n, n, n))
    for ax in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = 0
        hi[ax] = n - 1
        nb[tuple(lo)] += 1.0
        nb[tuple(hi)] += 1.0
    bsum = nb * kap / (h * h)
    return cx, cy, cz, bsum


def assemble(n: int, log_kappa=None, shift: float = 0.0) -> sp.csr_matrix:
    """Sparse ``N x N`` matrix ``A`` (``N = n^3``), lexicographic ``i + n j + n^2 k``."""
    cx, cy, cz, bsum = face_coefficients(n, log_kappa)
    idx = np.arange(n ** 3).reshape(n, n, n)
    diag = bsum.copy() + shift
    diag[:, :, :-1] += cx
    diag[:, :, 1:] += cx
    diag[:, :-1, :] += cy
    diag[:, 1:, :] += cy
    diag[:-1, :, :] += cz
    diag[1:, :, :] += cz
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [diag.ravel()]
    for c, a, b in (
        (cx, idx[:, :, :-1], idx[:, :, 1:]),
        (cy, idx[:, :-1, :], idx[:, 1:, :]),
        (cz, idx[:-1, :, :], idx[1:, :, :]),
    ):
        rows += [a.ravel(), b.ravel()]
        cols += [b.ravel(), a.ravel()]
        vals += [-c.ravel(), -c.ravel()]
    N = n ** 3
    A = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)
    )
    return A.tocsr()


def plane_blocks(n: int, log_kappa=None, shift: float = 0.0):
    """Dense plane blocks ``(D, E, F)`` of Eq. originalMatrix.

    ``D[k]`` is the ``n^2 x n^2`` in-plane block of plane ``k``; ``E[k]``
    couples plane ``k`` to ``k-1`` (sub-diagonal, ``E[0] = None``); ``F[k]``
    couples plane ``k`` to ``k+1`` (super-diagonal, ``F[n-1] = None``).
    In-plane order is lexicographic ``i + n j``.
    """
    A = assemble(n, log_kappa, shift).tocsr()
    m = n * n
    D, E, F = [], [], []
    for k in range(n):
        r = slice(k * m, (k + 1) * m)
        D.append(A[r, r].toarray())
        E.append(A[r, (k - 1) * m:k * m].toarray() if k > 0 else None)
        F.append(A[r, (k + 1) * m:(k + 2) * m].toarray() if k < n - 1 else None)
    return D, E, F


def apply(n: int, log_kappa, u: np.ndarray, shift: float = 0.0) -> np.ndarray:
    """Matrix-free ``A u`` for ``u`` of shape ``(N,)`` or ``(N, nrhs)``."""
    cx, cy, cz, bsum = face_coefficients(n, log_kappa)
    squeeze = u.ndim == 1
    U = u.reshape(n, n, n, -1)
    out = (bsum + shift)[..., None] * U
    for c, ax in ((cx, 2), (cy, 1), (cz, 0)):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, n - 1)
        hi[ax] = slice(1, n)
        lo, hi = tuple(lo), tuple(hi)
        d = U[lo] - U[hi]
        out[lo] += c[..., None] * d
        out[hi] -= c[..., None] * d
    out = out.reshape(n ** 3, -1)
    return out[:, 0] if squeeze else out
