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

Convection-diffusion (Section 5, Eq. codi): ``-Delta u + alpha b . grad u``
"discretized with a 7-point upwind finite difference scheme".  With the node
velocity ``beta = alpha b(x_p)`` (array ``velocity`` of shape ``(3, N)``), each
component's derivative is differenced toward the upstream neighbour:
``beta_d > 0``: ``beta_d (u_p - u_{p-e_d}) / h``; ``beta_d < 0``:
``beta_d (u_{p+e_d} - u_p) / h``.  So the diagonal gains ``|beta_d| / h`` and
the upstream neighbour ``-|beta_d| / h``; a neighbour outside the cube carries
the Dirichlet value (zero here; the manufactured problem moves it to the
right-hand side).  The result is a non-symmetric M-matrix.
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


def upwind_weights(n: int, velocity):
    """``(dplus, wminus, wplus)`` of the convection term: ``dplus[k,j,i]`` is the
    diagonal gain ``sum_d |beta_d|/h``; ``wminus[d]`` / ``wplus[d]`` (arrays
    ``[k][j][i]`` for ``d = x, y, z``) the weight of the neighbour at ``-e_d`` /
    ``+e_d`` in the row's ``- weight * u_neighbour`` term."""
    h = 1.0 / (n + 1)
    beta = np.asarray(velocity, dtype=np.float64).reshape(3, n, n, n)
    dplus = np.abs(beta).sum(axis=0) / h
    wminus = [np.maximum(beta[d], 0.0) / h for d in range(3)]
    wplus = [np.maximum(-beta[d], 0.0) / h for d in range(3)]
    return dplus, wminus, wplus


def assemble(n: int, log_kappa=None, shift: float = 0.0, velocity=None) -> sp.csr_matrix:
    """Sparse ``N x N`` matrix ``A`` (``N = n^3``), lexicographic ``i + n j + n^2 k``;
    ``velocity`` (``(3, N)`` or None) adds the upwind convection term."""
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
    if velocity is not None:
        dplus, wminus, wplus = upwind_weights(n, velocity)
        rows.append(idx.ravel())
        cols.append(idx.ravel())
        vals.append(dplus.ravel())
        for ax, d in ((2, 0), (1, 1), (0, 2)):  # array axis of x, y, z
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ax] = slice(0, n - 1)
            hi[ax] = slice(1, n)
            lo, hi = tuple(lo), tuple(hi)
            # row at hi, neighbour at lo (-e_d); row at lo, neighbour at hi (+e_d)
            rows += [idx[hi].ravel(), idx[lo].ravel()]
            cols += [idx[lo].ravel(), idx[hi].ravel()]
            vals += [-wminus[d][hi].ravel(), -wplus[d][lo].ravel()]
    N = n ** 3
    A = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N)
    )
    return A.tocsr()


def plane_blocks(n: int, log_kappa=None, shift: float = 0.0, velocity=None):
    """Dense plane blocks ``(D, E, F)`` of Eq. originalMatrix.

    ``D[k]`` is the ``n^2 x n^2`` in-plane block of plane ``k``; ``E[k]``
    couples plane ``k`` to ``k-1`` (sub-diagonal, ``E[0] = None``); ``F[k]``
    couples plane ``k`` to ``k+1`` (super-diagonal, ``F[n-1] = None``).
    In-plane order is lexicographic ``i + n j``.
    """
    A = assemble(n, log_kappa, shift, velocity).tocsr()
    m = n * n
    D, E, F = [], [], []
    for k in range(n):
        r = slice(k * m, (k + 1) * m)
        D.append(A[r, r].toarray())
        E.append(A[r, (k - 1) * m:k * m].toarray() if k > 0 else None)
        F.append(A[r, (k + 1) * m:(k + 2) * m].toarray() if k < n - 1 else None)
    return D, E, F


def apply(n: int, log_kappa, u: np.ndarray, shift: float = 0.0, velocity=None) -> np.ndarray:
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
    if velocity is not None:
        dplus, wminus, wplus = upwind_weights(n, velocity)
        out += dplus[..., None] * U
        for ax, dd in ((2, 0), (1, 1), (0, 2)):
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[ax] = slice(0, n - 1)
            hi[ax] = slice(1, n)
            lo, hi = tuple(lo), tuple(hi)
            out[hi] -= wminus[dd][hi][..., None] * U[lo]
            out[lo] -= wplus[dd][lo][..., None] * U[hi]
    out = out.reshape(n ** 3, -1)
    return out[:, 0] if squeeze else out


def codi_exact(n: int) -> np.ndarray:
    """The manufactured solution of the convection-diffusion problem (Section 5):
    ``u = sum_d sin(pi x_d) + sin(3 pi x_d)`` at the nodes."""
    h = 1.0 / (n + 1)
    c = (np.arange(n) + 1.0) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return sum(np.sin(np.pi * t) + np.sin(3 * np.pi * t) for t in (x, y, z)).ravel()


def codi_rhs(n: int, velocity) -> np.ndarray:
    """Right-hand side of the manufactured problem on the discrete operator
    ``assemble(n, None, 0, velocity)``: ``f = -Delta u + beta . grad u`` of the
    exact ``u`` at the nodes, plus the Dirichlet values ``u(x_b)`` of boundary
    neighbours times their row weight (diffusion ``1/h^2`` plus the upwind
    weight), moved from ``A`` to ``f``; ``velocity`` is ``beta`` at the nodes."""
    h = 1.0 / (n + 1)
    c = (np.arange(n) + 1.0) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    pi = np.pi

    def g(t):  # 1D part of u and its derivatives
        return np.sin(pi * t) + np.sin(3 * pi * t)

    def gp(t):
        return pi * np.cos(pi * t) + 3 * pi * np.cos(3 * pi * t)

    def gpp(t):
        return -pi ** 2 * np.sin(pi * t) - 9 * pi ** 2 * np.sin(3 * pi * t)

    beta = np.asarray(velocity, dtype=np.float64).reshape(3, n, n, n)
    f = -(gpp(x) + gpp(y) + gpp(z)) + beta[0] * gp(x) + beta[1] * gp(y) + beta[2] * gp(z)
    _, wminus, wplus = upwind_weights(n, velocity)
    coords = (x, y, z)
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        for side in (0, 1):
            sl = [slice(None)] * 3
            sl[ax] = 0 if side == 0 else n - 1
            sl = tuple(sl)
            pts = [t[sl].copy() for t in coords]
            pts[d] = np.full_like(pts[d], 0.0 if side == 0 else 1.0)
            ub = g(pts[0]) + g(pts[1]) + g(pts[2])
            w = 1.0 / h ** 2 + (wminus[d][sl] if side == 0 else wplus[d][sl])
            f[sl] += w * ub
    return f.ravel()
