"""Plain dense block cyclic reduction (Section 2.2.2-2.2.3, Algorithms 1-2).

Blocks are dense NumPy arrays; inverses are applied by LAPACK LU solves.  No
compression: this is classic CR, the exact solver that accelerated CR
approximates block by block.

Readings of the paper taken here:

* ``n = 2^q`` planes and ``q = log2 n`` reduction steps (the n = 8 example runs
  three steps to a single block ``D_0^{(3)}``, Section 2.2.2; the general
  algorithm's "q = log N" is read as log2 of the number of planes).
* Red/black schedule (Eq. permuted_system, Eq. next_step): at every step the
  planes at even positions of the current list are eliminated and those at
  odd positions are kept and renumbered 0, 1, ...; the last plane of the list
  has one neighbour, so terms with position ``j+1`` are dropped for it
  (the remark after Eq. schur_complement).  The final survivor is the
  original plane ``n-1``.
* Eq. elim, for kept position ``j`` with neighbours ``j-1``, ``j+1``::

      E'_j = -E_j D_{j-1}^{-1} E_{j-1}
      D'_j =  D_j - E_j D_{j-1}^{-1} F_{j-1} - F_j D_{j+1}^{-1} E_{j+1}
      F'_j = -F_j D_{j+1}^{-1} F_{j+1}
      f'_j =  f_j - E_j D_{j-1}^{-1} f_{j-1} - F_j D_{j+1}^{-1} f_{j+1}

  ``E`` is the sub-diagonal and ``F`` the super-diagonal block row
  (Eq. originalMatrix); ``E_0`` and ``F_last`` do not exist.
* Eq. all_backSubs prints ``E u^{(i+1)} + F u^{(i+1)}``; it is read as
  ``u_e = D_e^{-1} (f_e^{(r)} - E_e u_{e-1} - F_e u_{e+1})`` for an eliminated
  position ``e``, with the step-``r`` right-hand side and the already known
  neighbours ``e-1``, ``e+1`` (dropped when absent).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def schedule(n: int):
    """Red/black schedule: per step the original plane indices present, eliminated, kept."""
    if n < 1 or (n & (n - 1)):
        raise ValueError("number of planes must be a power of two")
    present = list(range(n))
    steps = []
    while len(present) > 1:
        steps.append(
            {"present": list(present), "eliminated": present[0::2], "kept": present[1::2]}
        )
        present = present[1::2]
    return steps, present[0]


class DenseCRFactor:
    """Per-step dense blocks of the reduction (kept for intermediate parity checks).

    ``steps[r]`` holds, for the planes present at step ``r`` (by position):
    ``D``, ``E``, ``F`` (lists of arrays or ``None``) and ``lu`` (LU factors of
    the eliminated positions, keyed by position).  ``coarse`` is the LU of the
    final block ``D^{(q)}``.
    """

    def __init__(self, steps, coarse_D, coarse_lu):
        self.steps = steps
        self.coarse_D = coarse_D
        self.coarse_lu = coarse_lu


def cr_factor(D, E, F) -> DenseCRFactor:
    """Eliminate with Eq. elim until one block is left (Algorithm 1)."""
    D = list(D)
    E = list(E)
    F = list(F)
    steps = []
    while len(D) > 1:
        cnt = len(D)
        lu = {t: sla.lu_factor(D[t]) for t in range(0, cnt, 2)}
        steps.append({"D": D, "E": E, "F": F, "lu": lu})
        nD, nE, nF = [], [], []
        for t in range(1, cnt, 2):
            left = t - 1
            right = t + 1 if t + 1 < cnt else None
            # E_j D_{j-1}^{-1} (.) : solve from the left, D^{-T} applied to E^T
            GE = sla.lu_solve(lu[left], E[t].T, trans=1).T  # E_t D_{t-1}^{-1}
            Dn = D[t] - GE @ F[left]
            En = -GE @ E[left] if E[left] is not None else None
            Fn = None
            if right is not None:
                HF = sla.lu_solve(lu[right], F[t].T, trans=1).T  # F_t D_{t+1}^{-1}
                Dn = Dn - HF @ E[right]
                Fn = -HF @ F[right] if F[right] is not None else None
            nD.append(Dn)
            nE.append(En)
            nF.append(Fn)
        D, E, F = nD, nE, nF
    return DenseCRFactor(steps, D[0], sla.lu_factor(D[0]))


def cr_solve(fac: DenseCRFactor, f_planes):
    """Forward reduction of the RHS (Algorithm 1), coarsest solve, back-substitution (Algorithm 2).

    ``f_planes`` is a list of ``n`` arrays ``(m,)`` or ``(m, r)``; returns the
    solution planes in the same layout.
    """
    f = [np.array(x, dtype=np.float64) for x in f_planes]
    saved = []
    for st in fac.steps:
        D, E, F, lu = st["D"], st["E"], st["F"], st["lu"]
        cnt = len(D)
        saved.append(f)
        nf = []
        for t in range(1, cnt, 2):
            v = f[t] - E[t] @ sla.lu_solve(lu[t - 1], f[t - 1])
            if t + 1 < cnt:
                v = v - F[t] @ sla.lu_solve(lu[t + 1], f[t + 1])
            nf.append(v)
        f = nf
    u = [sla.lu_solve(fac.coarse_lu, f[0])]
    for st, fr in zip(reversed(fac.steps), reversed(saved)):
        D, E, F, lu = st["D"], st["E"], st["F"], st["lu"]
        cnt = len(D)
        full = [None] * cnt
        for i, t in enumerate(range(1, cnt, 2)):
            full[t] = u[i]
        for t in range(0, cnt, 2):
            rhs = fr[t].copy()
            if t - 1 >= 0:
                rhs = rhs - E[t] @ full[t - 1]
            if t + 1 < cnt:
                rhs = rhs - F[t] @ full[t + 1]
            full[t] = sla.lu_solve(lu[t], rhs)
        u = full
    return u


def split_planes(n: int, v: np.ndarray):
    m = n * n
    return [v[k * m:(k + 1) * m] for k in range(n)]


def join_planes(planes) -> np.ndarray:
    return np.concatenate(planes, axis=0)


def transpose_blocks(D, E, F):
    """Blocks of ``A^T``: ``tridiag(F_{i-1}^T, D_i^T, E_{i+1}^T)``."""
    n = len(D)
    Dt = [d.T.copy() for d in D]
    Et = [None] + [F[i - 1].T.copy() for i in range(1, n)]
    Ft = [E[i + 1].T.copy() for i in range(n - 1)] + [None]
    return Dt, Et, Ft


def cr_solve_system(n: int, D, E, F, f: np.ndarray) -> np.ndarray:
    """Solve the block-tridiagonal system for a flat RHS ``(N,)`` or ``(N, r)``."""
    fac = cr_factor(D, E, F)
    return join_planes(cr_solve(fac, split_planes(n, f)))
