"""Block cyclic reduction with every stored plane block truncated on a block
cluster tree: ACR's accuracy under weak or standard admissibility
(Section 2.2.2, Eq. elim, with the H-arithmetic of Section 2.1).

Test infrastructure (see ``oracle/__init__.py``).  ACR replaces every
plane block of the reduction by an H-matrix and truncates the result of
every block operation to the tolerance.  This emulation keeps the dense
arithmetic of ``oracle.cr`` and truncates each block it stores, at the
step where Eq. elim produces it, on the chosen partition (weak = HODLR,
or standard admissibility with parameter eta), each low-rank block to
``sigma_i > tol sigma_1`` of that block:

  eliminated e:  X_e = T(D_e^{-1});   E_e, F_e = T(E_e), T(F_e)
  kept j:        G_j = T(E_j X_{j-1}),  H_j = T(F_j X_{j+1}),
                 D'_j = T(D_j - G_j F_{j-1} - H_j E_{j+1}),
                 E'_j = T(-G_j E_{j-1}),  F'_j = T(-H_j F_{j+1});

the coarsest block is solved densely.  The solve applies Eq. elim to the
right-hand side with the stored G, H and back-substitutes with X
(Eq. all_backSubs).  It measures what the choice of partition costs in
accuracy and rank, not ACR's operation counts.
"""
from __future__ import annotations

import numpy as np

from . import admissibility as adm
from .ordering import cluster_tree


class Truncator:
    """T(M) on a fixed partition of one plane, with storage and rank records."""

    def __init__(self, n: int, leaf: int, eta, tol: float):
        perm, _ = cluster_tree(n, leaf)
        self.P = np.array(perm)
        self.levels, self.blocks = adm.block_partition(n, leaf, eta)
        self.tol = tol
        self.m = n * n
        self.words = 0
        self.ranks = []

    def __call__(self, M, record: bool = True):
        if M is None:
            return None
        Mp = M[np.ix_(self.P, self.P)]
        comp = adm.compress(Mp, self.levels, self.blocks, self.tol)
        if record:
            st = adm.storage(comp)
            self.words += st["words"]
            self.ranks += [U.shape[1] for _, U, V in comp if V is not None]
        Tp = adm.expand(self.m, self.levels, comp)
        out = np.empty_like(Tp)
        out[np.ix_(self.P, self.P)] = Tp
        return out


def h_cr_factor(D, E, F, trunc: Truncator):
    """Eq. elim with every stored block truncated (see the module text)."""
    D, E, F = list(D), list(E), list(F)
    steps = []
    while len(D) > 1:
        cnt = len(D)
        X = {t: trunc(np.linalg.inv(D[t])) for t in range(0, cnt, 2)}
        Es = {t: trunc(E[t]) for t in range(0, cnt, 2)}
        Fs = {t: trunc(F[t]) for t in range(0, cnt, 2)}
        G, H = {}, {}
        nD, nE, nF = [], [], []
        for t in range(1, cnt, 2):
            left, right = t - 1, (t + 1 if t + 1 < cnt else None)
            G[t] = trunc(E[t] @ X[left])
            Dn = D[t] - G[t] @ F[left]
            En = trunc(-G[t] @ E[left], record=False) if E[left] is not None else None
            Fn = None
            if right is not None:
                H[t] = trunc(F[t] @ X[right])
                Dn = Dn - H[t] @ E[right]
                Fn = trunc(-H[t] @ F[right], record=False) if F[right] is not None else None
            nD.append(trunc(Dn, record=False))
            nE.append(En)
            nF.append(Fn)
        steps.append({"cnt": cnt, "X": X, "E": Es, "F": Fs, "G": G, "H": H})
        D, E, F = nD, nE, nF
    return {"steps": steps, "coarse_inv": np.linalg.inv(D[0])}


def h_cr_solve(fac, f_planes):
    f = [np.array(x, dtype=np.float64) for x in f_planes]
    saved = []
    for st in fac["steps"]:
        cnt = st["cnt"]
        saved.append(f)
        nf = []
        for t in range(1, cnt, 2):
            v = f[t] - st["G"][t] @ f[t - 1]
            if t + 1 < cnt:
                v = v - st["H"][t] @ f[t + 1]
            nf.append(v)
        f = nf
    u = [fac["coarse_inv"] @ f[0]]
    for st, fr in zip(reversed(fac["steps"]), reversed(saved)):
        cnt = st["cnt"]
        full = [None] * cnt
        for i, t in enumerate(range(1, cnt, 2)):
            full[t] = u[i]
        for t in range(0, cnt, 2):
            rhs = fr[t].copy()
            if t - 1 >= 0:
                rhs = rhs - st["E"][t] @ full[t - 1]
            if t + 1 < cnt:
                rhs = rhs - st["F"][t] @ full[t + 1]
            full[t] = st["X"][t] @ rhs
        u = full
    return u
