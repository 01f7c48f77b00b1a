"""Choosing several pivots per synchronisation in the rank-revealing QR of the
recompression (Section 2.1: every low-rank block truncated to its relative
accuracy; the GPU path uses a column-pivoted Householder QR whose pivot
search needs one cluster-wide barrier per column).

Test infrastructure, run as ``python -m oracle.pivoting_study``.  Three ways
to pick the pivots, each followed by the same Householder steps and the same
stop (largest remaining column norm <= tol x largest initial column norm):

* ``qrcp_rank``: one pivot at a time, the largest remaining column (the
  reference, what the GPU kernels do);
* ``sketch_rank``: b pivots at a time, chosen by a pivoted QR of a Gaussian
  sketch (b + p rows) of the trailing matrix;
* ``tournament_rank``: b pivots at a time by a tournament -- the columns are
  split in NC groups (the CTAs of a cluster), each group nominates b
  columns by its own pivoted QR, and a pivoted QR of the NC x b nominees
  picks the b pivots.

The rank each one reaches on a block measures how much rank a blocked
selection costs.
"""
from __future__ import annotations

import numpy as np


def _householder_step(A, st):
    x = A[st:, st]
    a = np.linalg.norm(x)
    if a == 0.0:
        return False
    v = x.copy()
    v[0] += np.copysign(a, x[0])
    v /= np.linalg.norm(v)
    A[st:, st:] -= 2.0 * np.outer(v, v @ A[st:, st:])
    return True


def _pivoted_selection(T, cnt):
    """Indices of up to ``cnt`` columns of T by a pivoted (Gram-Schmidt) QR."""
    T = T.copy()
    sel = []
    sn = (T * T).sum(0)
    for _ in range(min(cnt, T.shape[0], T.shape[1])):
        j = int(np.argmax(sn))
        if not sn[j] > 0.0:
            break
        sel.append(j)
        q = T[:, j] / np.linalg.norm(T[:, j])
        T -= np.outer(q, q @ T)
        sn = (T * T).sum(0)
        sn[sel] = -1.0
    return sel


def qrcp_rank(A, tol):
    A = np.array(A, dtype=np.float64)
    thr = tol * tol * (A * A).sum(0).max()
    for st in range(min(A.shape)):
        nrm = (A[st:, st:] ** 2).sum(0)
        j = int(np.argmax(nrm))
        if not nrm[j] > thr:
            return st
        A[:, [st, st + j]] = A[:, [st + j, st]]
        if not _householder_step(A, st):
            return st
    return min(A.shape)


def _blocked(A, tol, choose):
    A = np.array(A, dtype=np.float64)
    thr = tol * tol * (A * A).sum(0).max()
    st = 0
    while st < min(A.shape):
        T = A[st:, st:]
        if not (T * T).sum(0).max() > thr:
            return st
        sel = choose(T)
        rest = [j for j in range(T.shape[1]) if j not in set(sel)]
        A[:, st:] = A[:, st:][:, sel + rest]
        for _ in range(len(sel)):
            if not (A[st:, st:] ** 2).sum(0).max() > thr or not _householder_step(A, st):
                return st
            st += 1
    return st


def sketch_rank(A, tol, b=16, p=8, seed=0):
    rng = np.random.default_rng(seed)

    def choose(T):
        S = rng.standard_normal((min(b + p, T.shape[0]), T.shape[0])) @ T
        return _pivoted_selection(S, b)

    return _blocked(A, tol, choose)


def tournament_rank(A, tol, b=16, groups=8):
    def choose(T):
        nominees = []
        for g in np.array_split(np.arange(T.shape[1]), groups):
            if g.size:
                nominees += [int(g[j]) for j in _pivoted_selection(T[:, g], b)]
        return [nominees[j] for j in _pivoted_selection(T[:, nominees], b)]

    return _blocked(A, tol, choose)


def decaying_block(s, decade, seed):
    """Random s x s block with singular values 10^(-i / decade)."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((s, s)))
    V, _ = np.linalg.qr(rng.standard_normal((s, s)))
    return (U * 10.0 ** (-np.arange(s) / decade)) @ V.T


def schur_blocks(n=32, leaf=64, seed=1):
    """Off-diagonal blocks of the inverse Schur complements of dense block CR
    (Eq. elim), in the bisection order: what ACR truncates."""
    import synthetic

    from .cr import cr_factor
    from .operator import plane_blocks
    from .ordering import cluster_tree

    g = synthetic.gaussian_random_field(n, seed)
    D, E, F = plane_blocks(n, g)
    fac = cr_factor(D, E, F)
    perm, levels = cluster_tree(n, leaf)
    P = np.array(perm)
    out = []
    for r in range(1, len(fac.steps)):
        X = np.linalg.inv(fac.steps[r]["D"][0][np.ix_(P, P)])
        for lvl in (0, 1, 2):
            a, c = levels[lvl + 1][0]["range"], levels[lvl + 1][1]["range"]
            out.append(("inv(D^(%d)) level %d" % (r, lvl), X[a[0]:a[1], c[0]:c[1]]))
    return out


def main():
    tol = 1e-6
    cases = [("sigma_i = 10^(-i/12), 512", decaying_block(512, 12, 1)),
             ("sigma_i = 10^(-i/20), 512", decaying_block(512, 20, 2)),
             ("sigma_i = 10^(-i/12), 256", decaying_block(256, 12, 3))] + schur_blocks()
    print("| block | shape | one pivot per step | sketch b=16 p=8 | sketch b=8 p=56 | tournament b=8 | tournament b=16 |")
    print("|---|---|---:|---:|---:|---:|---:|")
    for name, A in cases:
        print(f"| {name} | {A.shape[0]} x {A.shape[1]} | {qrcp_rank(A, tol)} | {sketch_rank(A, tol, 16, 8)} | "
              f"{sketch_rank(A, tol, 8, 56)} | {tournament_rank(A, tol, 8)} | {tournament_rank(A, tol, 16)} |",
              flush=True)


if __name__ == "__main__":
    main()
