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
selection costs.  ``blocked_factor`` runs the sketch variant to the end, as a
cluster kernel would (stop located inside a round, dropped pivots, outputs in
the kernels' form), as the CPU reference for such a kernel.
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


def _fmix32(x):
    """MurmurHash3's 32-bit finaliser (a bijective integer mixer)."""
    x &= 0xFFFFFFFF
    x ^= x >> 16
    x = (x * 0x85EBCA6B) & 0xFFFFFFFF
    x ^= x >> 13
    x = (x * 0xC2B2AE35) & 0xFFFFFFFF
    x ^= x >> 16
    return x


def sketch_signs(rows, block, seed, L=24):
    """L x rows random signs: bit i of fmix32(row * 0x9e3779b9 + block * 0x85ebca77 + seed)."""
    S = np.empty((L, rows))
    for row in range(rows):
        h = _fmix32(row * 0x9E3779B9 + block * 0x85EBCA77 + seed)
        for i in range(L):
            S[i, row] = -1.0 if (h >> i) & 1 else 1.0
    return S


def blocked_factor(C, tol, floor2=0.0, b=16, L=24, seed=0x165667B1):
    """The truncation with b pivots per round, as a cluster kernel would run it:
    per round a random-sign sketch of the trailing rows picks up to b pivots
    (pivoted QR of the sketch), a Householder QR of those columns gives R11 and
    the reflectors, the reflectors update the other columns, and the stop
    (largest remaining column norm <= tol^2 x the largest initial one, or the
    noise floor) is located inside the round from the exact norms below it and
    the new rows inside it.  Returns ``(X, sig, Y, k)`` with
    ``C ~ X diag(sig) Y^T`` (the form of the one-pivot kernels)."""
    A = np.array(C, dtype=np.float64)
    kL, kR = A.shape
    kmax = min(kL, kR)
    tj = np.full(kR, -1)
    gmax = (A * A).sum(0).max()
    thr = tol * tol * gmax
    V = np.zeros((kL, kmax))
    taus, sigs = [], []
    st = 0
    if gmax > thr and gmax > floor2:
        rnd = 0
        while True:
            S = sketch_signs(kL, rnd, seed, L)
            S[:, :st] = 0.0
            rem = tj == -1
            Sk = S @ A
            Sk[:, ~rem] = 0.0
            piv = []
            for p in range(min(b, kL - st)):
                cn = (Sk[p:, :] ** 2).sum(0)
                c = int(np.argmax(cn))
                if not cn[c] > 0:
                    break
                x = Sk[p:, c].copy()
                a = np.linalg.norm(x)
                v = x.copy()
                v[0] += np.copysign(a, x[0])
                v /= np.linalg.norm(v)
                Sk[p:, :] -= 2.0 * np.outer(v, v @ Sk[p:, :])
                piv.append(c)
            npiv = len(piv)
            if npiv == 0:
                break
            P = A[:, piv].copy()
            R11 = np.zeros((npiv, npiv))
            Vb = np.zeros((kL, npiv))
            pt, pb = [], []
            for p in range(npiv):
                r0 = st + p
                x0, xn2 = P[r0, p], (P[r0 + 1:, p] ** 2).sum()
                beta, tau = x0, 0.0
                v = np.zeros(kL)
                v[r0] = 1.0
                if xn2 > 0:
                    beta = -np.copysign(np.sqrt(x0 * x0 + xn2), x0)
                    tau = (beta - x0) / beta
                    v[r0 + 1:] = P[r0 + 1:, p] / (x0 - beta)
                P[:, p:] -= tau * np.outer(v, v @ P[:, p:])
                R11[:p + 1, p] = P[st:st + p + 1, p]
                pt.append(tau)
                pb.append(beta)
                Vb[:, p] = v
            others = np.where(rem & ~np.isin(np.arange(kR), piv))[0]
            for p in range(npiv):
                A[:, others] -= pt[p] * np.outer(Vb[:, p], Vb[:, p] @ A[:, others])
            E = (A[st + npiv:, others] ** 2).sum(0)
            Xr = A[st:st + npiv, others]
            stop = None
            for t in range(1, npiv + 1):
                m = (E + (Xr[t:, :] ** 2).sum(0)).max() if others.size else 0.0
                for tp in range(t, npiv):
                    m = max(m, (R11[t:tp + 1, tp] ** 2).sum())
                if not (m > thr) or not (m > floor2):
                    stop = t
                    break
            cnt = stop if stop is not None else npiv
            for p in range(npiv):
                c = piv[p]
                if p < cnt:
                    taus.append(pt[p])
                    sigs.append(abs(pb[p]))
                    V[:, st + p] = Vb[:, p]
                    tj[c] = st + p
                    A[st:, c] = 0.0
                    A[st:st + p + 1, c] = R11[:p + 1, p]
                else:
                    A[st:st + cnt, c] = R11[:cnt, p]
            st += cnt
            rnd += 1
            if stop is not None or st >= kmax:
                break
    k = st
    X = np.zeros((kL, k))
    for t in range(k):
        qv = np.zeros(kL)
        qv[t] = 1.0
        for tp in range(t, -1, -1):
            qv -= taus[tp] * V[:, tp] * (V[:, tp] @ qv)
        X[:, t] = qv
    sig = np.array(sigs)
    Y = np.zeros((kR, k))
    for j in range(kR):
        for t in range(k):
            val = A[t, j] if (tj[j] < 0 or t <= tj[j]) else 0.0
            Y[j, t] = val / sig[t] if sig[t] > 0 else 0.0
    return X, sig, Y, k


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
