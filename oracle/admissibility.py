"""Block cluster trees of one plane under weak and standard admissibility, and
the H-compression of a dense plane block on such a partition (Section 2.1).

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this package.

Section 2.1 describes an H-matrix by an index set, a cluster tree, a block
cluster tree and an admissibility condition.  The paper's (standard)
condition: a block ``A_ts`` is stored in low-rank form when
``min(diam(tau), diam(sigma)) <= eta * dist(tau, sigma)``, ``tau`` and
``sigma`` being the convex hulls of the point sets of the clusters ``t`` and
``s``; other blocks are subdivided, and those that reach the leaves stay
dense.  Under weak admissibility the two off-diagonal children of every
diagonal block are low-rank blocks and only the diagonal blocks recurse.

Geometry (a reading: the paper gives no coordinates): the plane's points are
the grid nodes ``((i+1) h, (j+1) h)``, ``h = 1/(n+1)``.  A cluster of the
bisection tree (``oracle.ordering``) holds a full rectangle of nodes
``x0 <= i < x1, y0 <= j < y1``, so its convex hull is the rectangle
``[(x0+1)h, x1 h] x [(y0+1)h, y1 h]``: its diameter is the rectangle's
diagonal and the distance of two clusters is the Euclidean distance of their
rectangles.  Two different clusters of one level are disjoint, so their
distance is at least ``h``; a cluster has distance 0 only to itself.

Subdivision follows the (balanced) cluster tree: an inadmissible pair of
level-``l`` clusters is split into the four pairs of their children.
"""
from __future__ import annotations

import math

import numpy as np

from .ordering import cluster_tree


def _hull(rect, h):
    x0, x1, y0, y1 = rect
    return ((x0 + 1) * h, x1 * h, (y0 + 1) * h, y1 * h)


def diameter(rect, h: float) -> float:
    """Diameter of the convex hull of the cluster's nodes."""
    a0, a1, b0, b1 = _hull(rect, h)
    return math.hypot(a1 - a0, b1 - b0)


def distance(r1, r2, h: float) -> float:
    """Euclidean distance between the convex hulls of two clusters."""
    a0, a1, b0, b1 = _hull(r1, h)
    c0, c1, d0, d1 = _hull(r2, h)
    dx = max(0.0, c0 - a1, a0 - c1)
    dy = max(0.0, d0 - b1, b0 - d1)
    return math.hypot(dx, dy)


def _diam2(rect) -> int:
    """Squared diameter in grid steps (an integer)."""
    x0, x1, y0, y1 = rect
    return (x1 - 1 - x0) ** 2 + (y1 - 1 - y0) ** 2


def _dist2(r1, r2) -> int:
    """Squared distance in grid steps (an integer)."""
    dx = max(0, r2[0] - (r1[1] - 1), r1[0] - (r2[1] - 1))
    dy = max(0, r2[2] - (r1[3] - 1), r1[2] - (r2[3] - 1))
    return dx * dx + dy * dy


def admissible(r1, r2, h: float, eta: float) -> bool:
    """The standard admissibility inequality of Section 2.1 (a cluster is never
    admissible with itself: its distance to itself is 0).  Both sides scale
    with h, so the test is taken in grid steps and squared,
    ``min(diam1^2, diam2^2) <= eta^2 dist^2``: exact integers on the left,
    so ties (a diagonal neighbour at eta = 1) are decided exactly."""
    d2 = _dist2(r1, r2)
    return d2 > 0 and min(_diam2(r1), _diam2(r2)) <= eta * eta * d2


def block_partition(n: int, leaf: int, eta: float | None):
    """Block cluster tree leaves of one plane, in depth-first order (row child
    first, then column child).

    ``eta = None`` gives weak admissibility.  Returns ``(levels, blocks)`` with
    ``levels`` from ``oracle.ordering.cluster_tree`` and ``blocks`` a list of
    ``(level, t, s, lowrank)``: the block ``A[range(t), range(s)]`` of level
    ``level`` (in the permuted order), stored low-rank when ``lowrank``."""
    _, levels = cluster_tree(n, leaf)
    h = 1.0 / (n + 1)
    last = len(levels) - 1
    blocks = []

    def rec(lvl, t, s):
        if eta is None:
            lowrank = t != s
        else:
            lowrank = admissible(levels[lvl][t]["rect"], levels[lvl][s]["rect"], h, eta)
        if lowrank:
            blocks.append((lvl, t, s, True))
            return
        if lvl == last:
            blocks.append((lvl, t, s, False))
            return
        for ct in (2 * t, 2 * t + 1):
            for cs in (2 * s, 2 * s + 1):
                rec(lvl + 1, ct, cs)

    rec(0, 0, 0)
    return levels, blocks


def block_ranges(levels, blk):
    lvl, t, s, _ = blk
    return levels[lvl][t]["range"], levels[lvl][s]["range"]


def compress(A: np.ndarray, levels, blocks, tol: float):
    """H-compression of the dense (permuted) matrix ``A`` on ``blocks``.

    Every low-rank block keeps the singular triplets with ``sigma_i > tol *
    sigma_1`` of that block (the per-block relative accuracy of Section 2.1;
    a zero block gets rank 0); dense blocks are kept as they are.  Returns a
    list of ``(block, U, V)`` (``U @ V.T`` is the block; dense blocks have
    ``V = None`` and ``U`` the block itself)."""
    out = []
    for blk in blocks:
        (r0, r1), (c0, c1) = block_ranges(levels, blk)
        B = A[r0:r1, c0:c1]
        if not blk[3]:
            out.append((blk, B.copy(), None))
            continue
        U, sv, Vt = np.linalg.svd(B, full_matrices=False)
        k = int(np.sum(sv > tol * sv[0])) if sv.size and sv[0] > 0 else 0
        out.append((blk, U[:, :k] * sv[:k], Vt[:k].T))
    return out


def expand(m: int, levels, comp) -> np.ndarray:
    """Dense matrix of an H-compressed representation."""
    A = np.zeros((m, m))
    for blk, U, V in comp:
        (r0, r1), (c0, c1) = block_ranges(levels, blk)
        A[r0:r1, c0:c1] = U if V is None else U @ V.T
    return A


def storage(comp) -> dict:
    """Numbers stored by a compressed representation and its rank profile."""
    words = 0
    ranks = []
    dense_words = 0
    for blk, U, V in comp:
        if V is None:
            words += U.size
            dense_words += U.size
        else:
            words += U.size + V.size
            ranks.append(U.shape[1])
    return {
        "words": int(words),
        "dense_words": int(dense_words),
        "lowrank_blocks": len(ranks),
        "dense_blocks": len(comp) - len(ranks),
        "max_rank": max(ranks) if ranks else 0,
        "mean_rank": float(np.mean(ranks)) if ranks else 0.0,
    }
