"""2D planar bisection cluster tree of one plane (Section 3.1, Section 2.1.1).

The paper clusters the ``n^2`` unknowns of a plane by "binary space
partitioning" of the 2D plane and uses the geometry to build each block's
hierarchical matrix.  It does not state the split rule; the reading taken here
is: split the current rectangle in half along its longer side, along ``x``
when the sides are equal, until a cluster holds ``leaf`` points.  Clusters are
numbered level by level (children of node ``c`` are ``2c`` and ``2c+1``) and
the points of every leaf are listed in lexicographic order (``x`` fastest), so
every cluster is a contiguous range of the permuted index.

Under weak admissibility each level-``l`` node couples its two children by one
off-diagonal block; in the 5-point in-plane stencil those blocks hold exactly
one entry per grid edge cut by the bisection, which fixes their exact ranks.
"""
from __future__ import annotations


def cluster_tree(n: int, leaf: int):
    """Return ``(perm, levels)``.

    ``perm[p]`` is the lexicographic in-plane index ``i + n j`` of the point at
    permuted position ``p``.  ``levels[l]`` lists, for every node of level
    ``l`` (root = level 0, the last entry = leaves), a dict with its rectangle
    ``(x0, x1, y0, y1)``, its permuted range ``(start, stop)`` and, for
    non-leaf nodes, ``cut``: the list of cut edges ``(p, q)`` with ``p`` in the
    first child and ``q`` in the second, ordered along the cut.
    """
    m = n * n
    if m % leaf or (m // leaf) & (m // leaf - 1):
        raise ValueError("leaf size must split n^2 into a power-of-two number of leaves")
    rects = [[(0, n, 0, n)]]
    while (rects[-1][0][1] - rects[-1][0][0]) * (rects[-1][0][3] - rects[-1][0][2]) > leaf:
        nxt = []
        for x0, x1, y0, y1 in rects[-1]:
            if (x1 - x0) >= (y1 - y0):
                xm = (x0 + x1) // 2
                nxt += [(x0, xm, y0, y1), (xm, x1, y0, y1)]
            else:
                ym = (y0 + y1) // 2
                nxt += [(x0, x1, y0, ym), (x0, x1, ym, y1)]
        rects.append(nxt)
    perm = []
    for x0, x1, y0, y1 in rects[-1]:
        for y in range(y0, y1):
            for x in range(x0, x1):
                perm.append(x + n * y)
    pos = {g: p for p, g in enumerate(perm)}
    levels = []
    for lvl, rs in enumerate(rects):
        size = m // len(rs)
        nodes = []
        for c, (x0, x1, y0, y1) in enumerate(rs):
            node = {"rect": (x0, x1, y0, y1), "range": (c * size, (c + 1) * size)}
            if lvl + 1 < len(rects):
                a = rects[lvl + 1][2 * c]
                cut = []
                if a[1] < x1:  # split along x at a[1]
                    for y in range(y0, y1):
                        cut.append((pos[(a[1] - 1) + n * y], pos[a[1] + n * y]))
                else:  # split along y at a[3]
                    for x in range(x0, x1):
                        cut.append((pos[x + n * (a[3] - 1)], pos[x + n * a[3]]))
                node["cut"] = cut
            nodes.append(node)
        levels.append(nodes)
    return perm, levels
