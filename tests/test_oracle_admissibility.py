"""Pins for the block cluster trees of one plane (Section 2.1: weak and
standard admissibility) and the H-compression on them.

The partition is pinned by the properties that define it, each checked
against brute force from the nodes' coordinates rather than the rectangle
formulas: the blocks tile the matrix exactly once, every low-rank block
satisfies the admissibility inequality with the convex hulls' diameters and
distance computed point by point, every block that was subdivided violates it,
and only leaf pairs stay dense.  The geometry is pinned further by the 5-point
operator: clusters more than one grid step apart share no stencil coupling.
"""
import itertools
import math

import numpy as np
import pytest

import synthetic
from oracle import admissibility as adm
from oracle import operator as op
from oracle.ordering import cluster_tree


def _points(levels, n, lvl, t, perm):
    """The cluster's nodes in grid steps (integers)."""
    r0, r1 = levels[lvl][t]["range"]
    return np.array([(perm[p] % n + 1, perm[p] // n + 1) for p in range(r0, r1)], dtype=np.int64)


def _brute_diam2(P):
    d = P[:, None, :] - P[None, :, :]
    return int((d ** 2).sum(-1).max())


def _brute_dist2(P, Q):
    d = P[:, None, :] - Q[None, :, :]
    return int((d ** 2).sum(-1).min())


@pytest.mark.parametrize("n,leaf", [(8, 4), (8, 16), (16, 16), (16, 32)])
@pytest.mark.parametrize("eta", [None, 0.5, 1.0, 2.0])
def test_blocks_tile_the_plane_matrix_once(n, leaf, eta):
    levels, blocks = adm.block_partition(n, leaf, eta)
    m = n * n
    cover = np.zeros((m, m), dtype=int)
    for blk in blocks:
        (r0, r1), (c0, c1) = adm.block_ranges(levels, blk)
        cover[r0:r1, c0:c1] += 1
    assert np.all(cover == 1)


@pytest.mark.parametrize("n,leaf,eta", [(8, 4, 1.0), (8, 4, 2.0), (16, 16, 0.5), (16, 16, 1.0), (16, 8, 2.0)])
def test_standard_partition_matches_its_definition_by_brute_force(n, leaf, eta):
    """Low-rank blocks are admissible, every subdivided pair and every dense
    block is not (a dense block is a leaf pair), with diameters and distances
    taken over the clusters' nodes one pair at a time."""
    perm, _ = cluster_tree(n, leaf)
    levels, blocks = adm.block_partition(n, leaf, eta)
    last = len(levels) - 1

    def adm_bf(lvl, t, s):
        P, Q = _points(levels, n, lvl, t, perm), _points(levels, n, lvl, s, perm)
        if t == s:
            return False
        return min(_brute_diam2(P), _brute_diam2(Q)) <= eta * eta * _brute_dist2(P, Q)

    for lvl, t, s, lowrank in blocks:
        assert adm_bf(lvl, t, s) == lowrank
        if not lowrank:
            assert lvl == last
        # every ancestor pair was subdivided, so it is not admissible
        a, b = t, s
        for up in range(lvl - 1, -1, -1):
            a, b = a // 2, b // 2
            assert not adm_bf(up, a, b)


@pytest.mark.parametrize("n,leaf", [(8, 4), (16, 32), (32, 64)])
def test_weak_partition_is_the_hodlr_structure(n, leaf):
    """Weak admissibility: the two sibling off-diagonal blocks of every node
    are low rank, the diagonal leaves dense -- 2 (m/b - 1) + m/b blocks."""
    levels, blocks = adm.block_partition(n, leaf, None)
    nleaf = n * n // leaf
    lr = [b for b in blocks if b[3]]
    dn = [b for b in blocks if not b[3]]
    assert len(lr) == 2 * (nleaf - 1) and len(dn) == nleaf
    assert all(t // 2 == s // 2 and t != s for _, t, s, _ in lr)
    assert all(t == s and lvl == len(levels) - 1 for lvl, t, s, _ in dn)


def test_geometry_formulas_match_brute_force():
    n, leaf = 16, 8
    perm, levels = cluster_tree(n, leaf)
    h = 1.0 / (n + 1)
    for lvl in (1, 3, len(levels) - 1):
        for t, s in itertools.product(range(len(levels[lvl])), repeat=2):
            P, Q = _points(levels, n, lvl, t, perm), _points(levels, n, lvl, s, perm)
            assert math.isclose(adm.diameter(levels[lvl][t]["rect"], h), h * math.sqrt(_brute_diam2(P)),
                                rel_tol=1e-12, abs_tol=1e-15)
            if t != s:
                assert math.isclose(adm.distance(levels[lvl][t]["rect"], levels[lvl][s]["rect"], h),
                                    h * math.sqrt(_brute_dist2(P, Q)), rel_tol=1e-12)


@pytest.mark.parametrize("n,leaf,eta", [(16, 16, 1.0), (16, 32, 2.0), (32, 64, 1.0)])
def test_plane_operator_couples_only_neighbouring_clusters(n, leaf, eta):
    """The in-plane block D of the 5-point operator (Eq. originalMatrix): a
    block of two clusters more than one grid step apart (corner neighbours
    included, at sqrt(2) steps) is exactly zero, one of two clusters sharing an
    edge is not -- so with these parameters (no cluster's diameter within eta
    grid steps) every admissible block of D is zero."""
    g = synthetic.gaussian_random_field(n, 2)
    D, _, _ = op.plane_blocks(n, g)
    perm, _ = cluster_tree(n, leaf)
    P = np.array(perm)
    Dk = D[n // 2][np.ix_(P, P)]
    levels, blocks = adm.block_partition(n, leaf, eta)
    h = 1.0 / (n + 1)
    for blk in blocks:
        lvl, t, s, lowrank = blk
        (r0, r1), (c0, c1) = adm.block_ranges(levels, blk)
        B = Dk[r0:r1, c0:c1]
        d = adm.distance(levels[lvl][t]["rect"], levels[lvl][s]["rect"], h)
        if t != s and d > 1.01 * h:
            assert not np.any(B)
        elif t != s:
            assert np.any(B)
        if lowrank:
            assert not np.any(B)


def test_compression_exact_at_zero_tolerance_and_within_bound():
    """H-compression of the inverse of the 2D 5-point operator: exact with
    tol = 0; with tol > 0 every low-rank block's spectral error is at most tol
    times its largest singular value (truncated SVD)."""
    n, leaf = 16, 16
    g = synthetic.gaussian_random_field(n, 3)
    D, _, _ = op.plane_blocks(n, g)
    perm, _ = cluster_tree(n, leaf)
    P = np.array(perm)
    A = np.linalg.inv(D[0][np.ix_(P, P)])
    for eta in (None, 1.0):
        levels, blocks = adm.block_partition(n, leaf, eta)
        comp = adm.compress(A, levels, blocks, 0.0)
        assert np.abs(adm.expand(n * n, levels, comp) - A).max() <= 1e-12 * np.abs(A).max()
        tol = 1e-4
        comp = adm.compress(A, levels, blocks, tol)
        for blk, U, V in comp:
            if V is None:
                continue
            (r0, r1), (c0, c1) = adm.block_ranges(levels, blk)
            B = A[r0:r1, c0:c1]
            s1 = np.linalg.norm(B, 2)
            assert np.linalg.norm(B - U @ V.T, 2) <= tol * s1 * (1 + 1e-8) + 1e-15


def test_standard_admissibility_needs_smaller_ranks_than_weak():
    """Section 2.1 (Figure admisibilities): refining the off-diagonal blocks
    lets the H-inverse of the 2D variable-coefficient Poisson operator reach
    the same per-block accuracy with smaller ranks.  n = 32 plane, leaf 32,
    eta = 1, tol 1e-4."""
    n, leaf = 32, 32
    g = synthetic.gaussian_random_field(n, 1)
    D, _, _ = op.plane_blocks(n, g)
    perm, _ = cluster_tree(n, leaf)
    P = np.array(perm)
    A = np.linalg.inv(D[n // 2][np.ix_(P, P)])
    lw, bw = adm.block_partition(n, leaf, None)
    ls, bs = adm.block_partition(n, leaf, 1.0)
    sw = adm.storage(adm.compress(A, lw, bw, 1e-4))
    ss = adm.storage(adm.compress(A, ls, bs, 1e-4))
    assert ss["max_rank"] < sw["max_rank"]
    assert ss["mean_rank"] < sw["mean_rank"]


@pytest.mark.parametrize("eta", [None, 1.0, 2.0])
def test_truncated_block_cr_is_exact_at_zero_tolerance(eta):
    """oracle.hacr with tol = 0 stores every block exactly: its solve through
    the stored G, H and X (Eq. elim, Eq. all_backSubs) equals dense LU."""
    from oracle import direct
    from oracle.cr import join_planes, split_planes
    from oracle.hacr import Truncator, h_cr_factor, h_cr_solve

    n = 8
    g = synthetic.gaussian_random_field(n, 5)
    D, E, F = op.plane_blocks(n, g)
    f = synthetic.uniform_rhs(n, 1)
    fac = h_cr_factor(D, E, F, Truncator(n, 8, eta, 0.0))
    u = join_planes(h_cr_solve(fac, split_planes(n, f)))
    ref = direct.dense_solve(n, g, f)
    assert np.linalg.norm(u - ref) <= 1e-12 * np.linalg.norm(ref)


def test_truncated_block_cr_error_follows_the_tolerance():
    """Loosening the per-block tolerance by 1e4 raises the solve's error, and
    the error stays within a modest multiple of the tolerance (n = 8)."""
    from oracle import direct
    from oracle.cr import join_planes, split_planes
    from oracle.hacr import Truncator, h_cr_factor, h_cr_solve

    n = 8
    g = synthetic.gaussian_random_field(n, 5)
    D, E, F = op.plane_blocks(n, g)
    f = synthetic.uniform_rhs(n, 1)
    ref = direct.dense_solve(n, g, f)
    errs = []
    for tol in (1e-8, 1e-4):
        fac = h_cr_factor(D, E, F, Truncator(n, 4, 1.0, tol))
        u = join_planes(h_cr_solve(fac, split_planes(n, f)))
        errs.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    assert errs[0] < errs[1] < 1e3 * 1e-4
