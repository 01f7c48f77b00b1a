"""Pins for the plane cluster tree (Section 3.1) and the exact level-0 ranks."""
import numpy as np
import pytest

import synthetic
from oracle import operator as op
from oracle import ordering


@pytest.mark.parametrize("n,leaf,ranks", [(16, 32, [16, 8, 8]), (128, 64, [128, 64, 64, 32, 32, 16, 16, 8]), (64, 64, [64, 32, 32, 16, 16, 8])])
def test_cut_sizes(n, leaf, ranks):
    perm, levels = ordering.cluster_tree(n, leaf)
    assert sorted(perm) == list(range(n * n))
    assert len(levels) == len(ranks) + 1
    for lvl, nodes in enumerate(levels[:-1]):
        assert {len(nd["cut"]) for nd in nodes} == {ranks[lvl]}
    assert all(nd["range"][1] - nd["range"][0] == leaf for nd in levels[-1])


def test_cut_edges_are_grid_edges_between_children():
    n, leaf = 16, 16
    perm, levels = ordering.cluster_tree(n, leaf)
    for lvl, nodes in enumerate(levels[:-1]):
        for c, nd in enumerate(nodes):
            c1 = levels[lvl + 1][2 * c]["range"]
            c2 = levels[lvl + 1][2 * c + 1]["range"]
            for p, q in nd["cut"]:
                assert c1[0] <= p < c1[1] and c2[0] <= q < c2[1]
                a, b = perm[p], perm[q]
                dx, dy = abs(a % n - b % n), abs(a // n - b // n)
                assert dx + dy == 1


@pytest.mark.parametrize("n,leaf", [(8, 8), (16, 32)])
def test_offdiagonal_ranks_equal_cut_counts(n, leaf):
    """Weak admissibility on a 5-point plane: each off-diagonal block of D_k has
    numerical rank equal to the number of cut grid edges (LAPACK rank vs geometry)."""
    g = synthetic.gaussian_random_field(n, 2)
    D, _, _ = op.plane_blocks(n, g)
    perm, levels = ordering.cluster_tree(n, leaf)
    P = np.array(perm)
    Dk = D[n // 2][np.ix_(P, P)]
    for lvl, nodes in enumerate(levels[:-1]):
        for c, nd in enumerate(nodes):
            a = levels[lvl + 1][2 * c]["range"]
            b = levels[lvl + 1][2 * c + 1]["range"]
            blk = Dk[a[0]:a[1], b[0]:b[1]]
            assert np.linalg.matrix_rank(blk) == len(nd["cut"])
