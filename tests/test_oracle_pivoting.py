"""Pins for the pivot-selection study (oracle/pivoting_study.py): the
one-pivot reference finds exact ranks and stays within a few columns above
the SVD's rank on a decaying spectrum; blocked selections (sketch,
tournament) reach the same ranks within two on decaying and Schur-complement
blocks."""
import numpy as np

from oracle import pivoting_study as ps


def test_reference_finds_exact_rank():
    rng = np.random.default_rng(4)
    for r in (1, 7, 40):
        A = rng.standard_normal((128, r)) @ rng.standard_normal((r, 96))
        assert ps.qrcp_rank(A, 1e-10) == r


def test_reference_close_to_svd_rank():
    A = ps.decaying_block(256, 12, 3)
    s = np.linalg.svd(A, compute_uv=False)
    k_svd = int(np.sum(s > 1e-6 * s[0]))
    k = ps.qrcp_rank(A, 1e-6)
    assert k_svd <= k <= k_svd + 10


def test_blocked_selections_keep_the_rank():
    cases = [("decaying", ps.decaying_block(256, 12, 3))] + ps.schur_blocks(n=16, leaf=16)
    for name, A in cases:
        k = ps.qrcp_rank(A, 1e-6)
        for kb in (ps.sketch_rank(A, 1e-6, 8, 8), ps.tournament_rank(A, 1e-6, 8, 4)):
            assert abs(kb - k) <= 2, (name, k, kb)
