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


def test_blocked_factor_matches_one_pivot_accuracy():
    """The round-based factorisation (the reference for a blocked-pivot
    kernel): orthonormal X, C ~ X diag(sig) Y^T within a few times the
    one-pivot truncation's error, rank within two of it."""
    cases = [("decaying", ps.decaying_block(256, 12, 3))] + ps.schur_blocks(n=16, leaf=16)
    for name, C in cases:
        X, sig, Y, k = ps.blocked_factor(C, 1e-6)
        k0 = ps.qrcp_rank(C, 1e-6)
        assert abs(k - k0) <= 2, (name, k, k0)
        assert np.abs(X.T @ X - np.eye(k)).max() < 1e-12
        err = np.linalg.norm(C - (X * sig) @ Y.T, 2) / np.linalg.norm(C, 2)
        assert err < 5e-6, (name, err)
