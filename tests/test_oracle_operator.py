"""Pins for the oracle's 7-point operator (Section 2.2.1, Eq. probSta)."""
import numpy as np
import pytest

import synthetic
from oracle import operator as op


def test_symmetric_and_apply_matches_assembly():
    n = 6
    g = synthetic.gaussian_random_field(n, 11)
    A = op.assemble(n, g)
    assert abs(A - A.T).max() == 0.0
    u = np.random.default_rng(0).standard_normal((n ** 3, 3))
    np.testing.assert_allclose(op.apply(n, g, u), A @ u, rtol=1e-13, atol=1e-9)


def test_plane_blocks_rebuild_matrix():
    n = 4
    g = synthetic.gaussian_random_field(n, 5)
    A = op.assemble(n, g, shift=-3.0).toarray()
    D, E, F = op.plane_blocks(n, g, shift=-3.0)
    m = n * n
    B = np.zeros_like(A)
    for k in range(n):
        B[k * m:(k + 1) * m, k * m:(k + 1) * m] = D[k]
        if k > 0:
            B[k * m:(k + 1) * m, (k - 1) * m:k * m] = E[k]
        if k < n - 1:
            B[k * m:(k + 1) * m, (k + 1) * m:(k + 2) * m] = F[k]
    np.testing.assert_array_equal(A, B)
    # E, F couple only the same (i, j) column: diagonal blocks
    for k in range(1, n):
        assert np.count_nonzero(E[k] - np.diag(np.diag(E[k]))) == 0


@pytest.mark.parametrize("n", [5, 8])
def test_constant_coefficient_sine_eigenvectors(n):
    """kappa = 1: sin(pi a x) sin(pi b y) sin(pi c z) is an eigenvector with
    eigenvalue (4/h^2) sum sin^2(pi a_d h / 2) (closed form of the 7-point Laplacian)."""
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1) * h
    A = op.assemble(n, None)
    for a, b, c in [(1, 1, 1), (2, 3, 1), (n, 1, n - 1)]:
        v = np.einsum("k,j,i->kji", np.sin(np.pi * c * x), np.sin(np.pi * b * x), np.sin(np.pi * a * x)).ravel()
        lam = 4.0 / h ** 2 * (np.sin(np.pi * a * h / 2) ** 2 + np.sin(np.pi * b * h / 2) ** 2 + np.sin(np.pi * c * h / 2) ** 2)
        np.testing.assert_allclose(A @ v, lam * v, rtol=1e-11, atol=1e-8 * lam)


def _manufactured(n):
    """u* = sin(pi x) sin(2 pi y) sin(pi z), kappa = exp(0.4 sin(2 pi x) cos(pi y) + 0.3 z)."""
    h = 1.0 / (n + 1)
    t = (np.arange(n) + 1) * h
    Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
    g = 0.4 * np.sin(2 * np.pi * X) * np.cos(np.pi * Y) + 0.3 * Z
    kap = np.exp(g)
    u = np.sin(np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(np.pi * Z)
    ux = np.pi * np.cos(np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(np.pi * Z)
    uy = 2 * np.pi * np.sin(np.pi * X) * np.cos(2 * np.pi * Y) * np.sin(np.pi * Z)
    uz = np.pi * np.sin(np.pi * X) * np.sin(2 * np.pi * Y) * np.cos(np.pi * Z)
    lap = -(np.pi ** 2 + 4 * np.pi ** 2 + np.pi ** 2) * u
    gx = 0.8 * np.pi * np.cos(2 * np.pi * X) * np.cos(np.pi * Y)
    gy = -0.4 * np.pi * np.sin(2 * np.pi * X) * np.sin(np.pi * Y)
    gz = 0.3 * np.ones_like(Z)
    f = -kap * (lap + gx * ux + gy * uy + gz * uz)
    return g.ravel(), u.ravel(), f.ravel()


def test_manufactured_solution_second_order():
    """Interior truncation error and the discrete solution's error both fall as O(h^2).

    (Boundary nodes use kappa_p on the boundary face, an O(1) local
    inconsistency confined to one layer of nodes; the solution error is
    still second order.)"""
    from oracle import iterative
    trunc, sol = [], []
    for n in (15, 31):
        g, u, f = _manufactured(n)
        r = (op.apply(n, g, u) - f).reshape(n, n, n)
        trunc.append(np.abs(r[1:-1, 1:-1, 1:-1]).max() / np.abs(f).max())
        uh, _ = iterative.cg(op.assemble(n, g), f, rtol=1e-12)
        sol.append(np.abs(uh - u).max())
    for e in (trunc, sol):
        rate = np.log(e[0] / e[1]) / np.log(2.0)
        assert 1.7 < rate < 2.5, (e, rate)
    assert sol[1] < 5e-3
