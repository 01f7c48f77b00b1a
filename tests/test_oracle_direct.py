"""Pins for the exact solvers: dense LU vs the DST closed form."""
import numpy as np
import pytest

import synthetic
from oracle import direct, operator as op


@pytest.mark.parametrize("n,shift", [(8, 0.0), (8, -300.0), (12, 25.0)])
def test_dst_equals_dense_lu(n, shift):
    f = np.stack([synthetic.uniform_rhs(n, s) for s in (0, 1)], axis=1)
    u_lu = direct.dense_solve(n, None, f, shift)
    u_dst = direct.dst_solve(n, f, shift)
    assert np.linalg.norm(u_lu - u_dst) / np.linalg.norm(u_lu) < 1e-12


def test_dst_matrix_orthogonal_symmetric():
    S = direct.dst_matrix(9)
    np.testing.assert_allclose(S @ S, np.eye(9), atol=1e-14)
    np.testing.assert_allclose(S, S.T, atol=0)


def test_dense_solve_residual():
    n = 8
    g = synthetic.gaussian_random_field(n, 3)
    f = synthetic.uniform_rhs(n, 4)
    u = direct.dense_solve(n, g, f)
    r = f - op.apply(n, g, u)
    assert np.linalg.norm(r) / np.linalg.norm(f) < 1e-13
