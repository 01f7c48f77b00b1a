"""Convection-diffusion (Section 5, Eq. codi; first-order upwind, non-symmetric)
through the C ABI, against the oracle's upwind operator.

Bars: exact (tol = 0) FP64 factorisations match a sparse LU of the oracle's
matrix to 1e-11; the FP64 residual kernel matches the oracle's operator to
1e-13 of the residual scale; refined FP32 solves (forward and transpose) reach
1e-10 in the oracle's relative residual of A (resp. A^T)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic
from oracle import operator as op

from gpu_util import empty_like_cols, from_cols, rel, to_cols

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acr():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1701_00182_gb300 import build as b

    b.build()
    import paper_1701_00182_gb300 as m

    return m


def _solve(acr, h, f, trans=False):
    b = to_cols(f)
    x = empty_like_cols(b)
    (acr.acr_solve_transpose if trans else acr.acr_solve)(h, b, x)
    return from_cols(x)[:, 0]


@pytest.mark.parametrize("alpha,leaf", [(20.0, 32), (200.0, 64)])
def test_exact_fp64_matches_sparse_lu(acr, alpha, leaf):
    n = 16
    v = synthetic.vortex_velocity(n, alpha)
    A = op.assemble(n, None, 0.0, v).tocsc()
    f = synthetic.uniform_rhs(n, 11)
    h = acr.acr_factor(n, None, 0.0, leaf, velocity=v)
    u = _solve(acr, h, f)
    assert rel(u, spla.spsolve(A, f)) < 1e-11
    # the transpose solve inverts A^T (not A: the operator is non-symmetric)
    ut = _solve(acr, h, f, trans=True)
    assert rel(ut, spla.spsolve(A.T.tocsc(), f)) < 1e-11
    assert rel(ut, u) > 1e-3


def test_residual_kernel_matches_oracle(acr):
    n = 16
    v = synthetic.vortex_velocity(n, 100.0)
    g = synthetic.gaussian_random_field(n, 2)
    X = np.random.default_rng(3).standard_normal((n ** 3, 2))
    Bm = np.random.default_rng(4).standard_normal((n ** 3, 2))
    h = acr.acr_factor(n, g, 1e-2, 64, velocity=v)
    b, x = to_cols(Bm), to_cols(X)
    r = empty_like_cols(b)
    acr.acr_residual(h, b, x, r)
    want = Bm - op.apply(n, g, X, 0.0, v)
    assert np.abs(from_cols(r) - want).max() <= 1e-13 * np.abs(op.apply(n, g, X, 0.0, v)).max()


def test_manufactured_problem_fp32_refined(acr):
    """The paper's manufactured convection-diffusion problem (alpha = 100) by
    FP32 ACR (tensor cores) + FP64 refinement: relative residual 1e-10 in the
    oracle's operator, and the discrete solution's distance to the exact u
    equals the oracle's (sparse LU) discretisation error."""
    n = 32
    v = synthetic.vortex_velocity(n, 100.0)
    f = op.codi_rhs(n, v)
    h = acr.acr_factor(n, None, 1e-6, 64, precision=acr.ACR_FP32, tensor_cores=1, velocity=v)
    b = to_cols(f)
    x = empty_like_cols(b)
    it, relr, _ = acr.acr_solve_ir(h, b, x, rtol=1e-10, maxit=60)
    u = from_cols(x)[:, 0]
    A = op.assemble(n, None, 0.0, v)
    assert np.linalg.norm(f - A @ u) <= 1.01e-10 * np.linalg.norm(f)
    ref = spla.spsolve(A.tocsc(), f)
    assert rel(u, ref) < 1e-7  # residual 1e-10 times the operator's condition number
    ex = op.codi_exact(n)
    assert abs(np.abs(u - ex).max() - np.abs(ref - ex).max()) < 1e-5


def test_transpose_refinement_uses_the_transposed_residual(acr):
    n = 32
    v = synthetic.vortex_velocity(n, 100.0)
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 12)
    h = acr.acr_factor(n, g, 1e-6, 64, precision=acr.ACR_FP32, velocity=v)
    b = to_cols(f)
    x = empty_like_cols(b)
    it, relr, _ = acr.acr_solve_ir_transpose(h, b, x, rtol=1e-10, maxit=60)
    u = from_cols(x)[:, 0]
    A = op.assemble(n, g, 0.0, v)
    assert np.linalg.norm(f - A.T @ u) <= 1.01e-10 * np.linalg.norm(f)
    assert np.linalg.norm(f - A @ u) > 1e-6 * np.linalg.norm(f)  # A^T, not A, was inverted
