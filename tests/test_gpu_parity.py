"""Parity of the CUDA ACR path (through the C ABI) with the CPU oracle.

Bars: uncompressed (tol = 0) runs match the oracle to 1e-12 in relative
error; compressed FP64 runs to 10x the truncation tolerance; refined runs
reach the requested relative residual, checked with the oracle's operator.
"""
import numpy as np
import pytest

import synthetic
from oracle import cr, direct, iterative, operator as op

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
    return from_cols(x)[:, 0] if f.ndim == 1 else from_cols(x)


@pytest.mark.parametrize("n,leaf", [(2, 4), (4, 4), (8, 8), (8, 64), (16, 32)])
def test_uncompressed_matches_dense_lu(acr, n, leaf):
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 0)
    h = acr.acr_factor(n, g, 0.0, leaf)
    u = _solve(acr, h, f)
    ref = direct.dense_solve(n, g, f)
    assert rel(u, ref) < 1e-12


def test_uncompressed_constant_kappa_matches_dst(acr):
    n = 16
    f = synthetic.uniform_rhs(n, 0)
    h = acr.acr_factor(n, None, 0.0, 32)
    assert rel(_solve(acr, h, f), direct.dst_solve(n, f)) < 1e-12


def test_intermediate_blocks_match_dense_cr(acr):
    """Per-level X = D^{-1}, E, F of eliminated planes and G = E X_{j-1},
    H = F X_{j+1} of kept planes against the oracle's dense Eq. elim blocks."""
    n, leaf = 16, 32
    g = synthetic.gaussian_random_field(n, 4)
    D, E, F = op.plane_blocks(n, g)
    fac = cr.cr_factor(D, E, F)
    h = acr.acr_factor(n, g, 0.0, leaf)
    for r, st in enumerate(fac.steps):
        cnt = len(st["D"])
        for i in range(cnt // 2):
            e = 2 * i
            Xref = np.linalg.inv(st["D"][e])
            assert rel(acr.acr_get_factor_block(h, 0, r, i), Xref) < 1e-11
            if st["E"][e] is not None:
                assert rel(acr.acr_get_factor_block(h, 1, r, i), st["E"][e]) < 1e-11
            assert rel(acr.acr_get_factor_block(h, 2, r, i), st["F"][e]) < 1e-11
            k = e + 1
            Gref = st["E"][k] @ Xref
            assert rel(acr.acr_get_factor_block(h, 3, r, i), Gref) < 1e-11
            if k + 1 < cnt:
                Href = st["F"][k] @ np.linalg.inv(st["D"][k + 1])
                assert rel(acr.acr_get_factor_block(h, 4, r, i), Href) < 1e-11
    Xc = np.linalg.inv(fac.coarse_D)
    assert rel(acr.acr_get_factor_block(h, 5, 0, 0), Xc) < 1e-11


@pytest.mark.parametrize("core_svd", [1, 2])
@pytest.mark.parametrize("n,leaf,tol", [(16, 32, 1e-8), (16, 16, 1e-6), (32, 32, 1e-6)])
def test_compressed_fp64_within_ten_tol(acr, n, leaf, tol, core_svd):
    """FP64 ACR as a direct solver within 10x the truncation tolerance, with
    either truncation of the recompression core (1: Jacobi SVD, 2: pivoted QR)."""
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 0)
    h = acr.acr_factor(n, g, tol, leaf, core_svd=core_svd)
    u = _solve(acr, h, f)
    ref = direct.dense_solve(n, g, f) if n <= 16 else iterative.reference_solve(n, g, f, rtol=1e-13)
    assert rel(u, ref) < 10 * tol


def test_multi_rhs_padded_ld_and_alias(acr):
    n = 8
    g = synthetic.gaussian_random_field(n, 2)
    F = synthetic.multi_rhs(n, [5, 6, 7])
    h = acr.acr_factor(n, g, 0.0, 16)
    b = to_cols(F, ld_pad=5)
    assert b.stride(1) == n ** 3 + 5
    acr.acr_solve(h, b, b)  # in place
    ref = direct.dense_solve(n, g, F)
    assert rel(from_cols(b), ref) < 1e-12


def test_transpose_solve(acr):
    n = 8
    g = synthetic.gaussian_random_field(n, 3)
    f = synthetic.uniform_rhs(n, 1)
    h = acr.acr_factor(n, g, 0.0, 8)
    # A is symmetric: the exact transpose solve is the solve
    assert rel(_solve(acr, h, f, trans=True), direct.dense_solve(n, g, f)) < 1e-12
    # with truncation M^{-1} is not symmetric; <M^{-T} a, b> = <a, M^{-1} b> still holds
    h2 = acr.acr_factor(16, synthetic.gaussian_random_field(16, 3), 1e-3, 16)
    a = synthetic.uniform_rhs(16, 11)
    bb = synthetic.uniform_rhs(16, 12)
    lhs = _solve(acr, h2, a, trans=True) @ bb
    rhs = a @ _solve(acr, h2, bb)
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs) * 10


def test_residual_matches_oracle(acr):
    n = 8
    g = synthetic.gaussian_random_field(n, 5)
    f = synthetic.multi_rhs(n, [1, 2])
    u = np.random.default_rng(0).standard_normal(f.shape)
    h = acr.acr_factor(n, g, 0.0, 8)
    b, x = to_cols(f), to_cols(u)
    r = empty_like_cols(b)
    relg = acr.acr_residual(h, b, x, r)
    np.testing.assert_allclose(from_cols(r), f - op.apply(n, g, u), rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(relg, iterative.rel_residual(n, g, u, f), rtol=1e-12)


def test_fp32_factor_with_fp64_refinement(acr):
    n = 16
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.multi_rhs(n, [2, 3])
    h = acr.acr_factor(n, g, 1e-6, 32, precision=acr.ACR_FP32)
    b = to_cols(f)
    x = empty_like_cols(b)
    it, relr, _ = acr.acr_solve_ir(h, b, x, rtol=1e-10, maxit=30)
    u = from_cols(x)
    assert max(relr) <= 1e-10 and it <= 30
    assert np.all(iterative.rel_residual(n, g, u, f) <= 1e-10 * 1.01)
    assert rel(u, direct.dense_solve(n, g, f)) < 1e-8


def test_helmholtz_fgmres(acr):
    n = 16
    w = synthetic.helmholtz_omega(n)
    f = synthetic.point_source(n, 3)
    h = acr.acr_factor(n, None, 1e-4, 32, precision=acr.ACR_FP32, shift=-w * w)
    b = to_cols(f)
    x = empty_like_cols(b)
    it, relr, _ = acr.acr_solve_fgmres(h, b, x, rtol=1e-10, restart=50, maxit=200)
    assert max(relr) <= 1e-10
    assert rel(from_cols(x)[:, 0], direct.dst_solve(n, f, shift=-w * w)) < 1e-7


def test_stats_report_exact_level0_ranks(acr):
    n, leaf = 16, 32
    h = acr.acr_factor(n, None, 1e-8, leaf)
    s = acr.acr_get_stats(h)
    assert s["levels_cr"] == 4 and s["levels_h"] == 3
    assert s["max_rank_d"][0] == [16, 8, 8]
    assert s["factor_bytes"] > 0 and s["t_factor_ms"] > 0
    assert all(0 <= k <= 128 for row in s["max_rank"] for k in row)


def test_solve_graphs_replay_bit_identical(acr):
    """Captured solve sweeps (one CUDA graph per nrhs / transpose) give the
    same bits as the eager launches, on repeated and refined solves."""
    n = 16
    g = synthetic.gaussian_random_field(n, 6)
    F = synthetic.multi_rhs(n, [1, 2, 3])
    he = acr.acr_factor(n, g, 1e-6, 32, precision=acr.ACR_FP32)
    hg = acr.acr_factor(n, g, 1e-6, 32, precision=acr.ACR_FP32, graphs=1)
    for cols in ([0], [0, 1, 2], [0]):
        b = to_cols(F[:, cols])
        xe, xg = empty_like_cols(b), empty_like_cols(b)
        acr.acr_solve(he, b, xe)
        acr.acr_solve(hg, b, xg)
        np.testing.assert_array_equal(from_cols(xg), from_cols(xe))
        acr.acr_solve_transpose(he, b, xe)
        acr.acr_solve_transpose(hg, b, xg)
        np.testing.assert_array_equal(from_cols(xg), from_cols(xe))
    assert acr.acr_get_stats(hg)["graphs_captured"] == 4
    b = to_cols(F)
    xe, xg = empty_like_cols(b), empty_like_cols(b)
    ite, rele, _ = acr.acr_solve_ir(he, b, xe, rtol=1e-10)
    itg, relg, _ = acr.acr_solve_ir(hg, b, xg, rtol=1e-10)
    assert ite == itg and max(relg) <= 1e-10
    np.testing.assert_array_equal(from_cols(xg), from_cols(xe))
    hg.close()  # a handle with a private stream and captured graphs tears down cleanly
    he.close()


def test_fp32_tensor_core_gemms_match_fma_path(acr):
    """FP32 factorisation with the 3xTF32 tensor-core GEMM tiles agrees with the
    FP32-FMA tiles to FP32-level accuracy and still refines to 1e-10."""
    n = 32
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.multi_rhs(n, [4, 5])
    hf = acr.acr_factor(n, g, 1e-6, 32, precision=acr.ACR_FP32)
    ht = acr.acr_factor(n, g, 1e-6, 32, precision=acr.ACR_FP32, tensor_cores=1)
    Xf = acr.acr_get_factor_block(hf, 0, 0, 3)
    Xt = acr.acr_get_factor_block(ht, 0, 0, 3)
    assert rel(Xt, Xf) < 1e-4
    b = to_cols(f)
    x = empty_like_cols(b)
    it, relr, _ = acr.acr_solve_ir(ht, b, x, rtol=1e-10, maxit=40)
    assert max(relr) <= 1e-10
    assert np.all(iterative.rel_residual(n, g, from_cols(x), f) <= 1.01e-10)


@pytest.mark.parametrize("coarse_dense_max,dense", [(0, 1), (-1, 0)])
def test_coarsest_plane_dense_fp64_and_hodlr(acr, coarse_dense_max, dense):
    """The coarsest block is factorised densely in FP64 (default for n^2 <= 4096)
    or inverted as a HODLR matrix; both reach the oracle's coarsest inverse."""
    n = 16
    g = synthetic.gaussian_random_field(n, 8)
    D, E, F = op.plane_blocks(n, g)
    fac = cr.cr_factor(D, E, F)
    h = acr.acr_factor(n, g, 0.0, 32, coarse_dense_max=coarse_dense_max)
    assert acr.acr_get_stats(h)["coarse_dense"] == dense
    assert rel(acr.acr_get_factor_block(h, 5, 0, 0), np.linalg.inv(fac.coarse_D)) < 1e-12
    f = synthetic.uniform_rhs(n, 3)
    assert rel(_solve(acr, h, f), direct.dense_solve(n, g, f)) < 1e-12


@pytest.mark.parametrize("core_svd", [1, 2])
def test_core_truncation_jacobi_and_pivoted_qr(acr, core_svd):
    """Both truncations of the recompression core (Jacobi SVD, pivoted QR) give
    a FP64 direct solve within the accuracy bar, and compress the blocks."""
    n = 16
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 0)
    h = acr.acr_factor(n, g, 1e-6, 16, core_svd=core_svd)
    assert rel(_solve(acr, h, f), direct.dense_solve(n, g, f)) < 1e-5
    s = acr.acr_get_stats(h)
    assert max(s["max_rank"][1]) < 64
