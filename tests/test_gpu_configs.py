"""The benchmark's workload configurations, run through the C ABI and checked
with the oracle: the operator residual is exact at any size, and at n = 64 the
oracle's FP64 Krylov solution is the reference."""
import numpy as np
import pytest

import synthetic
from oracle import iterative

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


@pytest.fixture(scope="module")
def grf64():
    n = 64
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 2)
    ref = iterative.reference_solve(n, g, f, rtol=1e-13)
    return n, g, f, ref


@pytest.mark.parametrize("core_svd", [1, 2])
def test_variable_coefficient_n64_fp64_direct(acr, grf64, core_svd):
    """FP64 ACR as a direct solver: within 10x the truncation tolerance, with
    the Jacobi SVD (1) or the pivoted QR (2) truncating the recompression core."""
    n, g, f, ref = grf64
    h = acr.acr_factor(n, g, 1e-6, 64, core_svd=core_svd)
    b = to_cols(f)
    x = empty_like_cols(b)
    acr.acr_solve(h, b, x)
    assert rel(from_cols(x)[:, 0], ref) < 1e-5


@pytest.mark.parametrize("tensor_cores", [0, 1])
def test_variable_coefficient_n64_fp32_refined(acr, grf64, tensor_cores):
    """FP32 ACR + FP64 refinement to 1e-10, checked with the oracle's operator;
    CUDA-core GEMMs and the tcgen05 tensor-core path (3xTF32 GEMM tiles, TMA-fed
    tiles for large products, tensor-core HODLR expansion at 64-row leaves)."""
    n, g, f, ref = grf64
    h = acr.acr_factor(n, g, 1e-6, 64, precision=acr.ACR_FP32, tensor_cores=tensor_cores)
    b = to_cols(f)
    x = empty_like_cols(b)
    it, relr, _ = acr.acr_solve_ir(h, b, x, rtol=1e-10, maxit=40)
    u = from_cols(x)[:, 0]
    assert iterative.rel_residual(n, g, u, f)[0] <= 1.01e-10
    assert rel(u, ref) < 1e-8
    # the truncation actually compresses: every block rank stays well below its size
    s = acr.acr_get_stats(h)
    m = n * n
    for row in s["max_rank"][: s["levels_cr"]]:
        for lvl, k in enumerate(row):
            assert k <= (m >> (lvl + 1)) // 2, (lvl, k, row)


@pytest.mark.parametrize("precision,restart", [("fp32", 200), ("fp64", 50)])
def test_helmholtz_n64_fgmres_ranks(acr, precision, restart):
    """Indefinite Helmholtz, 10 points per wavelength: ACR at tol 1e-4 as the
    right preconditioner of FP64 FGMRES to 1e-10 (oracle residual), with the
    ranks reported per CR level and HODLR level.  The FP32 factorisation is a
    usable preconditioner of this operator only when its recompression
    resolves the tolerance (two pivoted-Cholesky passes; with one pass,
    FGMRES stalls near 1) and with a long restart (the preconditioned spectrum
    has many outliers: FGMRES(50) stalls near 0.33, FGMRES(200) converges in
    ~100 applications); FP64 converges with 50."""
    n = 64
    w = synthetic.helmholtz_omega(n)
    f = synthetic.point_source(n, 3)
    prec = acr.ACR_FP32 if precision == "fp32" else acr.ACR_FP64
    h = acr.acr_factor(n, None, 1e-4, 64, precision=prec, shift=-w * w, tensor_cores=1, chol_passes=2)
    b = to_cols(f)
    x = empty_like_cols(b)
    it, relr, _ = acr.acr_solve_fgmres(h, b, x, rtol=1e-10, restart=restart, maxit=400)
    u = from_cols(x)[:, 0]
    assert iterative.rel_residual(n, None, u, f, shift=-w * w)[0] <= 1.01e-10
    s = acr.acr_get_stats(h)
    assert len(s["max_rank"]) == s["levels_cr"] + 1
    assert all(len(row) == s["levels_h"] for row in s["max_rank"])
    # the level-0 operator's exact cut ranks, then compressed ranks below the block size
    assert s["max_rank_d"][0] == [64, 32, 32, 16, 16, 8]
    for row in s["max_rank_d"][1:]:
        for lvl, k in enumerate(row):
            assert 0 < k <= (n * n >> (lvl + 1)) // 2, (lvl, row)
    print("helmholtz %s: %d FGMRES(%d) applications; max rank per CR level %s"
          % (precision, it, restart, [max(r) for r in s["max_rank_d"]]))


def test_fp32_residual_pass_reaches_fp64_ranks(acr, grf64):
    """A second pivoted-Cholesky pass on the explicitly formed residual lets the
    FP32 recompression resolve the tolerance: its block ranks rise from the
    FP32 Gram floor's to within 10 % of the FP64 factorisation's, and the
    refined solve still converges."""
    n, g, f, ref = grf64
    ranks = {}
    for key, kw in (("f32x1", dict(precision=acr.ACR_FP32, chol_passes=1)),
                    ("f32x2", dict(precision=acr.ACR_FP32, chol_passes=2)),
                    ("f64", dict(precision=acr.ACR_FP64))):
        h = acr.acr_factor(n, g, 1e-6, 64, tensor_cores=1, **kw)
        s = acr.acr_get_stats(h)
        ranks[key] = max(max(r) for r in s["max_rank_d"])
        if key == "f32x2":
            b = to_cols(f)
            x = empty_like_cols(b)
            it, relr, _ = acr.acr_solve_ir(h, b, x, rtol=1e-10, maxit=40)
            assert iterative.rel_residual(n, g, from_cols(x)[:, 0], f)[0] <= 1.01e-10
        h.close()
    assert ranks["f32x2"] > ranks["f32x1"]
    assert abs(ranks["f32x2"] - ranks["f64"]) <= 0.1 * ranks["f64"], ranks


def test_full_size_multi_rhs_sampled(acr):
    """n = 128, 64 RHS, FP32 ACR + FP64 refinement in the benchmark's launch
    configuration (tensor cores, autotuned tilings, graph-captured sweeps);
    three sampled columns are re-checked on the CPU with the oracle's operator."""
    import torch

    n = 128
    g = synthetic.gaussian_random_field(n, 1)
    F = synthetic.multi_rhs(n, range(100, 164))
    h = acr.acr_factor(n, torch.from_numpy(g).cuda(), 1e-6, 64, precision=acr.ACR_FP32, tensor_cores=1,
                       autotune=1, graphs=1)
    b = to_cols(F)
    x = empty_like_cols(b)
    it, relr, _ = acr.acr_solve_ir(h, b, x, rtol=1e-10, maxit=60)
    assert np.all(relr <= 1e-10)
    X = from_cols(x)
    for c in (0, 31, 63):
        assert iterative.rel_residual(n, g, X[:, c], F[:, c])[0] <= 1.01e-10
