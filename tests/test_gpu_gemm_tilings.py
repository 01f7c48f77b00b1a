"""Each GEMM tiling of the batched product, forced on every product where it is
valid (ACR_GEMM_CFG), keeps the factorisation correct: FP64 uncompressed
factorisations still solve to dense-LU accuracy (1e-12) and FP32 compressed
factorisations agree with the default tilings to FP32-level accuracy and
refine to 1e-10.  Operand ranges are checked on the host (ACR_CHECK_BOUNDS).

Tilings: 0 = 64x64 FMA tile, 8 = one warp per column slab (M <= 32), 9 / 10 /
11 = 64x64 / 64x128 / 128x64 vector-read FMA tiles."""
import numpy as np
import pytest

import synthetic
from oracle import direct, iterative

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


def _solve(acr, h, f):
    b = to_cols(f)
    x = empty_like_cols(b)
    acr.acr_solve(h, b, x)
    return from_cols(x)


@pytest.mark.parametrize("cfg", [0, 8, 9, 10, 11])
def test_forced_tiling_fp64_uncompressed(acr, monkeypatch, cfg):
    n = 16
    monkeypatch.setenv("ACR_GEMM_CFG", str(cfg))
    monkeypatch.setenv("ACR_CHECK_BOUNDS", "1")
    g = synthetic.gaussian_random_field(n, 2)
    f = synthetic.multi_rhs(n, [6, 7, 8])
    h = acr.acr_factor(n, g, 0.0, 32)
    assert rel(_solve(acr, h, f), direct.dense_solve(n, g, f)) < 1e-12


@pytest.mark.parametrize("cfg", [0, 8, 9, 10, 11])
def test_forced_tiling_fp64_uncompressed_n32(acr, monkeypatch, cfg):
    """n = 32 (dense LU out of reach on the host): the oracle's residual of the
    exact factorisation's solution, and agreement with the default tilings."""
    n = 32
    g = synthetic.gaussian_random_field(n, 2)
    f = synthetic.multi_rhs(n, [6, 7])
    monkeypatch.delenv("ACR_GEMM_CFG", raising=False)
    u0 = _solve(acr, acr.acr_factor(n, g, 0.0, 64), f)
    monkeypatch.setenv("ACR_GEMM_CFG", str(cfg))
    monkeypatch.setenv("ACR_CHECK_BOUNDS", "1")
    u = _solve(acr, acr.acr_factor(n, g, 0.0, 64), f)
    assert np.all(iterative.rel_residual(n, g, u, f) < 1e-12)
    assert rel(u, u0) < 1e-12


@pytest.mark.parametrize("cfg", [8, 9, 10, 11])
def test_forced_tiling_fp32_compressed(acr, monkeypatch, cfg):
    n = 32
    g = synthetic.gaussian_random_field(n, 3)
    f = synthetic.multi_rhs(n, [9, 10])
    monkeypatch.delenv("ACR_GEMM_CFG", raising=False)
    h0 = acr.acr_factor(n, g, 1e-6, 32, precision=acr.ACR_FP32, tensor_cores=1)
    monkeypatch.setenv("ACR_GEMM_CFG", str(cfg))
    monkeypatch.setenv("ACR_CHECK_BOUNDS", "1")
    h = acr.acr_factor(n, g, 1e-6, 32, precision=acr.ACR_FP32, tensor_cores=1)
    assert rel(acr.acr_get_factor_block(h, 0, 0, 3), acr.acr_get_factor_block(h0, 0, 0, 3)) < 1e-4
    b = to_cols(f)
    x = empty_like_cols(b)
    it, relr, _ = acr.acr_solve_ir(h, b, x, rtol=1e-10, maxit=40)
    assert max(relr) <= 1e-10
    assert np.all(iterative.rel_residual(n, g, from_cols(x), f) <= 1.01e-10)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotuned_tilings(acr, precision):
    """With autotuning every valid tiling (and its split-K variant) is timed on
    each new shape class and the fastest kept; the result is still exact
    (FP64) or refines to 1e-10 (FP32)."""
    n = 32
    g = synthetic.gaussian_random_field(n, 5)
    f = synthetic.multi_rhs(n, [11, 12])
    if precision == "fp64":
        h = acr.acr_factor(n, g, 0.0, 32, autotune=1)
        assert np.all(iterative.rel_residual(n, g, _solve(acr, h, f), f) < 1e-12)
    else:
        h = acr.acr_factor(n, g, 1e-6, 32, precision=acr.ACR_FP32, tensor_cores=1, autotune=1)
        b = to_cols(f)
        x = empty_like_cols(b)
        it, relr, _ = acr.acr_solve_ir(h, b, x, rtol=1e-10, maxit=40)
        assert max(relr) <= 1e-10


def test_autotuned_choices_match_reference_tiling_n64(acr, monkeypatch, capfd):
    """Autotuned FP32 tensor-core factorisation at n = 64 with every product
    recomputed by the reference FMA tiling (ACR_GEMM_VERIFY): no product the
    chosen tilings compute differs from it beyond FP32 accuracy.  A shape class
    of the tuning cache holds M both below and above 32 (the one-warp-per-slab
    limit), so a choice made for one member is checked on the others."""
    monkeypatch.setenv("ACR_GEMM_VERIFY", "1")
    n = 64
    g = synthetic.gaussian_random_field(n, 1)
    h = acr.acr_factor(n, g, 1e-6, 64, precision=acr.ACR_FP32, tensor_cores=1, autotune=1)
    err = capfd.readouterr().err
    assert "MISMATCH" not in err, err[:2000]
    f = synthetic.multi_rhs(n, [13])
    b = to_cols(f)
    x = empty_like_cols(b)
    it, relr, _ = acr.acr_solve_ir(h, b, x, rtol=1e-10, maxit=40)
    assert max(relr) <= 1e-10


@pytest.mark.parametrize("mode", ["0", "1", "2"])
def test_core_truncation_register_and_shared_memory_variants(acr, monkeypatch, mode):
    """FP32 pivoted-QR truncation of the blocks beyond one CTA's shared memory:
    shared-memory cluster kernel (ACR_QRCP_REG=0), register-resident cluster
    kernel (1, default; 2 also for the blocks that fit one CTA).  The ranks
    agree within one or two (pivots can differ by rounding order), the factor
    blocks to FP32 truncation accuracy, and the refined solution reaches 1e-10."""
    n = 64
    g = synthetic.gaussian_random_field(n, 1)
    monkeypatch.setenv("ACR_QRCP_REG", "0")
    h0 = acr.acr_factor(n, g, 1e-6, 64, precision=acr.ACR_FP32, tensor_cores=1)
    monkeypatch.setenv("ACR_QRCP_REG", mode)
    h = acr.acr_factor(n, g, 1e-6, 64, precision=acr.ACR_FP32, tensor_cores=1)
    r0 = np.array(acr.acr_get_stats(h0)["max_rank_d"])
    r1 = np.array(acr.acr_get_stats(h)["max_rank_d"])
    assert np.all(np.abs(r1 - r0) <= 2), (r0, r1)
    assert rel(acr.acr_get_factor_block(h, 0, 0, 3), acr.acr_get_factor_block(h0, 0, 0, 3)) < 1e-4
    f = synthetic.multi_rhs(n, [14, 15])
    b = to_cols(f)
    x = empty_like_cols(b)
    it, relr, _ = acr.acr_solve_ir(h, b, x, rtol=1e-10, maxit=40)
    assert max(relr) <= 1e-10 and it <= 12
