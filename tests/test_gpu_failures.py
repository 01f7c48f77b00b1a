"""Failure paths of the C ABI, made on the host side: every call returns its
status code, no kernel traps, and the process (and, for solve-side failures,
the handle) stays usable -- the next call on it succeeds and still matches the
oracle."""
import numpy as np
import pytest

import synthetic
from oracle import direct

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


def _still_works(acr):
    """A fresh exact factorisation after the failure still matches dense LU."""
    n = 8
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 0)
    h = acr.acr_factor(n, g, 0.0, 8)
    b = to_cols(f)
    x = empty_like_cols(b)
    acr.acr_solve(h, b, x)
    assert rel(from_cols(x)[:, 0], direct.dense_solve(n, g, f)) < 1e-12
    h.close()


def _status(acr, fn):
    with pytest.raises(acr.AcrError) as e:
        fn()
    return e.value.status


def test_rank_cap(acr):
    g = synthetic.gaussian_random_field(16, 1)
    st = _status(acr, lambda: acr.acr_factor(16, g, 1e-6, 16, max_rank=1))
    assert st == acr.ACR_ERR_RANK_CAP
    _still_works(acr)


def test_device_allocation_failure_is_oom(acr):
    """A solve workspace far beyond the device's memory: the allocation fails,
    acr_factor returns ACR_ERR_OOM and frees what it had."""
    g = synthetic.gaussian_random_field(64, 1)
    st = _status(acr, lambda: acr.acr_factor(64, g, 1e-6, 64, precision=acr.ACR_FP32, nrhs_max=1 << 22))
    assert st == acr.ACR_ERR_OOM
    _still_works(acr)


def test_tiny_memory_budget_recomputes_everything(acr):
    """A budget too small for any level keeps nothing: every solve call
    re-assembles from kappa and recomputes all levels, with the same result."""
    n = 16
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 0)
    h0 = acr.acr_factor(n, g, 1e-6, 16)
    h1 = acr.acr_factor(n, g, 1e-6, 16, mem_budget=1 << 10)
    s = acr.acr_get_stats(h1)
    assert s["levels_stored"] == 0 and s["factor_bytes"] == 0
    b = to_cols(f)
    x0, x1 = empty_like_cols(b), empty_like_cols(b)
    acr.acr_solve(h0, b, x0)
    acr.acr_solve(h1, b, x1)
    acr.acr_solve_transpose(h1, b, x1)
    acr.acr_solve(h1, b, x1)
    np.testing.assert_array_equal(from_cols(x1), from_cols(x0))
    assert acr.acr_get_stats(h1)["tail_recomputes"] == 3
    _still_works(acr)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf, 800.0])
def test_non_finite_log_kappa(acr, bad):
    """NaN / infinite log kappa, or one whose exponential overflows, is an
    argument error (no NaN solution)."""
    g = synthetic.gaussian_random_field(8, 1)
    g[37] = bad
    st = _status(acr, lambda: acr.acr_factor(8, g, 0.0, 8))
    assert st == acr.ACR_ERR_ARG
    _still_works(acr)


def test_non_finite_velocity(acr):
    n = 8
    v = np.zeros(3 * n ** 3)
    v[5] = np.nan
    st = _status(acr, lambda: acr.acr_factor(n, None, 0.0, 8, velocity=v))
    assert st == acr.ACR_ERR_ARG
    _still_works(acr)


def test_singular_leaf_is_breakdown(acr):
    """n = 2, kappa = 1: every plane block is 54 I - 9 (4-cycle adjacency) with
    eigenvalues 36, 54, 54, 72 (h = 1/3), so the shift -36 makes the
    eliminated plane's single leaf exactly singular: the Gauss-Jordan kernel
    records the zero pivot in a device flag and acr_factor returns
    ACR_ERR_BREAKDOWN."""
    st = _status(acr, lambda: acr.acr_factor(2, None, 0.0, 4, shift=-36.0))
    assert st == acr.ACR_ERR_BREAKDOWN
    _still_works(acr)


def test_refinement_not_converged_then_handle_reused(acr):
    n = 16
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 0)
    h = acr.acr_factor(n, g, 1e-3, 16, precision=acr.ACR_FP32)
    b = to_cols(f)
    x = empty_like_cols(b)
    it, relr, st = acr.acr_solve_ir(h, b, x, rtol=1e-10, maxit=1, check=False)
    assert st == acr.ACR_ERR_NOT_CONVERGED and it == 1 and relr[0] > 1e-10 and np.isfinite(relr[0])
    it, relr, st = acr.acr_solve_fgmres(h, b, x, rtol=1e-10, restart=5, maxit=2, check=False)
    assert st == acr.ACR_ERR_NOT_CONVERGED and it == 2
    # the same handle then converges
    it, relr, st = acr.acr_solve_ir(h, b, x, rtol=1e-10, maxit=60)
    assert st == acr.ACR_OK and relr[0] <= 1e-10
    assert rel(from_cols(x)[:, 0], direct.dense_solve(n, g, f)) < 1e-8


def test_bad_arguments(acr):
    g = synthetic.gaussian_random_field(8, 1)
    assert _status(acr, lambda: acr.acr_factor(6, None, 0.0, 4)) == acr.ACR_ERR_ARG   # n not a power of two
    assert _status(acr, lambda: acr.acr_factor(8, g, -1.0, 8)) == acr.ACR_ERR_ARG     # negative tolerance
    assert _status(acr, lambda: acr.acr_factor(8, g, 0.0, 3)) == acr.ACR_ERR_ARG      # leaf
    h = acr.acr_factor(8, g, 0.0, 8)
    b = to_cols(synthetic.uniform_rhs(8, 0))
    # refinement needs separate b and x
    it, relr, st = acr.acr_solve_ir(h, b, b, check=False)
    assert st == acr.ACR_ERR_ARG
    _still_works(acr)
