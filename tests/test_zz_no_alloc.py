"""acr_residual_noalloc, the allocation-free residual entry point, against
acr_residual (which takes its reduction scratch from the allocator): the same
residual and relative norms on two calls in a row, and a clear rejection of
requests larger than its fixed scratch.  Runs last so that a failure here
leaves every other test already run."""
import numpy as np
import pytest

import synthetic

from gpu_util import empty_like_cols, from_cols, to_cols

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acr():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1701_00182_gb300 import build as b

    b.build()
    import paper_1701_00182_gb300 as m

    return m


def test_matches_allocating_residual_on_two_calls(acr):
    n = 16
    g = synthetic.gaussian_random_field(n, 7)
    h = acr.acr_factor(n, g, 0.0, 32)
    rng = np.random.default_rng(3)
    for call, nrhs in enumerate((3, 64)):
        F = synthetic.multi_rhs(n, range(10 * call, 10 * call + nrhs))
        U = rng.standard_normal(F.shape)
        b, x = to_cols(F, ld_pad=call), to_cols(U, ld_pad=call)
        r_ref = empty_like_cols(b)
        r_new = empty_like_cols(b)
        rel_ref = acr.acr_residual(h, b, x, r_ref)
        rel_new = acr.acr_residual_noalloc(h, b, x, r_new)
        a, c = from_cols(r_new), from_cols(r_ref)
        assert np.max(np.abs(a - c)) <= 1e-12 * np.max(np.abs(c))
        np.testing.assert_allclose(rel_new, rel_ref, rtol=1e-12)


def test_rejects_more_rhs_than_its_scratch(acr):
    n = 4
    h = acr.acr_factor(n, None, 0.0, 4)
    F = np.ones((n ** 3, 65))
    b, x = to_cols(F), to_cols(F)
    r = empty_like_cols(b)
    with pytest.raises(acr.AcrError) as e:
        acr.acr_residual_noalloc(h, b, x, r)
    assert e.value.status == acr.ACR_ERR_ARG
