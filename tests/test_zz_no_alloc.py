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


def _pool_bytes():
    """(reserved, used, used high-water) of the device's default memory pool,
    which the library's allocating calls draw from, or None without libcudart."""
    import ctypes as C

    import torch

    rt = None
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            rt = C.CDLL(name)
            break
        except OSError:
            continue
    if rt is None:
        return None
    pool = C.c_void_p()
    if rt.cudaDeviceGetDefaultMemPool(C.byref(pool), torch.cuda.current_device()) != 0:
        return None
    out = []
    for attr in (5, 7, 8):  # ReservedMemCurrent, UsedMemCurrent, UsedMemHigh
        v = C.c_uint64()
        assert rt.cudaMemPoolGetAttribute(pool, attr, C.byref(v)) == 0
        out.append(v.value)
    return out, rt, pool


def test_call_allocates_no_device_memory(acr):
    """After a warm-up call, a call changes neither the free device memory, nor
    the memory pool the library allocates from (its high-water mark included),
    nor PyTorch's allocator."""
    import ctypes as C

    import torch

    n = 16
    h = acr.acr_factor(n, synthetic.gaussian_random_field(n, 7), 0.0, 32)
    F = synthetic.multi_rhs(n, range(8))
    b, x = to_cols(F), to_cols(F[:, ::-1].copy())
    r = empty_like_cols(b)
    acr.acr_residual_noalloc(h, b, x, r)  # warm-up: kernels loaded, symbol address looked up
    torch.cuda.synchronize()
    pb = _pool_bytes()
    if pb is not None:
        (_, used0, _), rt, pool = pb
        zero = C.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, 8, C.byref(zero)) == 0  # high-water mark := current use
    free0 = torch.cuda.mem_get_info()[0]
    nalloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(3):
        acr.acr_residual_noalloc(h, b, x, r)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == nalloc0
    if pb is not None:
        (res1, used1, high1), _, _ = _pool_bytes()
        # a reset high-water mark reads as the current use (or 0 until the next
        # allocation): any allocation during the calls would have raised it above
        assert used1 == used0 and high1 in (0, used0) and res1 == pb[0][0]


def test_rejects_more_rhs_than_its_scratch(acr):
    n = 4
    h = acr.acr_factor(n, None, 0.0, 4)
    F = np.ones((n ** 3, 65))
    b, x = to_cols(F), to_cols(F)
    r = empty_like_cols(b)
    with pytest.raises(acr.AcrError) as e:
        acr.acr_residual_noalloc(h, b, x, r)
    assert e.value.status == acr.ACR_ERR_ARG
