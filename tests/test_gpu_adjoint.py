"""Adjoint (acr_solve_transpose + acr_grad_logkappa behind torch.autograd):
loss ||u - u_obs||^2, gradients w.r.t. log kappa (N parameters) and f."""
import numpy as np
import pytest

import synthetic
from oracle import adjoint, iterative

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acr():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1701_00182_gb300 import build as b

    b.build()
    import paper_1701_00182_gb300 as m

    return m


def _grads(acr, n, g, f, u_obs, tol, leaf, precision, rtol):
    import torch

    gt = torch.from_numpy(g).cuda().requires_grad_(True)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    uo = torch.from_numpy(u_obs).cuda()
    u = acr.acr_solve_autograd(gt, ft, n, tol, leaf, precision, rtol)
    L = ((u - uo) ** 2).sum()
    L.backward()
    return float(L), gt.grad.cpu().numpy(), ft.grad.cpu().numpy()


@pytest.mark.parametrize("precision,tol,rtol,bar", [(0, 0.0, None, 1e-10), (1, 1e-6, 1e-12, 1e-7)])
def test_gradient_matches_dense_oracle_n16(acr, precision, tol, rtol, bar):
    n = 16
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 2)
    _, u_obs = adjoint.loss(n, synthetic.gaussian_random_field(n, 4), f, np.zeros(n ** 3))
    L_ref, dg_ref, df_ref = adjoint.loss_and_grad(n, g, f, u_obs)
    L, dg, df = _grads(acr, n, g, f, u_obs, tol, 32, precision, rtol)
    assert abs(L - L_ref) <= bar * abs(L_ref)
    assert np.linalg.norm(dg - dg_ref) <= bar * np.linalg.norm(dg_ref)
    assert np.linalg.norm(df - df_ref) <= bar * np.linalg.norm(df_ref)


def test_gradient_finite_differences_n64_twenty_directions(acr):
    """FP32 ACR + FP64 refinement (forward and adjoint) at n = 64; central
    differences along 20 seeded unit directions in log kappa, and one in f."""
    import torch

    n = 64
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 2)
    u_obs = iterative.reference_solve(n, synthetic.gaussian_random_field(n, 4), f, rtol=1e-12)
    L, dg, df = _grads(acr, n, g, f, u_obs, 1e-6, 64, acr.ACR_FP32, 1e-12)
    dirs = synthetic.random_directions(n ** 3, range(200, 220))
    eps = 1.0  # unit directions: about 2e-3 per entry of log kappa

    def loss_at(gg, ff):
        h = acr.acr_factor(n, gg, 1e-6, 64, precision=acr.ACR_FP32, nrhs_max=1)
        b = torch.from_numpy(ff).cuda()
        x = torch.zeros_like(b)
        acr.acr_solve_ir(h, b, x, rtol=1e-12, maxit=80)
        h.close()
        return float(((x.cpu().numpy() - u_obs) ** 2).sum())

    for d in dirs:
        fd = (loss_at(g + eps * d, f) - loss_at(g - eps * d, f)) / (2 * eps)
        assert abs(fd - dg @ d) <= 2e-3 * abs(fd) + 1e-9 * abs(L), (fd, dg @ d)
    e = synthetic.random_directions(n ** 3, [300])[0]
    fd = (loss_at(g, f + 1e-3 * e) - loss_at(g, f - 1e-3 * e)) / 2e-3
    assert abs(fd - df @ e) <= 1e-4 * abs(fd) + 1e-9 * abs(L)
