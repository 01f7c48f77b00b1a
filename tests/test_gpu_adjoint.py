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


def _grads(acr, n, g, f, u_obs, tol, leaf, precision, rtol, mem_budget=0):
    import torch

    gt = torch.from_numpy(g).cuda().requires_grad_(True)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    uo = torch.from_numpy(u_obs).cuda()
    u = acr.acr_solve_autograd(gt, ft, n, tol, leaf, precision, rtol, mem_budget=mem_budget)
    L = ((u - uo) ** 2).sum()
    L.backward()
    return float(L.detach()), gt.grad.cpu().numpy(), ft.grad.cpu().numpy()


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


def _store_bytes(acr, n, g, tol, leaf, precision):
    h = acr.acr_factor(n, g, tol, leaf, precision=precision, nrhs_max=1)
    s = acr.acr_get_stats(h)
    h.close()
    return s["factor_bytes"], s["levels_cr"]


@pytest.mark.parametrize("frac", [0.5, 0.0])
def test_budgeted_store_gradient_matches_dense_oracle_n16(acr, frac):
    """With a memory budget below the full factor store (half of it, or none:
    every level recomputed from kappa) the levels that do not fit are
    recomputed for the forward and the backward solve, and the gradient still
    matches the dense oracle."""
    n = 16
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 2)
    _, u_obs = adjoint.loss(n, synthetic.gaussian_random_field(n, 4), f, np.zeros(n ** 3))
    L_ref, dg_ref, df_ref = adjoint.loss_and_grad(n, g, f, u_obs)
    full, q = _store_bytes(acr, n, g, 0.0, 32, acr.ACR_FP64)
    budget = max(1, int(frac * full))
    h = acr.acr_factor(n, g, 0.0, 32, mem_budget=budget, nrhs_max=1)
    s = acr.acr_get_stats(h)
    assert s["levels_cr"] == q and s["levels_stored"] < q
    assert s["factor_bytes"] <= budget or s["levels_stored"] == 0
    h.close()
    L, dg, df = _grads(acr, n, g, f, u_obs, 0.0, 32, acr.ACR_FP64, None, mem_budget=budget)
    assert abs(L - L_ref) <= 1e-10 * abs(L_ref)
    assert np.linalg.norm(dg - dg_ref) <= 1e-10 * np.linalg.norm(dg_ref)
    assert np.linalg.norm(df - df_ref) <= 1e-10 * np.linalg.norm(df_ref)


def test_budgeted_store_gradient_equals_unbudgeted_n64(acr):
    """n = 64, FP64 ACR at tol 1e-6: a budget of 60 % of the full store keeps
    the first CR levels and recomputes the rest (once per solve call); the
    recomputed factors are the same arithmetic on the same inputs, so the
    gradient equals the unbudgeted one to 1e-12."""
    n = 64
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 2)
    u_obs = iterative.reference_solve(n, synthetic.gaussian_random_field(n, 4), f, rtol=1e-12)
    full, q = _store_bytes(acr, n, g, 1e-6, 64, acr.ACR_FP64)
    budget = int(0.6 * full)
    h = acr.acr_factor(n, g, 1e-6, 64, mem_budget=budget, nrhs_max=1)
    s = acr.acr_get_stats(h)
    assert 0 < s["levels_stored"] < q and s["factor_bytes"] <= budget
    h.close()
    L0, dg0, df0 = _grads(acr, n, g, f, u_obs, 1e-6, 64, acr.ACR_FP64, None)
    L1, dg1, df1 = _grads(acr, n, g, f, u_obs, 1e-6, 64, acr.ACR_FP64, None, mem_budget=budget)
    assert abs(L1 - L0) <= 1e-12 * abs(L0)
    assert np.linalg.norm(dg1 - dg0) <= 1e-12 * np.linalg.norm(dg0)
    assert np.linalg.norm(df1 - df0) <= 1e-12 * np.linalg.norm(df0)
