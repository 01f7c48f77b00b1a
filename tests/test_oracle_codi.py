"""Pins of the oracle's convection-diffusion operator (Section 5, Eq. codi):
7-point upwind differences of alpha b(x) . grad u added to -Delta u.

Each test fixes a property the paper's scheme has independently of the code:
reduction to the (already pinned) diffusion operator at zero velocity, the
M-matrix sign pattern that only upstream differencing gives, the exact action
on a quadratic (which fixes the upwind direction and the 1/h scaling), and the
truncation-error order against the paper's manufactured solution (second order
without convection, first order with it)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic
from oracle import cr
from oracle import operator as op


def test_zero_velocity_is_the_diffusion_operator():
    n = 5
    g = synthetic.gaussian_random_field(n, 3)
    zero = np.zeros((3, n ** 3))
    assert abs(op.assemble(n, g, 0.0, zero) - op.assemble(n, g)).max() == 0.0
    u = np.random.default_rng(1).standard_normal(n ** 3)
    assert np.array_equal(op.apply(n, g, u, 0.0, zero), op.apply(n, g, u))


@pytest.mark.parametrize("alpha", [1.0, 50.0])
def test_upwind_operator_is_a_nonsymmetric_m_matrix(alpha):
    n = 6
    v = synthetic.vortex_velocity(n, alpha)
    A = op.assemble(n, None, 0.0, v).toarray()
    off = A - np.diag(np.diag(A))
    assert off.max() <= 0.0  # upstream differencing never adds a positive coupling
    scale = np.abs(A).max()
    assert (A.sum(axis=1) >= -1e-12 * scale).all()  # weakly diagonally dominant rows
    assert np.abs(A - A.T).max() > 0.1 * alpha / (1.0 / (n + 1))  # convection breaks the symmetry
    u = np.random.default_rng(2).standard_normal(n ** 3)
    assert np.allclose(op.apply(n, None, u, 0.0, v), A @ u, rtol=0, atol=1e-10 * scale)


def test_upwind_direction_on_quadratic():
    """u = x^2: -Delta_h u = -2 exactly and the upstream difference of x^2 is
    2 x - sign(beta_x) h, so at nodes whose six neighbours are inside the cube
    (A u)_p = -2 + beta_x (2 x_p - sign(beta_x) h).  Downstream differencing
    would give + sign(beta_x) h instead."""
    n = 9
    h = 1.0 / (n + 1)
    v = synthetic.vortex_velocity(n, 20.0)
    c = (np.arange(n) + 1.0) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    u = (x ** 2).ravel()
    Au = op.apply(n, None, u, 0.0, v).reshape(n, n, n)
    bx = v[0].reshape(n, n, n)
    want = -2.0 + bx * (2.0 * x - np.sign(bx) * h)
    inner = (slice(1, n - 1),) * 3
    assert np.abs(Au[inner] - want[inner]).max() < 1e-9


@pytest.mark.parametrize("alpha,order", [(0.0, 4.0), (100.0, 2.0)])
def test_manufactured_truncation_error_order(alpha, order):
    """tau = A u* - f at the nodes for the paper's exact solution: halving h
    divides it by 4 without convection and by 2 with first-order upwinding."""
    taus = []
    for n in (31, 63):
        v = synthetic.vortex_velocity(n, alpha)
        us = op.codi_exact(n)
        taus.append(np.abs(op.apply(n, None, us, 0.0, v) - op.codi_rhs(n, v)).max())
    assert abs(taus[0] / taus[1] - order) < 0.1 * order


def test_manufactured_solution_converges_without_convection():
    errs = []
    for n in (7, 15):
        v = synthetic.vortex_velocity(n, 0.0)
        A = op.assemble(n, None, 0.0, v).tocsc()
        u = spla.spsolve(A, op.codi_rhs(n, v))
        errs.append(np.abs(u - op.codi_exact(n)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_block_cr_solves_the_nonsymmetric_system():
    """The oracle's dense block CR (Eq. elim and the back-substitution) on the
    upwind operator equals a sparse LU solve: CR needs no symmetry."""
    n = 8
    v = synthetic.vortex_velocity(n, 40.0)
    f = synthetic.uniform_rhs(n, 5)
    D, E, F = op.plane_blocks(n, None, 0.0, v)
    u = cr.cr_solve_system(n, D, E, F, f)
    ref = spla.spsolve(op.assemble(n, None, 0.0, v).tocsc(), f)
    assert np.linalg.norm(u - ref) <= 1e-12 * np.linalg.norm(ref)


def test_direction_pin_rejects_a_downwind_operator(monkeypatch):
    """Plant the most plausible mistake (differencing toward the downstream
    neighbour: the two upwind weights swapped) in the oracle and check that
    the quadratic test above fails for it while the real operator passes."""
    n = 9
    h = 1.0 / (n + 1)
    v = synthetic.vortex_velocity(n, 20.0)
    c = (np.arange(n) + 1.0) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    u = (x ** 2).ravel()
    bx = v[0].reshape(n, n, n)
    want = -2.0 + bx * (2.0 * x - np.sign(bx) * h)
    inner = (slice(1, n - 1),) * 3

    def miss(apply_fn):
        Au = apply_fn(n, None, u, 0.0, v).reshape(n, n, n)
        return np.abs(Au[inner] - want[inner]).max()

    assert miss(op.apply) < 1e-9
    real = op.upwind_weights

    def downwind(n_, velocity):
        dplus, wminus, wplus = real(n_, velocity)
        return dplus, wplus, wminus

    monkeypatch.setattr(op, "upwind_weights", downwind)
    assert miss(op.apply) > 1.0  # off by 2 |beta_x| h at the inner nodes
