"""Pins for the dense block cyclic-reduction oracle (Section 2.2, Eq. elim, Algorithms 1-2)."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import synthetic
from oracle import cr, direct, operator as op

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_schedule_matches_worked_example_n8():
    gold = json.load(open(os.path.join(GOLD, "permuted_system_n8.json")))
    steps, survivor = cr.schedule(8)
    order = steps[0]["eliminated"] + steps[0]["kept"]
    assert order == gold["order"]
    # block layout of P A P^T for a tridiagonal block pattern
    def label(r, c):
        if r == c:
            return "D%d" % r
        if c == r - 1:
            return "E%d" % r
        if c == r + 1:
            return "F%d" % r
        return ""
    layout = [[label(r, c) for c in order] for r in order]
    assert layout == gold["blocks"]
    assert steps[1]["present"] == gold["next_step_survivors"]
    assert len(steps) == gold["steps_to_single_block"]
    assert survivor == 7


@pytest.mark.parametrize("n", [2, 4, 16, 64])
def test_schedule_general(n):
    steps, survivor = cr.schedule(n)
    assert survivor == n - 1
    assert len(steps) == int(np.log2(n))
    for r, st in enumerate(steps):
        assert all(j % (2 ** r) == 2 ** r - 1 for j in st["present"])
        assert all(j % (2 ** (r + 1)) == 2 ** r - 1 for j in st["eliminated"])
        assert all(j % (2 ** (r + 1)) == 2 ** (r + 1) - 1 for j in st["kept"])


@pytest.mark.parametrize("nonsym", [False, True])
def test_scalar_cr_equals_banded_solver(nonsym):
    """Plane size 1: block CR reduces to scalar CR on a tridiagonal system
    and must agree with LAPACK's banded solver."""
    rng = np.random.default_rng(7)
    n = 32
    sub = -rng.uniform(0.5, 1.0, n)
    sup = -rng.uniform(0.5, 1.0, n) if nonsym else np.roll(sub, -1)
    dia = 2.5 + rng.uniform(0, 1, n)
    D = [np.array([[dia[k]]]) for k in range(n)]
    E = [None] + [np.array([[sub[k]]]) for k in range(1, n)]
    F = [np.array([[sup[k]]]) for k in range(n - 1)] + [None]
    f = rng.standard_normal(n)
    u = cr.cr_solve_system(1, D, E, F, f) if False else cr.join_planes(cr.cr_solve(cr.cr_factor(D, E, F), [f[k:k + 1] for k in range(n)]))
    ab = np.zeros((3, n))
    ab[0, 1:] = sup[:-1]
    ab[1] = dia
    ab[2, :-1] = sub[1:]
    ref = sla.solve_banded((1, 1), ab, f)
    np.testing.assert_allclose(u, ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("n,shift,seed", [(8, 0.0, 1), (16, 0.0, 2), (8, -400.0, 3)])
def test_dense_cr_equals_dense_lu(n, shift, seed):
    g = synthetic.gaussian_random_field(n, seed)
    f = np.stack([synthetic.uniform_rhs(n, seed + 10), synthetic.uniform_rhs(n, seed + 11)], axis=1)
    D, E, F = op.plane_blocks(n, g, shift)
    u = cr.cr_solve_system(n, D, E, F, f)
    ref = direct.dense_solve(n, g, f, shift)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-12


def test_first_step_equals_global_schur_complement():
    """Eq. elim (block form) against Eq. schur_complement evaluated on the whole permuted matrix."""
    n = 8
    m = n * n
    g = synthetic.gaussian_random_field(n, 9)
    A = op.assemble(n, g).toarray()
    D, E, F = op.plane_blocks(n, g)
    fac = cr.cr_factor(D, E, F)
    ev = [k for k in range(n) if k % 2 == 0]
    od = [k for k in range(n) if k % 2 == 1]
    ie = np.concatenate([np.arange(k * m, (k + 1) * m) for k in ev])
    io = np.concatenate([np.arange(k * m, (k + 1) * m) for k in od])
    S = A[np.ix_(io, io)] - A[np.ix_(io, ie)] @ np.linalg.solve(A[np.ix_(ie, ie)], A[np.ix_(ie, io)])
    st1 = fac.steps[1]
    for t in range(len(od)):
        blk = S[t * m:(t + 1) * m, t * m:(t + 1) * m]
        np.testing.assert_allclose(st1["D"][t], blk, rtol=1e-11, atol=1e-9 * np.abs(blk).max())
        if t > 0:
            blk = S[t * m:(t + 1) * m, (t - 1) * m:t * m]
            np.testing.assert_allclose(st1["E"][t], blk, rtol=1e-10, atol=1e-9 * np.abs(blk).max())
        if t < len(od) - 1:
            blk = S[t * m:(t + 1) * m, (t + 1) * m:(t + 2) * m]
            np.testing.assert_allclose(st1["F"][t], blk, rtol=1e-10, atol=1e-9 * np.abs(blk).max())
    # the Schur complement of a block-tridiagonal matrix is block-tridiagonal (Eq. next_step)
    far = S[0:m, 2 * m:]
    assert np.abs(far).max() < 1e-9 * np.abs(S).max()


def test_transpose_solve_nonsymmetric():
    rng = np.random.default_rng(3)
    n, m = 8, 5
    D = [np.eye(m) * 6 + rng.standard_normal((m, m)) for _ in range(n)]
    E = [None] + [rng.standard_normal((m, m)) for _ in range(n - 1)]
    F = [rng.standard_normal((m, m)) for _ in range(n - 1)] + [None]
    A = np.zeros((n * m, n * m))
    for k in range(n):
        A[k * m:(k + 1) * m, k * m:(k + 1) * m] = D[k]
        if k:
            A[k * m:(k + 1) * m, (k - 1) * m:k * m] = E[k]
        if k < n - 1:
            A[k * m:(k + 1) * m, (k + 1) * m:(k + 2) * m] = F[k]
    g = rng.standard_normal(n * m)
    Dt, Et, Ft = cr.transpose_blocks(D, E, F)
    fac = cr.cr_factor(Dt, Et, Ft)
    y = cr.join_planes(cr.cr_solve(fac, [g[k * m:(k + 1) * m] for k in range(n)]))
    np.testing.assert_allclose(A.T @ y, g, atol=1e-11)
