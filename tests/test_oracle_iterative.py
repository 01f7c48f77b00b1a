"""Pins for the FP64 Krylov references against the DST closed form."""
import numpy as np

import synthetic
from oracle import direct, iterative, operator as op


def test_cg_matches_dst():
    n = 16
    f = synthetic.uniform_rhs(n, 0)
    u, it = iterative.cg(op.assemble(n, None), f, rtol=1e-13)
    ref = direct.dst_solve(n, f)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-11
    assert iterative.rel_residual(n, None, u, f)[0] < 1e-12


def test_gmres_indefinite_matches_dst():
    n = 8
    w = synthetic.helmholtz_omega(n)
    f = synthetic.point_source(n, 3)
    u = iterative.reference_solve(n, None, f, shift=-w * w, rtol=1e-13)
    ref = direct.dst_solve(n, f, shift=-w * w)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-9
