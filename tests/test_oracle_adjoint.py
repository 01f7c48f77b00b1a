"""Pin of the oracle's dense adjoint gradient: central finite differences of dense solves."""
import numpy as np

import synthetic
from oracle import adjoint


def test_gradient_matches_central_differences():
    n = 5
    g = synthetic.gaussian_random_field(n, 1)
    f = synthetic.uniform_rhs(n, 2)
    g_star = synthetic.gaussian_random_field(n, 4)
    _, u_obs = adjoint.loss(n, g_star, f, np.zeros(n ** 3))
    L, dg, df = adjoint.loss_and_grad(n, g, f, u_obs)
    rng = np.random.default_rng(0)
    for _ in range(4):
        d = rng.standard_normal(n ** 3)
        eps = 1e-5
        lp, _ = adjoint.loss(n, g + eps * d, f, u_obs)
        lm, _ = adjoint.loss(n, g - eps * d, f, u_obs)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - dg @ d) <= 1e-6 * abs(fd) + 1e-12
        e = rng.standard_normal(n ** 3)
        lp, _ = adjoint.loss(n, g, f + eps * e, u_obs)
        lm, _ = adjoint.loss(n, g, f - eps * e, u_obs)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - df @ e) <= 1e-6 * abs(fd) + 1e-12


def test_gradient_of_boundary_node_includes_boundary_faces():
    """Dropping the boundary-face term must break the pin (a planted mistake)."""
    n = 4
    g = synthetic.gaussian_random_field(n, 3)
    f = synthetic.uniform_rhs(n, 3)
    _, u_obs = adjoint.loss(n, g + 0.3, f, np.zeros(n ** 3))
    L, dg, _ = adjoint.loss_and_grad(n, g, f, u_obs)
    d = np.zeros(n ** 3)
    d[0] = 1.0  # corner node: three boundary faces
    eps = 1e-6
    lp, _ = adjoint.loss(n, g + eps * d, f, u_obs)
    lm, _ = adjoint.loss(n, g - eps * d, f, u_obs)
    fd = (lp - lm) / (2 * eps)
    assert abs(fd - dg[0]) <= 1e-5 * abs(fd)
    # the same gradient without boundary faces is measurably wrong
    import oracle.adjoint as adj
    from oracle import operator as op
    import scipy.linalg as sla
    A = op.assemble(n, g).toarray()
    u = sla.solve(A, f)
    lam = sla.solve(A.T, 2 * (u - u_obs))
    kap = np.exp(g)
    h = 1.0 / (n + 1)
    wrong = dg[0] + kap[0] * 3 * lam[0] * u[0] / (h * h)
    assert abs(fd - wrong) > 1e-3 * abs(fd)
    del adj
