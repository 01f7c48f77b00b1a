"""Checks of the seeded input generators (not the solver)."""
import numpy as np

import synthetic


def test_reproducible():
    np.testing.assert_array_equal(synthetic.gaussian_random_field(8, 1), synthetic.gaussian_random_field(8, 1))
    assert not np.array_equal(synthetic.uniform_rhs(8, 1), synthetic.uniform_rhs(8, 2))


def test_grf_pointwise_variance():
    vals = np.stack([synthetic.gaussian_random_field(12, s) for s in range(40)])
    assert abs(vals.mean()) < 0.1
    assert 0.8 < vals.var() < 1.2


def test_rhs_range_and_layout():
    b = synthetic.multi_rhs(4, [5, 6, 7])
    assert b.shape == (64, 3) and b.flags.f_contiguous
    assert b.min() >= -1 and b.max() <= 1
    np.testing.assert_array_equal(b[:, 1], synthetic.uniform_rhs(4, 6))


def test_helmholtz_points_per_wavelength():
    n = 64
    w = synthetic.helmholtz_omega(n)
    ppw = 2 * np.pi / (w / (n + 1))
    assert 9.5 < ppw <= 10.0


def test_vortex_velocity_is_divergence_free():
    """The vortex field of Eq. codi is solenoidal: its six cross terms cancel in
    pairs, and on the node grid the central-difference divergence cancels to
    rounding (each component is a product of per-axis factors).  A changed sign,
    phase or factor in any component breaks the cancellation."""
    n = 31
    h = synthetic.grid_h(n)
    v = synthetic.vortex_velocity(n, 1.0).reshape(3, n, n, n)  # [component][k][j][i]
    div = (
        (v[0][1:-1, 1:-1, 2:] - v[0][1:-1, 1:-1, :-2])
        + (v[1][1:-1, 2:, 1:-1] - v[1][1:-1, :-2, 1:-1])
        + (v[2][2:, 1:-1, 1:-1] - v[2][:-2, 1:-1, 1:-1])
    ) / (2 * h)
    assert np.abs(div).max() < 1e-11 * np.abs(v).max() / h
    assert np.abs(v).max() > 1.0  # and the field is not trivially zero
    assert np.allclose(synthetic.vortex_velocity(n, 7.0), 7.0 * synthetic.vortex_velocity(n, 1.0))
