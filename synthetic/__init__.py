"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds none of the solver's arithmetic: it only draws the inputs the
workloads are defined on (coefficient fields, right-hand sides, the Helmholtz
wavenumber choice) from NumPy ``PCG64`` streams, so that the CPU oracle and the
CUDA path see bit-identical inputs.

Conventions (shared with the C ABI): the unknown ``(i, j, k)`` with
``i, j, k in [0, n)`` sits at lexicographic index ``i + n*j + n*n*k``; ``k`` is
the plane (cyclic-reduction) axis.  The grid is vertex centred on the unit cube
with ``h = 1/(n+1)`` and node coordinates ``((i+1)h, (j+1)h, (k+1)h)``.

The paper (Section 2.2.1, model problem) states only the PDE and the 7-point
stencil; the workload recipes below (Gaussian random field, uniform RHS, point
source) are the benchmark's synthetic stand-ins and are not from the paper.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "grid_h",
    "node_coords_1d",
    "gaussian_random_field",
    "uniform_rhs",
    "multi_rhs",
    "point_source",
    "random_directions",
    "helmholtz_omega",
    "vortex_velocity",
]


def grid_h(n: int) -> float:
    """Mesh width of the vertex-centred grid with ``n`` interior points per axis."""
    return 1.0 / (n + 1)


def node_coords_1d(n: int) -> np.ndarray:
    """Coordinates ``(a+1)h`` of the ``n`` interior nodes along one axis."""
    return (np.arange(n, dtype=np.float64) + 1.0) * grid_h(n)


def gaussian_random_field(n: int, seed: int, length: float = 0.1, sigma: float = 1.0) -> np.ndarray:
    """Sample ``g`` on the ``n^3`` nodes with covariance ``sigma^2 exp(-|x-y|^2/(2 length^2))``.

    The squared-exponential kernel factorises over the three axes, so the
    covariance is ``K1 (x) K1 (x) K1`` and ``g = (S (x) S (x) S) z`` with ``S``
    the symmetric square root of ``K1`` (eigenvalues clamped at zero) and ``z``
    standard normal from ``PCG64(seed)``.  Returned in lexicographic order,
    float64, length ``n^3``.
    """
    x = node_coords_1d(n)
    k1 = np.exp(-((x[:, None] - x[None, :]) ** 2) / (2.0 * length * length))
    w, q = np.linalg.eigh(k1)
    w = np.clip(w, 0.0, None)
    s = (q * np.sqrt(w)[None, :]) @ q.T
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal((n, n, n))  # axes [k][j][i]
    g = np.einsum("ka,jb,ic,abc->kji", s, s, s, z, optimize=True)
    return (sigma * g).reshape(-1).astype(np.float64)


def uniform_rhs(n: int, seed: int) -> np.ndarray:
    """One right-hand side, i.i.d. uniform on [-1, 1], from ``PCG64(seed)``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=n ** 3).astype(np.float64)


def multi_rhs(n: int, seeds) -> np.ndarray:
    """Column-major ``N x nrhs`` block whose column ``c`` is ``uniform_rhs(n, seeds[c])``."""
    cols = [uniform_rhs(n, int(s)) for s in seeds]
    return np.asfortranarray(np.stack(cols, axis=1))


def point_source(n: int, seed: int) -> np.ndarray:
    """Gaussian bump ``exp(-|x-x0|^2 / (2 (2h)^2))`` with ``x0`` uniform in [0.25, 0.75]^3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x0 = rng.uniform(0.25, 0.75, size=3)
    h = grid_h(n)
    x = node_coords_1d(n)
    dk = (x - x0[2]) ** 2
    dj = (x - x0[1]) ** 2
    di = (x - x0[0]) ** 2
    r2 = dk[:, None, None] + dj[None, :, None] + di[None, None, :]
    return np.exp(-r2 / (2.0 * (2.0 * h) ** 2)).reshape(-1)


def random_directions(size: int, seeds) -> np.ndarray:
    """Unit-norm standard-normal directions, one per seed (rows)."""
    out = []
    for s in seeds:
        rng = np.random.Generator(np.random.PCG64(int(s)))
        v = rng.standard_normal(size)
        out.append(v / np.linalg.norm(v))
    return np.stack(out, axis=0)


def helmholtz_omega(n: int, points_per_wavelength: float = 10.0) -> float:
    """Wavenumber giving ``points_per_wavelength`` grid points per wavelength.

    ``2*pi / (omega*h) = ppw``  =>  ``omega = 2*pi*(n+1)/ppw``.  If ``omega^2``
    falls within a relative 1e-3 of an eigenvalue of the constant-coefficient
    7-point Laplacian (whose eigenvalues are ``(4/h^2) sum_d sin^2(pi a_d h/2)``,
    ``a_d = 1..n``), omega is raised by 0.5% until it does not, so the shifted
    operator stays safely non-singular.
    """
    h = grid_h(n)
    omega = 2.0 * np.pi * (n + 1) / points_per_wavelength
    s = (4.0 / h ** 2) * np.sin(np.pi * np.arange(1, n + 1) * h / 2.0) ** 2
    lam = (s[:, None, None] + s[None, :, None] + s[None, None, :]).reshape(-1)
    for _ in range(100):
        gap = np.min(np.abs(lam - omega ** 2)) / omega ** 2
        if gap >= 1e-3:
            break
        omega *= 1.005
    return float(omega)


def vortex_velocity(n: int, alpha: float, a: float = 1.0) -> np.ndarray:
    """Convection velocity ``alpha * b(x)`` of the convection-diffusion problem
    (Section 5, Eq. codi) at the nodes, shape ``(3, n^3)`` (planar x, y, z
    components in the node order above).  ``b`` is the paper's three-dimensional
    vortex field; its frequency ``a`` is not given in the paper (read as 1).
    """
    t = 2.0 * np.pi * a
    c = node_coords_1d(n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")  # [k][j][i]
    sx, cx = np.sin(t * x), np.cos(t * x)
    sy, cy = np.sin(t * (0.125 + y)), np.cos(t * (0.125 + y))
    sz8, cz8 = np.sin(t * (0.125 + z)), np.cos(t * (0.125 + z))
    sz, cz = np.sin(t * z), np.cos(t * z)
    bx = sx * sy + sz8 * sx
    by = cx * cy + cy * cz
    bz = cx * cz8 + sy * sz
    return alpha * np.stack([bx.ravel(), by.ravel(), bz.ravel()], axis=0)
