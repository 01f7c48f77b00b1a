"""Weak versus standard admissibility on the plane blocks ACR stores
(Section 2.1: the standard condition refines the off-diagonal blocks so that
the same per-block accuracy needs smaller ranks; Figure admisibilities and
Table flopsTable make the comparison on the H-inverse of a 2D Poisson
operator).

Test infrastructure, run as ``python -m oracle.admissibility_study`` (and
``--large`` for one n = 128 plane, ``--acr`` for (c)): for
(a) the inverse of one level-0 plane block ``D_k`` (what the first
elimination stores, ``X = D_k^{-1}``) and (b) the Schur complements
``D^(r)`` and their inverses through the reduction (dense block CR, Eq.
elim), the H-compression on the weak (HODLR) partition and on standard
partitions, each block truncated to the same per-block relative tolerance;
printed: numbers stored (MB of FP64), dense blocks, largest and mean rank;
(c) block CR with every stored block truncated on each partition
(``oracle.hacr``): the accuracy of the solve against the ranks and storage.
"""
from __future__ import annotations

import sys
import time

import numpy as np

import synthetic

from . import admissibility as adm
from .cr import cr_factor
from .operator import assemble, plane_blocks
from .ordering import cluster_tree


def _row(label, M, n, leaf, tol, etas, weak=True):
    perm, _ = cluster_tree(n, leaf)
    P = np.array(perm)
    Mp = M[np.ix_(P, P)]
    out = []
    for eta in ([None] if weak else []) + list(etas):
        levels, blocks = adm.block_partition(n, leaf, eta)
        st = adm.storage(adm.compress(Mp, levels, blocks, tol))
        out.append((label, n, leaf, tol, "weak" if eta is None else "eta=%g" % eta, st["words"] * 8 / 2 ** 20,
                    st["dense_blocks"], st["max_rank"], st["mean_rank"]))
    return out


def plane_inverse(n: int, leaf, tol: float, etas, seed: int = 1, weak_leaf=None):
    """(a): the inverse of the in-plane block of plane n/2 (GRF kappa), on
    the partitions of every leaf size in ``leaf`` (the weak partition only for
    ``weak_leaf``, default the first)."""
    g = synthetic.gaussian_random_field(n, seed)
    A = assemble(n, g).tocsr()
    m = n * n
    k = n // 2
    D = A[k * m:(k + 1) * m, k * m:(k + 1) * m].toarray()
    X = np.linalg.inv(D)
    leaves = [leaf] if isinstance(leaf, int) else list(leaf)
    wl = leaves[0] if weak_leaf is None else weak_leaf
    rows = []
    for lf in leaves:
        rows += _row("X = inv(D_k), level 0", X, n, lf, tol, etas, weak=(lf == wl))
    return rows


def reduction(n: int, leaf: int, tol: float, etas, seed: int = 1):
    """(b): D^(r) and inv(D^(r)) of the first eliminated plane of every step."""
    g = synthetic.gaussian_random_field(n, seed)
    D, E, F = plane_blocks(n, g)
    fac = cr_factor(D, E, F)
    rows = []
    for r, step in enumerate(fac.steps):
        if r == 0:
            continue  # D^(0) is the sparse operator: its admissible blocks are zero
        Dr = step["D"][0]
        rows += _row("D^(%d)" % r, Dr, n, leaf, tol, etas)
        rows += _row("inv(D^(%d))" % r, np.linalg.inv(Dr), n, leaf, tol, etas)
    return rows


def acr_accuracy(n: int, leaf: int, tol: float, etas, seed: int = 1):
    """(c): block CR with every stored block truncated on each partition
    (``oracle.hacr``): relative residual and error of one solve, ranks and
    storage of the stored blocks."""
    from .cr import cr_solve_system, join_planes, split_planes
    from .hacr import Truncator, h_cr_factor, h_cr_solve
    from .operator import apply

    g = synthetic.gaussian_random_field(n, seed)
    D, E, F = plane_blocks(n, g)
    f = synthetic.uniform_rhs(n, 0)
    ref = cr_solve_system(n, D, E, F, f)
    rows = []
    for eta in [None] + list(etas):
        T = Truncator(n, leaf, eta, tol)
        fac = h_cr_factor(D, E, F, T)
        u = join_planes(h_cr_solve(fac, split_planes(n, f)))
        res = np.linalg.norm(f - apply(n, g, u)) / np.linalg.norm(f)
        err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
        rows.append(("ACR solve, n=%d" % n, n, leaf, tol, "weak" if eta is None else "eta=%g" % eta,
                     T.words * 8 / 2 ** 20, res, err, max(T.ranks), float(np.mean(T.ranks))))
    return rows


def _print_acr(rows):
    print("| problem | leaf | tol | partition | stored MB | rel. residual | rel. error | max rank | mean rank |")
    print("|---|---:|---:|---|---:|---:|---:|---:|---:|")
    for lab, n, leaf, tol, part, mb, res, err, mx, mean in rows:
        print(f"| {lab} | {leaf} | {tol:g} | {part} | {mb:.1f} | {res:.2e} | {err:.2e} | {mx} | {mean:.1f} |")
    sys.stdout.flush()


def _print(rows):
    print("| matrix | n | leaf | tol | partition | stored MB | dense blocks | max rank | mean rank |")
    print("|---|---:|---:|---:|---|---:|---:|---:|---:|")
    for lab, n, leaf, tol, part, mb, nd, mx, mean in rows:
        print(f"| {lab} | {n} | {leaf} | {tol:g} | {part} | {mb:.2f} | {nd} | {mx} | {mean:.1f} |")
    sys.stdout.flush()


def main():
    t0 = time.time()
    etas = (1.0, 2.0)
    if "--acr" in sys.argv:
        _print_acr(acr_accuracy(16, 16, 1e-4, etas) + acr_accuracy(16, 16, 1e-6, etas) +
                   acr_accuracy(32, 32, 1e-4, etas) + acr_accuracy(32, 32, 1e-6, etas))
    elif "--large" in sys.argv:
        # the plane size of Table flopsTable's dense reference (16384^2 FP64 = 2147 MB)
        _print(plane_inverse(128, (64, 16), 1e-4, etas))
    else:
        _print(plane_inverse(32, 32, 1e-4, etas) + plane_inverse(64, 64, 1e-4, etas) +
               plane_inverse(32, 32, 1e-6, etas) + plane_inverse(64, 64, 1e-6, etas))
        _print(reduction(32, 32, 1e-6, etas))
    print("(%.0f s)" % (time.time() - t0))


if __name__ == "__main__":
    main()
