"""CPU FP64 oracle for the accelerated-cyclic-reduction hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA product path never calls it and shares no code with it; the
two meet only through the seeded generators in ``synthetic``.

What it computes (each module cites the passage it follows):

* ``operator``  -- the 7-point discretisation of -div(kappa grad u) (+ shift u)
  as a sparse matrix and as block-tridiagonal plane blocks (Section 2.2.1,
  Eq. probSta / Eq. originalMatrix); optionally plus the first-order upwind
  convection term of the convection-diffusion problem (Section 5, Eq. codi),
  with its manufactured solution and right-hand side.
* ``direct``    -- the exact solution by dense LU and, for constant kappa, by
  the discrete-sine-transform closed form (the FFT route of FACR, Section 1).
* ``cr``        -- plain dense block cyclic reduction: the red/black schedule
  (Eq. permuted_system, Eq. next_step), the block Schur-complement updates of
  Eq. elim, the coarsest solve (Eq. first_backSubs) and back-substitution
  (Eq. all_backSubs, Algorithm 2); plus the transpose solve.
* ``ordering``  -- the 2D planar bisection cluster tree of one plane and the
  grid edges each bisection cuts (Section 3.1, Section 2.1.1).
* ``iterative`` -- FP64 conjugate gradients / GMRES on the sparse operator,
  the refinement reference at sizes where dense CR does not fit.
* ``adjoint``   -- the loss of the inverse problem and its gradient with respect
  to log kappa and f by dense solves (the reference of the adjoint kernels).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against dense LU, closed forms, the paper's n=8 worked example, the Thomas
algorithm, library routines, finite differences (adjoint) and, for the upwind
operator, its M-matrix structure, exact action on a quadratic and truncation
orders.  No function is "parity unpinned".
"""
