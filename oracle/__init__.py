"""FP64 CPU oracle for the split exponential Euler method (Caliari & Cassini).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with the CUDA library (no kernels, headers, tables, constants
or pre/post-processing); the two meet only through the seeded input
generators, which hold none of the method's arithmetic.

What it computes, in plain numpy/scipy FP64 and in the paper's order:

* ``axes``      -- the one-dimensional grids and finite-difference matrices of
                   Section 3 (eqs. A_theta, disk_discr, ball_discr, syscn/A_phi,
                   A_z) plus the Neumann-caps reading of A_z.
* ``operators`` -- the Kronecker-sum semidiscretisations of Section 2
                   (eqs. disk, sphere, ball, cylinder), assembled sparse.
* ``phi``       -- the scalar phi_1 of Section 4 and phi_1 of a 1-D matrix by
                   the symmetrisation of Proposition 1 and an eigen-solve.
* ``reactions`` -- the reaction terms of the workloads.
* ``stepper``   -- one split exponential Euler step (eq. ee with the split
                   approximation eq. splitorder), applying phi_1(tau d M_mu)
                   fibre by fibre with the highest mode first.
* ``unsplit``   -- unsplit exponential Euler (eq. ee with phi_1 of the whole
                   assembled operator, dense expm): the baseline the splitting
                   error is measured against.
* ``coupled``   -- the bulk-surface Schnakenberg system of Section 5.5 (ball
                   and its boundary sphere coupled through Robin boundary
                   conditions and the surface reactions).
* ``coupled_dib`` -- the bulk-surface DIB model of Section 5.6 (cylinder with a
                   Dirichlet top and its bottom disk, coupled through flux
                   conditions and the surface kinetics p, q).
* ``adjoint``   -- gradients of a scalar loss by complex-step differentiation
                   through ``stepper`` (no transposed code path of its own).

Every function that is pinned by the tests says by what; "parity unpinned"
marks the ones no test fixes independently of the oracle itself.
"""
