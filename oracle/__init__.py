"""FP64 CPU oracle of the cavity fractional-step method (TEST INFRASTRUCTURE).

This package is the plain, slow, obviously correct statement of what the CUDA
path computes, used only to check it.  Only the test suite, the smoke check
and the benchmark's CPU-baseline leg may import it; the product path
(``paper_2504_03697_gb300``) never does, and the oracle never imports the
product.  The two share no code: the only common module is the seeded input
generator (``paper_2504_03697_gb300.synthetic``), which the tests call and
whose outputs are handed to both sides as plain arrays.

Layout of the oracle, in the order the paper's time step runs (Sec. 3.1):

* ``mac``             staggered (MAC) grid, wall/ghost rules, index helpers
* ``operators``       explicit CSR assembly of the pressure Poisson matrix and
                      the implicit-diffusion matrices (Sec. 3.1, "CSR")
* ``krylov``          textbook preconditioned conjugate gradients with the
                      identity, Jacobi and DIC preconditioners (Sec. 3.1)
* ``fractional_step`` applyForces, semi-Lagrangian advection, implicit
                      diffusion, divergence, pressure solve, pressure
                      correction, and the whole step (Sec. 3.1, Table 1)

Every array is float64, shaped (z, y, x) with x fastest.  Parity status of
each function is stated in its module header; every function here is pinned
by a test in ``tests/test_oracle_*.py`` against closed forms, invariants or
brute force, except where a header says "parity unpinned".
"""
