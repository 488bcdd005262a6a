"""Plain FP64 CPU oracle for the spatiotemporal two-level method.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only the test suite, the smoke check and the CPU
baseline leg of the benchmark use it.  It shares no code with the CUDA path;
its only input dependency is the seeded workload description module.

Contents
  fem       exact Q1 hexahedral element matrices, global CSR assembly, laser
            and coarse box source load vectors, trilinear interpolation.
  twolevel  Algorithm 1 of the paper (macro step = predictor, m micro steps
            of the time-local problem Eq. (localProblemTime), correction by
            restriction) with a single-level backward-Euler step, patch motion
            and the powder/solid/melted state rule.

Every linear system is solved with a sparse direct solver (SciPy SuperLU)
up to 60000 unknowns and with SciPy CG to a relative residual of 1e-14
beyond that.

Pins (tests/test_oracle_*.py): element matrices against Gauss quadrature;
laser and box loads against adaptive quadrature and the erf closed form;
the closed-form discrete eigenmode decay and the second-order convergence of
the oracle's own eigenmode solutions to the continuum decay; the discrete
energy identity; the patch-covers-domain identity; the r = m = 1 identity;
brute-force dense solves on tiny meshes; patch-motion copy/interpolation
exactness; the coarse box source's total power and first moments against the
swept rectangles (track turns included); the injection set against the
coarse nodes at free fine nodes; the CG branch of the sparse solver against a
direct solve; the saw-tooth of the multirate scheme's error (Section 5.1).
"""
