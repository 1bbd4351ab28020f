"""FP64 CPU oracle for the overlap operator at nonzero chemical potential.

TEST INFRASTRUCTURE.  This package is a plain, slow, obviously correct
restatement of the method of Bloch, Breu and Wettig, "Comparing iterative
methods to compute the overlap Dirac operator at nonzero chemical
potential" (Lattice 2008), written from the paper in FP64 with numpy and
scipy.  Only the test suite, the smoke check and the CPU-baseline leg of
the benchmark may import it; the product path (the CUDA library and its
Python binding) never does, and this package imports nothing from the
product path either.  The two sides share only the seeded input
generators of ``paper_0810_4228_gb300.synth``, which hold none of the
method's arithmetic.

Modules and the part of the paper each follows:

* ``wilson``    -- gamma matrices, D_w(mu), A = gamma5 D_w(mu)   (Sec. 1, Eq. 1.1-1.2)
* ``sign``      -- complex sign, spectral f(A), Roberts/Newton   (Sec. 1 Eq. 1.3-1.4, Sec. 2)
* ``krylov``    -- Arnoldi, two-sided Lanczos, LR deflation,
                   two-pass short-recurrence variant             (Secs. 2-5)
* ``deflation`` -- critical left/right eigenpairs, bi-orthonormalisation (Sec. 3, Sec. 5)
* ``freefield`` -- closed form of D_w and D_ov for U = 1 (plane waves), used as a pin
* ``frechet``   -- Frechet derivative of sgn via the block upper-triangular form

Equation numbers are (section.n), counting the displayed, numbered
equations of each section in order of appearance.

Parity status: every function listed here is pinned by the ``-m "not gpu"``
tests in ``tests/test_oracle_*.py`` against closed forms, invariants,
special cases and brute force; none is "parity unpinned".
"""
