"""FP64 CPU oracle for the PNP-cDFT hot path (arXiv:1407.0674).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product library.  It shares no
code with the CUDA path.

Parity pins: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, analytic Fourier transforms,
brute-force sums, complex-step adjoint, exact discrete solutions, Table 1 units).
"""
