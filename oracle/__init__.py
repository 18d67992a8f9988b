"""FP64 CPU oracle for PFASST-SH (Hamon, Schreiber, Minion 2019).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately
un-optimised statement of what the method computes, written from the paper
in float64 NumPy.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library under
``paper_1904_05988_gb300`` never does, and the two share no code.  Its
inputs come from ``synthetic`` (seeded generators without method arithmetic).

Modules
-------
``sht``     Gaussian grid, orthonormal associated Legendre functions,
            spectral synthesis/analysis (Section 3).
``swe``     Spectral SWE operators: velocity recovery, nonlinear term F_E,
            linear term F_I and the implicit solve (Sections 2, 4, 5.4).
``sdc``     Gauss-Lobatto IMEX-SDC sweep and collocation operator (Section 5.1.1).
``pfasst``  Restriction, interpolation, FAS correction, PFASST predictor and
            iteration (Sections 5.1.2, 5.2, 5.3; Algorithm 1).

Parity pins for every function live in ``tests/test_oracle_*.py``; each
module docstring lists which pin covers which function.
"""
