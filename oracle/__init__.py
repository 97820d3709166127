"""FP64 CPU oracle for the EFIE/RWG impedance matrix Z and its products.

TEST INFRASTRUCTURE ONLY.  Only the tests, the benchmark's CPU-baseline and
reference legs, and the package smoke check import this package.  It shares
no code with the GPU library (different languages, separately written
quadrature, basis and singular-integral code) and never calls it.

Modules
- ``rwg``     RWG basis list in canonical order, built from the raw mesh.
- ``efie``    ctypes driver for ``efie_oracle.c``: dense symmetric Z, selected
              rows of Z, inner potential integrals (Section II, Eqs. (1)-(5)).
- ``cm``      dense characteristic-mode eigensolve of X J = lambda R J
              (Section II, Eq. (GEP)) with R = -Re Z and X = Im Z: QZ, LU +
              Arnoldi, or (large N) the reduction to the symmetric L^T X^-1 L
              with R = L L^T; eigenvalue slopes d lambda / dk.
- ``build``   compiles ``efie_oracle.c`` with gcc + OpenMP.

Parity status: every function here is pinned by a CPU test against
closed forms, brute-force quadrature, invariants or the paper's Table I
(see tests/test_oracle_*.py); none is "parity unpinned".
"""
