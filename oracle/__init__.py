"""CPU oracle for the divide-and-conquer merge step (TEST INFRASTRUCTURE).

Plain, slow, FP64 NumPy restatements of what the GPU library computes, written
from the paper (Li, Rouet, Liu, Huang, Gao, Chi, "An efficient hybrid tridiagonal
divide-and-conquer algorithm on distributed memory architectures") and from the
textbook results it relies on.  It shares no code with the CUDA path and never
imports it.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU arms of
``bench.py`` may import this package; the library itself must never route
through it.

Modules
-------
dc        Cuppen DC: tearing (Eq. 2), merge form (Eq. 3), deflation (Eq. 5),
          secular roots (Section 1), Loewner z (Remark 1), eigenvector
          assembly (Eq. 6).
sturm     Sturm-count bisection and brute-force characteristic polynomial
          roots (independent eigenvalue pins).
hss       RandHSS (Algorithm 1), HSS reconstruction and HSS x dense product
          (Eqs. 7-8).
backward  Dense reference gradient of (lambda, Q) with respect to (d, e).
metrics   Residual, orthogonality and subspace comparisons.
"""
