"""CPU oracle for parareal matrix-function evaluation.  TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, float64 statement of what the GPU library
computes, written from the paper (Chehab & Petcu, "Parallel Matrix Function
Evaluation via Initial value ODE modelling"): the matrix flows of Section 2
(Examples 1 and 2) and the steady-state framework (eq. "stat", Section 4),
classical RK4 and forward-Euler propagators, and the classical parareal
algorithm (Algorithm 1, eqs. eqStep0 and eqStepk+1).

Only the test-suite, the smoke check and the bench's CPU-baseline leg may
import it.  It shares no code with the CUDA library and imports nothing from
it; the library never imports this package.

Modules
-------
parareal   matrix oracle: flows, propagators, Algorithm 1, sequential fine solve
scalar     eigenvalue-space evaluation of the same iterates (exact when X0 = I)
closed     closed forms: A^{-1} by LU, exp(A) and A^{1/2} by eigh, scalar solutions
brute      pure-Python Fraction / Decimal re-computation for tiny cases
refine     float64 Newton-Schulz (inverse) and Newton-Sylvester (square root)
learned    learned coarse propagator: features, Taylor terms, MLP forward/backward
"""
