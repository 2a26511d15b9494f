"""Accelerated inverse-matrix approximation (Algorithm 8, Section 4): float64 statement.
TEST INFRASTRUCTURE ONLY.

Section 4 speeds up the convergence in time of dX/dt = I - A X (whose steady state is A^{-1} for,
e.g., SPD A) by adding a control u(t) to the right-hand side.  Discretised by explicit Euler with
step dt, Algorithm 8 reads:

    X^(0) = X0;  e = X~ - X^(0) with X~ an approximation of A^{-1} (from a preconditioner);
    u^(0) = e;
    repeat:  X^(k+1) = X^(k) + dt (I - A X^(k) + u^(k)),
             u^(k+1) = (I - dt A) u^(k).

`aima` returns every iterate's residual ||I - A X^(k)||_F, the quantity the paper plots against
time (its Figures for Example 5).
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np


def aima(A: np.ndarray, X0: np.ndarray, e: np.ndarray, dt: float, steps: int
         ) -> Tuple[np.ndarray, List[float]]:
    """`steps` iterations of Algorithm 8 from X0 with the initial error estimate e.  Returns
    (X^(steps), [||I - A X^(k)||_F for k = 0..steps])."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    I = np.eye(n)
    X = np.asarray(X0, dtype=np.float64).copy()
    u = np.asarray(e, dtype=np.float64).copy()
    res = [float(np.linalg.norm(I - A @ X))]
    for _ in range(steps):
        X, u = X + dt * (I - A @ X + u), u - dt * (A @ u)
        res.append(float(np.linalg.norm(I - A @ X)))
    return X, res

