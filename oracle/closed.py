"""Closed forms the flows converge to.  TEST INFRASTRUCTURE ONLY.

* A^{-1} by LU (numpy.linalg.solve): the end state Q(1) of Example 1.
* exp(A) and A^{1/2} of a symmetric A by its eigendecomposition (numpy.linalg.eigh):
  the end state of Example 2 and the steady state of dX/dt = A - X^2.
* The scalar solutions of the three flows on one eigenvalue lam, from x(0) = 1:
  - inverse:     x(t) = 1 / (1 + t (lam - 1))     (the homotopy path of eq. eqAt with X0 = I)
  - exponential: x(t) = exp(lam t)
  - square root: with s = sqrt(lam), x(t) = s (1 + s tanh(s t)) / (s + tanh(s t)),
    which solves x' = lam - x^2, x(0) = 1 and tends to s.
"""
from __future__ import annotations

import numpy as np


def inv_lu(A: np.ndarray) -> np.ndarray:
    return np.linalg.solve(A, np.eye(A.shape[0]))


def sym_fun(A: np.ndarray, f) -> np.ndarray:
    mu, V = np.linalg.eigh(0.5 * (A + A.T))
    return (V * f(mu)[None, :]) @ V.T


def expm_sym(A: np.ndarray) -> np.ndarray:
    return sym_fun(A, np.exp)


def sqrtm_spd(A: np.ndarray) -> np.ndarray:
    return sym_fun(A, np.sqrt)


def scalar_solution(flow: int, lam: np.ndarray, t: float) -> np.ndarray:
    lam = np.asarray(lam, dtype=np.float64)
    if flow == 0:
        return 1.0 / (1.0 + t * (lam - 1.0))
    if flow == 1:
        return np.exp(lam * t)
    if flow == 2:
        s = np.sqrt(lam)
        th = np.tanh(s * t)
        return s * (1.0 + s * th) / (s + th)
    raise ValueError(flow)
