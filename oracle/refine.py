"""Float64 refinement of a low-precision end state.  TEST INFRASTRUCTURE ONLY.

The paper integrates in one precision; these refinement steps belong to the
mixed-precision form of the library and are standard Newton iterations:

* inverse: the Newton-Schulz (Hotelling) iteration X <- X (2I - A X), the
  Newton step for X^{-1} - A = 0; it doubles the number of correct digits per
  step while ||I - A X|| < 1.
* square root: the full Newton step for X^2 - A = 0, i.e. solve the Sylvester
  equation X E + E X = A - X^2 and set X <- X + E.  The Sylvester equation is
  solved in the eigenbasis of the symmetrised iterate X = V diag(mu) V^T:
  E = V [ (V^T R V)_ij / (mu_i + mu_j) ] V^T with R = A - X^2.
"""
from __future__ import annotations

import numpy as np


def newton_schulz_inv(A: np.ndarray, X: np.ndarray, steps: int) -> np.ndarray:
    n = A.shape[0]
    for _ in range(steps):
        X = X @ (2.0 * np.eye(n) - A @ X)
    return X


def newton_sylvester_sqrt(A: np.ndarray, X: np.ndarray, steps: int) -> np.ndarray:
    for _ in range(steps):
        Xs = 0.5 * (X + X.T)
        mu, V = np.linalg.eigh(Xs)
        R = A - Xs @ Xs
        Rt = V.T @ R @ V
        Et = Rt / (mu[:, None] + mu[None, :])
        X = Xs + V @ Et @ V.T
    return X
