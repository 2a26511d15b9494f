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
* the same Sylvester equation by matrix multiplications only (the library's form): for SPD X,
  sign([[X, R], [0, -X]]) = [[I, 2E], [0, -I]] (Roberts 1980), and the Newton-Schulz sign
  iteration S <- S (3I - S^2) / 2, started from the block matrix divided by mu >= lambda_max(X)
  / sqrt(3), keeps the block form [[P, Q], [0, -P]] with
      T = 3I - P^2,  Q <- (P Q P + T Q + Q T - 3Q) / 2,  P <- P T / 2,
  so P -> I and Q -> 2E.
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


def sylvester_sign(X: np.ndarray, R: np.ndarray, steps: int, mu: float = None):
    """E with X E + E X = R by `steps` Newton-Schulz sign steps on the block matrix (module
    docstring); mu defaults to the largest eigenvalue of the symmetrised X.  Returns (E, P)."""
    n = X.shape[0]
    if mu is None:
        mu = float(np.linalg.eigvalsh(0.5 * (X + X.T))[-1])
    P = X / mu
    Q = R / mu
    I = np.eye(n)
    for _ in range(steps):
        T = 3.0 * I - P @ P
        Q = 0.5 * (P @ Q @ P + T @ Q + Q @ T - 3.0 * Q)
        P = 0.5 * P @ T
    return 0.5 * Q, P


def newton_sign_sqrt(A: np.ndarray, X: np.ndarray, steps: int, sign_steps: int) -> np.ndarray:
    """Newton steps for X^2 = A with the Sylvester equation solved by sylvester_sign."""
    for _ in range(steps):
        R = A - X @ X
        E, _ = sylvester_sign(X, R, sign_steps)
        X = X + E
    return X
