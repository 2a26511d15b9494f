"""Cosine (and sine) of a matrix through the block linear flow of Example 3, with Algorithm 5's
scaling and double-angle recovery: float64 statement.  TEST INFRASTRUCTURE ONLY.

Section 3, Example 3: with the homotopy A(t) = t A (X0 = 0), X(t) = sin(t A) and Y(t) = cos(t A)
satisfy dX/dt = A Y, dY/dt = -A X, i.e. dU/dt = B U (eq. eqB) with U = (X; Y) stacked (2n x n),
B = [[0, A], [-A, 0]], U(0) = (0; I), so U(1) = (sin A; cos A).

Algorithm 5 evaluates cos(A) by
  1. the smallest integer m >= 0 with 2^-m ||A||_inf <= 1,
  2. A0 = 2^-m A,
  3. C_0 = cos(A0) by the (modified) parareal algorithm on eq. eqB for A0,
  4. C_{i+1} = 2 C_i^2 - I for i = 0..m-1 (cos 2M = 2 cos^2 M - I), cos(A) = C_m.
"""
from __future__ import annotations

import math
from typing import Callable

import numpy as np

from . import modified as M
from . import parareal as P


def block_matrix(A0: np.ndarray) -> np.ndarray:
    """B = [[0, A0], [-A0, 0]] of eq. eqB."""
    n = A0.shape[0]
    Z = np.zeros((n, n))
    return np.block([[Z, A0], [-A0, Z]])


def start_state(n: int) -> np.ndarray:
    """U(0) = (X(0); Y(0)) = (sin 0; cos 0) = (0; I)."""
    return np.vstack([np.zeros((n, n)), np.eye(n)])


def scaling_exponent(A: np.ndarray) -> int:
    """Algorithm 5, step 1: the smallest m >= 0 with 2^-m ||A||_inf <= 1 (||.||_inf: the largest
    absolute row sum)."""
    a = float(np.max(np.sum(np.abs(A), axis=1)))
    m = 0
    while a > 1.0:
        a *= 0.5
        m += 1
    return m


def scheme_map(scheme: str, B: np.ndarray, dT: float, steps: int) -> Callable:
    """One slice of dU/dt = B U: `steps` explicit-Euler or classical-RK4 steps."""
    h = dT / steps

    def euler(U):
        for _ in range(steps):
            U = U + h * (B @ U)
        return U

    def rk4(U):
        for _ in range(steps):
            k1 = B @ U
            k2 = B @ (U + (h / 2) * k1)
            k3 = B @ (U + (h / 2) * k2)
            k4 = B @ (U + h * k3)
            U = U + (h / 6) * (k1 + 2 * k2 + 2 * k3 + k4)
        return U

    if scheme == "euler":
        return euler
    if scheme == "rk4":
        return rk4
    raise ValueError(scheme)


def double_angle(C0: np.ndarray, m: int) -> np.ndarray:
    """Algorithm 5, step 4: m steps of C <- 2 C^2 - I."""
    n = C0.shape[0]
    C = C0
    for _ in range(m):
        C = 2.0 * (C @ C) - np.eye(n)
    return C


def cos_algorithm5(A: np.ndarray, N: int, J: int, K_max: int, tol: float, method: str = "modified",
                   fine: str = "euler", coarse: str = "euler", m_coarse: int = 1,
                   drop: float = 1e-12):
    """cos(A) by Algorithm 5 with classical (Algorithm 1) or modified (Algorithm 3) parareal on
    eq. eqB over [0, 1].  Returns (cos A, sin(A0), m, the parareal result)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    m = scaling_exponent(A)
    A0 = A * 2.0 ** -m
    B = block_matrix(A0)
    dT = 1.0 / N
    F = scheme_map(fine, B, dT, J)
    G = scheme_map(coarse, B, dT, m_coarse)
    U0 = start_state(n)
    if method == "modified":
        r = M.modified_parareal_generic(U0, N, G, F, K_max, tol, drop)
    elif method == "classical":
        r = P.parareal_generic(U0, N, lambda _n, x: G(x), lambda _n, x: F(x), K_max, tol)
    else:
        raise ValueError(method)
    UN = r.U[N]
    S0, C0 = UN[:n], UN[n:]
    return double_angle(C0, m), S0, m, r
