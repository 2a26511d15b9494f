"""Eigenvalue-space evaluation of the parareal iterates.  TEST INFRASTRUCTURE ONLY.

With X0 = I every map of the method is a polynomial in the symmetric matrix
A = Q diag(lam) Q^T: the inverse flow X(I-A)X, the exponential flow AX, the
square-root flow A - X^2, their RK4 stages, the Euler substeps and the
parareal correction (eq. eqStepk+1) are sums and products of such
polynomials.  So every iterate is U^k_n = Q diag(u^k_n) Q^T, where u^k_n is
the same recurrence run on the eigenvalues, and Frobenius norms of
differences are 2-norms of the eigenvalue vectors.  This gives the oracle's
result at sizes where the matrix oracle would take hours (one eigen-sized
vector recurrence plus one matrix product), exact up to rounding.

This module runs its own loops (it does not call the matrix oracle) so that
the two can pin each other.
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

FLOW_INV = 0
FLOW_EXP = 1
FLOW_SQRT = 2


def rhs(flow: int, x: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Per-eigenvalue right-hand side: x(1-lam)x, lam x, or lam - x^2."""
    if flow == FLOW_INV:
        return x * (1.0 - lam) * x
    if flow == FLOW_EXP:
        return lam * x
    if flow == FLOW_SQRT:
        return lam - x * x
    raise ValueError(flow)


def euler(flow, x, lam, dT, m):
    dt = dT / m
    for _ in range(m):
        x = x + dt * rhs(flow, x, lam)
    return x


def rk4(flow, x, lam, dT, J):
    h = dT / J
    for _ in range(J):
        k1 = rhs(flow, x, lam)
        k2 = rhs(flow, x + (h / 2) * k1, lam)
        k3 = rhs(flow, x + (h / 2) * k2, lam)
        k4 = rhs(flow, x + h * k3, lam)
        x = x + (h / 6) * (k1 + 2 * k2 + 2 * k3 + k4)
    return x


@dataclasses.dataclass
class ScalarResult:
    u: List[np.ndarray]          # u_n (eigenvalue vectors), n = 0..N
    iterations: int
    dx_history: List[float]
    dx_last_slice: List[float]


def parareal(lam: np.ndarray, flow: int, T: float, N: int, m: int, J: int, K_max: int,
             tol: float) -> ScalarResult:
    """Algorithm 1 on diag(lam) from X0 = I (same stopping rule as the matrix oracle)."""
    lam = np.asarray(lam, dtype=np.float64)
    dT = T / N
    u = [np.ones_like(lam)]
    g_old = []
    for n in range(N):
        g = euler(flow, u[n], lam, dT, m)
        g_old.append(g)
        u.append(g)
    hist, hist_last, it = [], [], 0
    for _ in range(K_max):
        f_old = [rk4(flow, u[n], lam, dT, J) for n in range(N)]
        v = [np.ones_like(lam)]
        g_new = []
        for n in range(N):
            g = euler(flow, v[n], lam, dT, m)
            g_new.append(g)
            v.append(g + (f_old[n] - g_old[n]))
        ratios = [float(np.linalg.norm(v[n] - u[n]) / np.linalg.norm(v[n])) for n in range(1, N + 1)]
        u, g_old = v, g_new
        it += 1
        hist.append(float(np.max(ratios)))
        hist_last.append(ratios[-1])
        if float(np.max(ratios)) < tol:
            break
    return ScalarResult(u=u, iterations=it, dx_history=hist, dx_last_slice=hist_last)


def sequential_fine(lam, flow, T, N, J):
    x = np.ones_like(np.asarray(lam, dtype=np.float64))
    for _ in range(N):
        x = rk4(flow, x, lam, T / N, J)
    return x


def to_matrix(Q: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Q diag(x) Q^T."""
    return (Q * x[None, :]) @ Q.T
