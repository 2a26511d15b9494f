"""Float64 matrix oracle: flows, propagators and classical parareal.  TEST INFRASTRUCTURE ONLY.

Everything here is a direct statement of the paper's definitions in NumPy
float64, with no blocking, fusion or reordering:

* Flows (right-hand sides Fl of dX/dt = Fl(X)):
  - inverse, Example 1 / eq. eqQ of Section 2: dQ/dt = -Q (A - I) Q = Q (I - A) Q,
    Q(0) = I, so Q(1) = A^{-1} (also the introduction's F(X) = X(Id - A)X);
  - exponential, Example 2 of Section 2: dQ/dt = A Q, Q(0) = I, Q(1) = exp(A);
  - square root, steady-state framework (eq. "stat" of the introduction and
    Section 4): dX/dt = A - X^2, X(0) = I, whose stable steady state for SPD A is
    A^{1/2}.  The paper does not print this flow; it is an instance of that
    framework (reading recorded with the library's design notes).
* Fine propagator F: J classical RK4 steps of size h = dT/J per slice (the paper
  allows "any time marching scheme", Section 1; classical RK4 is the reading).
* Coarse propagator G: m forward-Euler substeps of size dT/m per slice (the
  paper's explicit Euler propagator, Example 1).
* Parareal: Algorithm 1 (Section 2), Step 0 by eq. eqStep0 and the correction
  of Step k+1 by eq. eqStepk+1, slices T_n = n dT, dT = T/N, propagating from
  T_n to T_{n+1}.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional

import numpy as np

FLOW_INV = 0
FLOW_EXP = 1
FLOW_SQRT = 2


def rhs(flow: int, X: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Fl(X) for one flow (Section 2, Examples 1 and 2; steady-state framework)."""
    n = A.shape[0]
    if flow == FLOW_INV:
        # Example 1, eq. eqQ: dQ/dt = -Q (A - I) Q, written as Q (I - A) Q.
        return X @ (np.eye(n) - A) @ X
    if flow == FLOW_EXP:
        # Example 2: dQ/dt = A Q.
        return A @ X
    if flow == FLOW_SQRT:
        # Steady state of dX/dt = A - X^2 is A^{1/2} for SPD A.
        return A - X @ X
    raise ValueError(f"unknown flow {flow}")


def euler(flow: int, X: np.ndarray, A: np.ndarray, dT: float, m: int) -> np.ndarray:
    """Coarse propagator G over one slice: m forward-Euler substeps of size dT/m."""
    dt = dT / m
    for _ in range(m):
        X = X + dt * rhs(flow, X, A)
    return X


def rk4(flow: int, X: np.ndarray, A: np.ndarray, dT: float, J: int) -> np.ndarray:
    """Fine propagator F over one slice: J classical RK4 steps of size h = dT/J.

    Stages k1 = Fl(X), k2 = Fl(X + h/2 k1), k3 = Fl(X + h/2 k2), k4 = Fl(X + h k3);
    update X + h/6 (k1 + 2 k2 + 2 k3 + k4).
    """
    h = dT / J
    for _ in range(J):
        k1 = rhs(flow, X, A)
        k2 = rhs(flow, X + (h / 2) * k1, A)
        k3 = rhs(flow, X + (h / 2) * k2, A)
        k4 = rhs(flow, X + h * k3, A)
        X = X + (h / 6) * (k1 + 2 * k2 + 2 * k3 + k4)
    return X


def crank_nicolson(flow: int, X: np.ndarray, A: np.ndarray, dT: float, J: int) -> np.ndarray:
    """J Crank-Nicolson steps of size h = dT/J for the linear flow dX/dt = A X (the propagator
    of Section 2, Example 2): (I - h/2 A) X_{j+1} = (I + h/2 A) X_j, solved by LU per step."""
    if flow != FLOW_EXP:
        raise ValueError("Crank-Nicolson is used for the linear (exponential) flow")
    n = A.shape[0]
    h = dT / J
    Lm = np.eye(n) - (h / 2) * A
    Rm = np.eye(n) + (h / 2) * A
    for _ in range(J):
        X = np.linalg.solve(Lm, Rm @ X)
    return X


def propagator(scheme: str, flow: int, A: np.ndarray, dT: float, steps: int):
    """The one-slice map of a scheme: "rk4" (classical RK4), "euler" (explicit Euler, Example
    1's propagators) or "cn" (Crank-Nicolson, Example 2's), `steps` steps per slice."""
    if scheme == "rk4":
        return lambda x: rk4(flow, x, A, dT, steps)
    if scheme == "euler":
        return lambda x: euler(flow, x, A, dT, steps)
    if scheme == "cn":
        return lambda x: crank_nicolson(flow, x, A, dT, steps)
    raise ValueError(scheme)


def fro(X: np.ndarray) -> float:
    """Frobenius norm ||X||_F = tr(X^T X)^{1/2} (Section 3's <.,.>_F norm)."""
    return float(np.sqrt(np.sum(X * X)))


@dataclasses.dataclass
class PararealResult:
    U: List[np.ndarray]              # U^k_n, n = 0..N, of the last iteration
    iterations: int                  # fine sweeps performed after Step 0
    dx_history: List[float]          # max_n ||U^{k+1}_n - U^k_n||_F / ||U^{k+1}_n||_F
    dx_last_slice: List[float]       # the same ratio for n = N only
    all_U: Optional[List[List[np.ndarray]]] = None  # U^k for k = 0..iterations


def parareal_generic(X0: np.ndarray, N: int,
                     G: Callable[[int, np.ndarray], np.ndarray],
                     F: Callable[[int, np.ndarray], np.ndarray],
                     K_max: int, tol: float, keep_all: bool = False) -> PararealResult:
    """Algorithm 1 (classical parareal) with propagators G(n, x), F(n, x) from T_n to T_{n+1}.

    Step 0 (eq. eqStep0):     U^0_0 = X0, U^0_{n+1} = G(U^0_n).
    Step k+1 (eq. eqStepk+1): F(U^k_n) for all n (the parallel part), then
                              U^{k+1}_0 = X0,
                              U^{k+1}_{n+1} = G(U^{k+1}_n) + (F(U^k_n) - G(U^k_n)).
    G(U^k_n) is kept from the previous sweep (it was computed there), so each
    iteration evaluates G once per slice.  The loop stops after K_max fine
    sweeps, or once max_{n=1..N} ||U^{k+1}_n - U^k_n||_F / ||U^{k+1}_n||_F < tol.
    """
    U = [X0]
    G_old = []
    for n in range(N):
        g = G(n, U[n])
        G_old.append(g)
        U.append(g)
    all_U = [list(U)] if keep_all else None
    hist, hist_last = [], []
    it = 0
    for _ in range(K_max):
        F_old = [F(n, U[n]) for n in range(N)]          # parallel over n
        V = [X0]
        G_new = []
        for n in range(N):                                # sequential correction
            g = G(n, V[n])
            G_new.append(g)
            V.append(g + (F_old[n] - G_old[n]))
        ratios = [fro(V[n] - U[n]) / fro(V[n]) for n in range(1, N + 1)]
        dx = float(np.max(ratios))        # a non-finite slice makes the measure non-finite
        U, G_old = V, G_new
        it += 1
        hist.append(dx)
        hist_last.append(ratios[-1])
        if keep_all:
            all_U.append(list(U))
        if dx < tol:
            break
    return PararealResult(U=U, iterations=it, dx_history=hist, dx_last_slice=hist_last, all_U=all_U)


def parareal(A: np.ndarray, flow: int, T: float, N: int, m: int, J: int, K_max: int,
             tol: float, X0: Optional[np.ndarray] = None, keep_all: bool = False,
             coarse: str = "euler", fine: str = "rk4") -> PararealResult:
    """Parareal for one matrix flow: G = m steps of the coarse scheme (forward Euler, or
    Crank-Nicolson with coarse="cn"), F = J steps of the fine scheme ("rk4", "euler" or "cn")
    per slice.

    coarse="fine" replaces G by F (a special case in which the correction makes
    every slice exact after one iteration).
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if X0 is None:
        X0 = np.eye(n)
    dT = T / N
    f_map = propagator(fine, flow, A, dT, J)

    def F(_n, x):
        return f_map(x)

    if coarse in ("euler", "cn"):
        g_map = propagator(coarse, flow, A, dT, m)

        def G(_n, x):
            return g_map(x)
    elif coarse == "fine":
        G = F
    else:
        raise ValueError(coarse)
    return parareal_generic(np.asarray(X0, dtype=np.float64), N, G, F, K_max, tol, keep_all)


def sequential_fine(A: np.ndarray, flow: int, T: float, N: int, J: int,
                    X0: Optional[np.ndarray] = None, all_slices: bool = False, fine: str = "rk4"):
    """The sequential fine solution: F applied N times from X0 (N*J steps of the scheme)."""
    A = np.asarray(A, dtype=np.float64)
    X = np.eye(A.shape[0]) if X0 is None else np.asarray(X0, dtype=np.float64)
    dT = T / N
    f_map = propagator(fine, flow, A, dT, J)
    out = [X]
    for _ in range(N):
        X = f_map(X)
        out.append(X)
    return out if all_slices else X


def fine_sweep(A: np.ndarray, flow: int, T: float, N: int, J: int, U: List[np.ndarray]):
    """F(U_n) for n = 0..N-1: the parallel step of Algorithm 1 as one call."""
    dT = T / N
    return [rk4(flow, np.asarray(U[n], dtype=np.float64), A, dT, J) for n in range(N)]


def coarse_sweep(A: np.ndarray, flow: int, T: float, N: int, m: int, U0: np.ndarray,
                 D: Optional[List[np.ndarray]] = None):
    """Sequential part of Algorithm 1: V_0 = U0, G_n = G(V_n), V_{n+1} = G_n + D_n.

    With D = None (or all zero) this is Step 0 (eq. eqStep0); with
    D_n = F(U^k_n) - G(U^k_n) it is the correction of eq. eqStepk+1.
    Returns (V[0..N], G[0..N-1]).
    """
    dT = T / N
    V = [np.asarray(U0, dtype=np.float64)]
    Gs = []
    for n in range(N):
        g = euler(flow, V[n], A, dT, m)
        Gs.append(g)
        V.append(g if D is None else g + D[n])
    return V, Gs


def rel_fro(X: np.ndarray, Y: np.ndarray) -> float:
    """||X - Y||_F / ||Y||_F."""
    return fro(np.asarray(X) - np.asarray(Y)) / fro(np.asarray(Y))


def paper_norm(E: np.ndarray, ref: np.ndarray) -> float:
    """The error measure of Examples 1 and 2: max_ij |E_ij| / max_ij |ref_ij|."""
    return float(np.max(np.abs(E)) / np.max(np.abs(ref)))
