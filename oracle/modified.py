"""Modified (subspace-enhanced) parareal for linear problems: float64 statement.
TEST INFRASTRUCTURE ONLY.

Section 3 of the paper adapts the modified parareal algorithm to matrix-valued problems:

* the Frobenius inner product <A, B>_F = tr(B^T A) and the diamond product: for block rows
  A = [A_1 .. A_p], B = [B_1 .. B_l] of n x s blocks, (A^T <> B)_ij = <A_i, B_j>_F;
* globalQR (Algorithm 2): Gram-Schmidt over the blocks Z_1 .. Z_k in <.,.>_F, in the modified
  form (each coefficient r_ji = <Q, Q_j>_F is taken from the partly reduced Q), r_ii = ||Q||_F,
  Q_i = Q / r_ii, and a block with r_ii = 0 is removed with its row and column of R, so that
  Z = Q (R kron I_s) over the kept blocks;
* the projection P_Q Y = sum_i alpha_i Q_i, alpha = Q^T <> Y, onto Span{Q_1 .. Q_l};
* Algorithm 3, for U' = B U with a linear fine propagator F and coarse propagator G: Step 0 is
  the coarse sweep of Algorithm 1; Step k+1 enlarges S^k = Span(S^{k-1} and U^k_0 .. U^k_N) by
  globalQR of [S^{k-1}, U^k_0, ..., U^k_N] (the basis of S^{k-1} is kept and completed), applies
  F to the new basis blocks only (in parallel; F(Q_i) of older blocks is kept), and updates
  sequentially U^{k+1}_{n+1} = F(P^k U^{k+1}_n) + G((I - P^k) U^{k+1}_n) with
  F(P^k U) = sum_i alpha_i F(Q_i) (F is linear);
* Algorithm 4, for affine propagators (U' = B U + C): F(0) and G(0) first (Step -1), then the
  update U_{n+1} = sum_i alpha_i (F(Q_i) - F(0)) + F(0) + G((I - P) U_n) - G(0).

Floating point (the paper states the algorithm in exact arithmetic; these readings are recorded
with the library's design notes): "r_ii = 0" becomes r_ii <= drop * ||Z_i||_F, and each block is
reduced against the current basis in `passes` sweeps of the modified Gram-Schmidt loop (two:
"twice is enough" reorthogonalisation).  The blocks U^k_n of one step are nearly dependent (for
X0 = I every iterate is a polynomial in the matrix), and one sweep leaves a basis that is far from
F-orthonormal, with which the projection is not one and the iteration stalls.  The stopping test
is Algorithm 1's: max over n = 1..N of ||U^{k+1}_n - U^k_n||_F / ||U^{k+1}_n||_F < tol.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional

import numpy as np

from . import parareal as P


def fro_inner(A: np.ndarray, B: np.ndarray) -> float:
    """<A, B>_F = tr(B^T A) (Section 3)."""
    return float(np.trace(B.T @ A))


def diamond(As: List[np.ndarray], Bs: List[np.ndarray]) -> np.ndarray:
    """A^T <> B: the p x l matrix of <A_i, B_j>_F (Section 3's definition)."""
    return np.array([[fro_inner(a, b) for b in Bs] for a in As])


def global_qr(Z: List[np.ndarray], passes: int = 1, drop: float = 0.0):
    """Algorithm 2 on the blocks Z_1 .. Z_k.  Returns (Q, R, kept): the kept F-orthonormal blocks,
    R (len(kept) x k) with Z_i = sum_j R[j, i] Q_j, and the indices of the kept blocks.  A block is
    removed when its reduced norm r_ii <= drop * ||Z_i||_F (drop = 0: only an exact zero)."""
    Q: List[np.ndarray] = []
    cols = []
    kept = []
    for i, z in enumerate(Z):
        q = z.copy()
        r = np.zeros(len(Q) + 1)
        for _ in range(passes):
            for j in range(len(Q)):
                c = fro_inner(q, Q[j])
                r[j] += c
                q = q - c * Q[j]
        rii = P.fro(q)
        if rii > drop * P.fro(z) and rii > 0.0:
            r[len(Q)] = rii
            Q.append(q / rii)
            kept.append(i)
        cols.append(r)
    R = np.zeros((len(Q), len(Z)))
    for i, r in enumerate(cols):
        R[:len(r[:len(Q)]), i] = r[:len(Q)]
    return Q, R, kept


def projection_coefficients(Q: List[np.ndarray], Y: np.ndarray) -> np.ndarray:
    """alpha = Q^T <> Y."""
    return np.array([fro_inner(Y, q) for q in Q])


def project(Q: List[np.ndarray], Y: np.ndarray) -> np.ndarray:
    """P_Q Y = sum_i alpha_i Q_i."""
    a = projection_coefficients(Q, Y)
    out = np.zeros_like(Y)
    for ai, q in zip(a, Q):
        out = out + ai * q
    return out


@dataclasses.dataclass
class ModifiedResult:
    U: List[np.ndarray]               # U^k_n, n = 0..N, of the last iteration
    iterations: int
    dx_history: List[float]
    new_blocks: List[int]             # basis blocks added (and propagated by F) per iteration
    basis: List[np.ndarray]           # the final basis Q
    all_U: Optional[List[List[np.ndarray]]] = None


def modified_parareal_generic(X0: np.ndarray, N: int, G: Callable[[np.ndarray], np.ndarray],
                              F: Callable[[np.ndarray], np.ndarray], K_max: int, tol: float,
                              drop: float, passes: int = 2, keep_all: bool = False,
                              affine: bool = False) -> ModifiedResult:
    """Algorithm 3 (affine=False) or Algorithm 4 (affine=True) with propagators G, F from one
    slice to the next (the same map for every slice: autonomous problems)."""
    F0 = F(np.zeros_like(X0)) if affine else None       # Step -1 (Algorithm 4)
    G0 = G(np.zeros_like(X0)) if affine else None
    U = [X0]
    for n in range(N):                                   # Step 0: the coarse sweep
        U.append(G(U[n]))
    all_U = [list(U)] if keep_all else None
    Q: List[np.ndarray] = []
    FQ: List[np.ndarray] = []
    hist, added = [], []
    it = 0
    for _ in range(K_max):
        # enlarge the space: globalQR of [S^{k-1}, U^k_0, ..., U^k_N]
        Qk, _, kept = global_qr(Q + U, passes=passes, drop=drop)
        new = Qk[len(Q):]
        assert kept[:len(Q)] == list(range(len(Q)))     # the old basis is kept and completed
        FQ.extend(F(q) for q in new)                    # the parallel step: new blocks only
        Q = Qk
        added.append(len(new))
        # the sequential update (eq. eq_update / update2)
        V = [X0]
        for n in range(N):
            a = projection_coefficients(Q, V[n])
            PV = np.zeros_like(X0)
            FPV = np.zeros_like(X0)
            for ai, q, fq in zip(a, Q, FQ):
                PV = PV + ai * q
                FPV = FPV + ai * (fq - F0 if affine else fq)
            if affine:
                V.append(FPV + F0 + G(V[n] - PV) - G0)
            else:
                V.append(FPV + G(V[n] - PV))
        ratios = [P.fro(V[n] - U[n]) / P.fro(V[n]) for n in range(1, N + 1)]
        dx = float(np.max(ratios))
        U = V
        it += 1
        hist.append(dx)
        if keep_all:
            all_U.append(list(U))
        if dx < tol:
            break
    return ModifiedResult(U=U, iterations=it, dx_history=hist, new_blocks=added, basis=Q,
                          all_U=all_U)


def modified_parareal(A: np.ndarray, flow: int, T: float, N: int, m: int, J: int, K_max: int,
                      tol: float, drop: float, passes: int = 2, X0: Optional[np.ndarray] = None,
                      keep_all: bool = False) -> ModifiedResult:
    """Algorithm 3 for the exponential flow dX/dt = A X (Example 2): RK4 F (J steps per slice),
    forward-Euler G (m substeps per slice), X0 = I unless given."""
    if flow != P.FLOW_EXP:
        raise ValueError("the modified parareal needs a linear flow")
    A = np.asarray(A, dtype=np.float64)
    X0 = np.eye(A.shape[0]) if X0 is None else np.asarray(X0, dtype=np.float64)
    dT = T / N
    return modified_parareal_generic(X0, N, lambda x: P.euler(flow, x, A, dT, m),
                                     lambda x: P.rk4(flow, x, A, dT, J), K_max, tol, drop,
                                     passes, keep_all)
