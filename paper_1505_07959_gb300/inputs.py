"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module builds matrices and nothing else: it holds none of the method's
arithmetic (no flow, no time stepping, no parareal step).  Both the CUDA path
and the CPU oracle receive the arrays made here as plain inputs.

Every matrix is A = Q diag(lam) Q^T with Q Haar-random orthogonal: the QR
factorisation of an n x n standard Gaussian matrix with the signs of R's
diagonal moved into Q (so Q is Haar distributed), formed in float64 and
symmetrised as (A + A^T)/2.  The spectra follow the matrix families of the
workloads:

* inverse flow (Example 1 of the paper, dQ/dt = Q(I-A)Q): lam ~ U[0.5, 2];
* exponential flow (Example 2, dQ/dt = AQ): lam ~ U[-4, 0];
* square-root steady state (dX/dt = A - X^2): lam log-uniform in [1e-3, 1];
* inverse flow, wider spectrum: lam log-uniform in [1e-2, 1].

The 1D Laplacian of the paper's Examples 1 and 2 is generated from its
definition as well (tridiag(-1, 2, -1), optionally scaled by 1/h^2).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FLOW_INV = 0
FLOW_EXP = 1
FLOW_SQRT = 2
FLOW_NAMES = {FLOW_INV: "inv", FLOW_EXP: "exp", FLOW_SQRT: "sqrt"}


def rng_for(seed: int) -> np.random.Generator:
    """PCG64 generator for one problem; problem p of a batch uses seed base + p."""
    return np.random.default_rng(int(seed))


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-random orthogonal n x n matrix (QR of a Gaussian, R diagonal made positive)."""
    z = rng.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def spectrum(n: int, kind: str, rng: np.random.Generator) -> np.ndarray:
    """Eigenvalues for one matrix family (see the module docstring)."""
    if kind == "inv":
        return rng.uniform(0.5, 2.0, n)
    if kind == "exp":
        return rng.uniform(-4.0, 0.0, n)
    if kind == "sqrt":
        return np.exp(rng.uniform(math.log(1e-3), math.log(1.0), n))
    if kind == "inv_wide":
        return np.exp(rng.uniform(math.log(1e-2), math.log(1.0), n))
    raise ValueError(f"unknown spectrum kind {kind!r}")


@dataclasses.dataclass
class SymMatrix:
    """A symmetric test matrix with its generating eigen-decomposition."""

    A: np.ndarray      # (n, n) float64, symmetric
    Q: np.ndarray      # (n, n) float64, orthogonal
    lam: np.ndarray    # (n,) float64


def sym_matrix(n: int, kind: str, seed: int) -> SymMatrix:
    """A = Q diag(lam) Q^T, float64, symmetrised."""
    rng = rng_for(seed)
    q = haar_orthogonal(n, rng)
    lam = spectrum(n, kind, rng)
    a = (q * lam[None, :]) @ q.T
    a = 0.5 * (a + a.T)
    return SymMatrix(A=np.ascontiguousarray(a), Q=q, lam=lam)


def laplacian_1d(n: int, scaled: bool = True) -> np.ndarray:
    """tridiag(-1, 2, -1) of order n, times 1/h^2 with h = 1/(n+1) when `scaled`."""
    a = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    if scaled:
        a *= float(n + 1) ** 2
    return a


def laplacian_2d(m: int) -> np.ndarray:
    """The five-point finite-difference Laplacian on an m x m grid (order m^2): tridiag(-1, 4,
    -1) diagonal blocks coupled by -I.  Section 4, Example 5 inverts it after scaling by its
    Frobenius norm."""
    T = 4.0 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    return np.kron(np.eye(m), T) - np.kron(np.eye(m, k=1) + np.eye(m, k=-1), np.eye(m))


def aima_example(m: int = 63, threshold: float = 0.01):
    """Example 5's inputs: A = L2 / ||L2||_F (L2 the m x m grid Laplacian), X0 = 0, and the
    initial error estimate e = (A^{-1} with the entries below `threshold` times its largest
    magnitude set to zero) - X0, the thresholding of the paper's first experiment (the second uses
    e = A^{-1} exactly: threshold 0).  Returns (A, X0, e)."""
    L = laplacian_2d(m)
    A = L / np.linalg.norm(L)
    Ainv = np.linalg.inv(A)
    e = np.where(np.abs(Ainv) >= threshold * np.max(np.abs(Ainv)), Ainv, 0.0)
    return A, np.zeros_like(A), e


@dataclasses.dataclass
class Workload:
    """One parareal problem: flow, matrix family, slices and step counts."""

    name: str
    flow: int
    n: int
    kind: str
    T: float
    N: int            # time slices
    m: int            # forward-Euler substeps of the coarse propagator per slice
    J: int            # RK4 steps of the fine propagator per slice
    K_max: int        # maximum parareal iterations (fine sweeps after Step 0)
    tol: float        # stop when max_n ||U^{k+1}_n - U^k_n||_F / ||U^{k+1}_n||_F < tol
    seed: int = 0
    dtype: str = "f64"  # arithmetic of the propagators' products (fa_dtype name)
    mixed_tol: float = 0.0  # stopping tolerance used with BF16 products (0 = use tol)


# The five workloads, named by what they are.
INV_N64 = Workload("inverse flow, n=64, lam~U[0.5,2], N=8, J=16, fp64", FLOW_INV, 64, "inv",
                   1.0, 8, 1, 16, 8, 1e-10)
EXP_N2048 = Workload("exp flow, n=2048, lam~U[-4,0], N=64, J=64", FLOW_EXP, 2048, "exp",
                     1.0, 64, 1, 64, 64, 1e-10, dtype="bf16x6", mixed_tol=1e-8)
SQRT_N4096 = Workload("sqrt steady state, n=4096, lam~logU[1e-3,1], T=20, N=128, J=32",
                      FLOW_SQRT, 4096, "sqrt", 20.0, 128, 1, 32, 128, 1e-10)
INV_N1024_WIDE = Workload("inverse flow, n=1024, lam~logU[1e-2,1], N=64, J=64", FLOW_INV,
                          1024, "inv_wide", 1.0, 64, 1, 64, 64, 1e-8)


def paper_example_matrix(example: int, n: int = 80) -> np.ndarray:
    """The matrices of the paper's Section 2 examples, from the 1-D Laplacian L (order 80, scaled
    by 1/h^2, h = 1/81: the reading under which the examples' explicit propagators resolve the
    spectrum): Example 1 inverts L / 2^10, Example 2 exponentiates B = -L / 2^10."""
    a = laplacian_1d(n, scaled=True) / 2.0 ** 10
    if example == 1:
        return a
    if example == 2:
        return -a
    raise ValueError(example)


@dataclasses.dataclass
class PaperExample:
    """The paper's own parareal setups (Section 2): N slices of [0, 1], J fine steps per slice,
    the schemes of F and G, one coarse step per slice."""

    name: str
    flow: int
    example: int
    N: int = 25
    J: int = 200
    fine: str = "euler"
    coarse: str = "euler"
    T: float = 1.0


PAPER_EX1 = PaperExample("Example 1: inverse of L/2^10 (n=80), explicit Euler G and F, N=25, J=200",
                         FLOW_INV, 1)
PAPER_EX2 = PaperExample("Example 2: exp(-L/2^10) (n=80), Crank-Nicolson G and F, N=25, J=200",
                         FLOW_EXP, 2, fine="cn", coarse="cn")


def batched_problems(count: int = 512, n_lo: int = 32, n_hi: int = 512, base_seed: int = 0):
    """Mixed batch: n log-uniform in [n_lo, n_hi], flows cycling inv/exp/sqrt.

    Square-root problems integrate to T=20 with two Euler substeps per coarse
    slice (one substep of length 1.25 is unstable); the others use T=1 and one.
    Returns a list of (Workload, SymMatrix).
    """
    rng = rng_for(base_seed + 1_000_003)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count))
    out = []
    for p in range(count):
        n = int(round(ns[p]))
        flow = p % 3
        if flow == FLOW_SQRT:
            w = Workload(f"batch[{p}] sqrt n={n}", FLOW_SQRT, n, "sqrt", 20.0, 16, 2, 32, 16, 1e-6,
                         base_seed + p)
        elif flow == FLOW_EXP:
            w = Workload(f"batch[{p}] exp n={n}", FLOW_EXP, n, "exp", 1.0, 16, 1, 32, 16, 1e-6,
                         base_seed + p)
        else:
            w = Workload(f"batch[{p}] inv n={n}", FLOW_INV, n, "inv", 1.0, 16, 1, 32, 16, 1e-6,
                         base_seed + p)
        out.append((w, sym_matrix(n, w.kind, w.seed)))
    return out
