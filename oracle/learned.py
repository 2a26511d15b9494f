"""Learned coarse propagator: float64 statement.  TEST INFRASTRUCTURE ONLY.

The coarse propagator is a degree-4 polynomial update in the flow's Taylor terms,

    G_theta(X) = X + sum_{j=1..4} c_j dT^j X_[j],

where X_[j] is the j-th Taylor coefficient of the flow's solution through X (so
c = (1, 0, 0, 0) is the forward-Euler step of the paper's coarse propagator,
Example 1, and c = (1, 1, 1, 1) the degree-4 Taylor step), and the coefficients
c come from a small network evaluated on cheap features of the slice:

    features = [t_n / T, dT, Gershgorin lower and upper bounds of A,
                Hutchinson estimates tr(A)/n and tr(X)/n (Rademacher probes),
                ||Fl(X)||_F / sqrt(n), ||X||_F / sqrt(n)]
    network  = Linear(8, 128) - GELU - Linear(128, 128) - GELU - Linear(128, 4),
               applied to the standardised features (mean mu, deviation sd).

Training pairs are consecutive states (X_n, X_{n+1}) of fine-propagator trajectories.
With D = X_{n+1} - X_n and Z_j = dT^j X_[j] the relative residual
||sum_j c_j Z_j - D||_F^2 / ||D||_F^2 is quadratic in c, so a pair is summarised by
the Gram matrix M_ij = <Z_i, Z_j>_F, the vector b_i = <Z_i, D>_F and dd = ||D||_F^2:
loss(c) = (c^T M c - 2 c^T b + dd) / dd.  GELU is x Phi(x) (exact, erf form).
Parameters are updated with Adam.

The values the library uses are the "deployed" parameters: the weight matrices W1, W2, W3
rounded to BF16 (round to nearest even from float32), everything else float32; gradients are
taken at the deployed values and applied to the float32 master copy.  The Rademacher probes of
the Hutchinson estimates come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): output c of the stream with seed s is
mix(s + (c + 1) * 0x9E3779B97F4A7C15) (mod 2^64), and probe k, entry j is -1 when bit 63 of
output k * n + j is set and +1 otherwise.
"""
from __future__ import annotations

import math
from typing import Dict

import numpy as np

FLOW_INV, FLOW_EXP, FLOW_SQRT = 0, 1, 2
NFEAT, HID, NOUT = 8, 128, 4
NPROBES = 8
PROBE_SEED = 0x1505_07959
_M64 = (1 << 64) - 1


# --- probes and BF16 rounding ------------------------------------------------------------------

def splitmix64(seed: int, count: int) -> list:
    """The first `count` outputs of SplitMix64 seeded with `seed` (Python integers)."""
    out = []
    for c in range(count):
        z = (seed + (c + 1) * 0x9E3779B97F4A7C15) & _M64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out.append(z ^ (z >> 31))
    return out


def probes(n: int, m: int = NPROBES, seed: int = PROBE_SEED) -> np.ndarray:
    """(m, n) Rademacher probe vectors (see the module docstring)."""
    bits = splitmix64(seed, m * n)
    return np.array([-1.0 if (b >> 63) else 1.0 for b in bits]).reshape(m, n)


def bf16_round(x) -> np.ndarray:
    """float32 -> nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def deployed(p) -> Dict[str, np.ndarray]:
    """The parameter values the library computes with (module docstring)."""
    q = {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in p.items()}
    for k in ("W1", "W2", "W3"):
        q[k] = bf16_round(p[k])
    return q


# --- Taylor terms of the flows ---------------------------------------------------------------

def taylor_terms(flow: int, A: np.ndarray, X: np.ndarray, q: int = 4):
    """[X_[1], ..., X_[q]]: Taylor coefficients of the solution through X of dX/dt = Fl(X).

    inverse  Fl = X (I - A) X:  X_[j] = X (B X)^j with B = I - A (the solution is the
             Neumann series X (I - t B X)^{-1});
    exp      Fl = A X:          X_[j] = A^j X / j!;
    sqrt     Fl = A - X^2:      X_[j+1] = (delta_{j0} A - sum_{i=0..j} X_[i] X_[j-i]) / (j+1),
             X_[0] = X (Cauchy product of the series).
    """
    n = A.shape[0]
    out = []
    if flow == FLOW_INV:
        P = (np.eye(n) - A) @ X
        T = X @ P
        for _ in range(q):
            out.append(T)
            T = T @ P
    elif flow == FLOW_EXP:
        T = X
        for j in range(1, q + 1):
            T = A @ T / j
            out.append(T)
    elif flow == FLOW_SQRT:
        c = [X]
        for j in range(q):
            s = sum(c[i] @ c[j - i] for i in range(j + 1))
            c.append(((A if j == 0 else 0.0) - s) / (j + 1))
        out = c[1:]
    else:
        raise ValueError(flow)
    return out


def g_theta(flow: int, A: np.ndarray, X: np.ndarray, dT: float, c) -> np.ndarray:
    T = taylor_terms(flow, A, X, 4)
    return X + sum(c[j] * dT ** (j + 1) * T[j] for j in range(4))


# --- features ---------------------------------------------------------------------------------

def gershgorin(A: np.ndarray):
    d = np.diag(A)
    r = np.sum(np.abs(A), axis=1) - np.abs(d)
    return float(np.min(d - r)), float(np.max(d + r))


def hutchinson(X: np.ndarray, probes: np.ndarray) -> float:
    """(1/m) sum_k z_k^T X z_k for the m probe vectors in the rows of `probes`."""
    return float(np.mean([z @ X @ z for z in probes]))


def features(flow, A, X, t_over_T, dT, Z, gersh=None, trA=None) -> np.ndarray:
    """The 8 raw features of the state X at slice time t_over_T * T (Z: probe rows)."""
    n = A.shape[0]
    lo, hi = gershgorin(A) if gersh is None else gersh
    ta = hutchinson(A, Z) if trA is None else trA
    F1 = taylor_terms(flow, A, X, 1)[0]
    return np.array([t_over_T, dT, lo, hi, ta / n, hutchinson(X, Z) / n,
                     np.linalg.norm(F1) / math.sqrt(n), np.linalg.norm(X) / math.sqrt(n)])


def pair_record(flow, A, X0, X1, dT):
    """(M, b, dd) of one training pair (see the module docstring)."""
    Z = [dT ** (j + 1) * T for j, T in enumerate(taylor_terms(flow, A, X0, 4))]
    D = X1 - X0
    M = np.array([[np.sum(Zi * Zj) for Zj in Z] for Zi in Z])
    b = np.array([np.sum(Zi * D) for Zi in Z])
    return M, b, float(np.sum(D * D))


# --- the network --------------------------------------------------------------------------------

def gelu(x):
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def init_params(seed: int = 0) -> Dict[str, np.ndarray]:
    """He-style hidden layers; zero last layer with bias (1, 0, 0, 0), so the untrained
    network returns the Euler coefficients."""
    rng = np.random.default_rng(seed)
    return {
        "mu": np.zeros(NFEAT), "sd": np.ones(NFEAT),
        "W1": rng.standard_normal((HID, NFEAT)) * math.sqrt(2.0 / NFEAT), "b1": np.zeros(HID),
        "W2": rng.standard_normal((HID, HID)) * math.sqrt(2.0 / HID), "b2": np.zeros(HID),
        "W3": np.zeros((NOUT, HID)), "b3": np.array([1.0, 0.0, 0.0, 0.0]),
    }


def forward(p, x):
    """x: (B, 8) raw features -> (c (B, 4), cache)."""
    xs = (x - p["mu"]) / p["sd"]
    z1 = xs @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    c = h2 @ p["W3"].T + p["b3"]
    return c, (xs, z1, h1, z2, h2)


def loss_and_grad(p, x, M, b, dd):
    """Mean relative residual over the batch and its gradient w.r.t. W1..b3."""
    B = x.shape[0]
    c, (xs, z1, h1, z2, h2) = forward(p, x)
    Mc = np.einsum("bij,bj->bi", M, c)
    per = (np.einsum("bi,bi->b", c, Mc) - 2 * np.einsum("bi,bi->b", c, b) + dd) / dd
    dc = 2.0 * (Mc - b) / dd[:, None] / B
    g = {"W3": dc.T @ h2, "b3": dc.sum(0)}
    dh2 = dc @ p["W3"]
    dz2 = dh2 * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * gelu_grad(z1)
    g["W1"] = dz1.T @ xs
    g["b1"] = dz1.sum(0)
    return float(per.mean()), g


def adam(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on W1..b3 (state holds m, v and the step count t)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[:] = b1 * m + (1 - b1) * g[k]
        v[:] = b2 * v + (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p


# --- weight blob (the library's binary layout) ---------------------------------------------------

BLOB_ORDER = ("mu", "sd", "W1", "b1", "W2", "b2", "W3", "b3")


def to_blob(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in BLOB_ORDER]).astype(np.float32)


def from_blob(blob) -> Dict[str, np.ndarray]:
    shapes = {"mu": (NFEAT,), "sd": (NFEAT,), "W1": (HID, NFEAT), "b1": (HID,), "W2": (HID, HID),
              "b2": (HID,), "W3": (NOUT, HID), "b3": (NOUT,)}
    out, off = {}, 0
    blob = np.asarray(blob, dtype=np.float64)
    for k in BLOB_ORDER:
        sz = int(np.prod(shapes[k]))
        out[k] = blob[off:off + sz].reshape(shapes[k])
        off += sz
    return out


# --- the coarse propagator and parareal with it -------------------------------------------------

def coefficients(p, feat) -> np.ndarray:
    """c = network(features) at the deployed parameters; Euler (1, 0, 0, 0) if not finite."""
    c, _ = forward(deployed(p), np.atleast_2d(feat))
    c = c[0]
    return c if np.all(np.isfinite(c)) else np.array([1.0, 0.0, 0.0, 0.0])


def learned_G(p, flow, A, T, N, Z=None, gersh=None, trA=None):
    """G(n, X) = G_theta applied to slice n's state X (for parareal_generic)."""
    n = A.shape[0]
    Z = probes(n) if Z is None else Z
    gersh = gershgorin(A) if gersh is None else gersh
    trA = hutchinson(A, Z) if trA is None else trA
    dT = T / N

    def G(s, X):
        c = coefficients(p, features(flow, A, X, s / N, dT, Z, gersh, trA))
        return g_theta(flow, A, X, dT, c)
    return G


def parareal_learned(p, A, flow, T, N, J, K_max, tol, X0=None):
    """Algorithm 1 with the learned coarse propagator and the RK4 fine propagator."""
    from . import parareal as P
    n = A.shape[0]
    dT = T / N
    F = lambda _s, X: P.rk4(flow, X, A, dT, J)
    X0 = np.eye(n) if X0 is None else X0
    return P.parareal_generic(X0, N, learned_G(p, flow, A, T, N), F, K_max, tol)
