"""Pure-Python re-computation of Algorithm 1 in exact or 50-digit arithmetic.  TEST INFRASTRUCTURE ONLY.

Matrices are lists of lists over any number type with + - * (fractions.Fraction
for exact rational arithmetic, decimal.Decimal at high precision).  Every
coefficient of RK4 (1/2, 1/6, 2), of forward Euler and of the parareal
correction is rational, so on rational inputs the whole algorithm is exact in
Fraction arithmetic.  The loops are written out independently of the NumPy
oracle, element by element, so that a transposed operand, a wrong stage
weight or a dropped term in either would show up as a disagreement.
"""
from __future__ import annotations

from decimal import Decimal, localcontext
from fractions import Fraction


def mat(rows):
    return [list(r) for r in rows]


def eye(n, one, zero):
    return [[one if i == j else zero for j in range(n)] for i in range(n)]


def mm(X, Y, zero):
    n, p, q = len(X), len(Y), len(Y[0])
    out = [[zero] * q for _ in range(n)]
    for i in range(n):
        for j in range(q):
            s = zero
            for k in range(p):
                s = s + X[i][k] * Y[k][j]
            out[i][j] = s
    return out


def add(X, Y):
    return [[a + b for a, b in zip(r, s)] for r, s in zip(X, Y)]


def sub(X, Y):
    return [[a - b for a, b in zip(r, s)] for r, s in zip(X, Y)]


def scale(c, X):
    return [[c * a for a in r] for r in X]


def rhs(flow, X, A, one, zero):
    n = len(A)
    if flow == 0:   # X (I - A) X
        return mm(mm(X, sub(eye(n, one, zero), A), zero), X, zero)
    if flow == 1:   # A X
        return mm(A, X, zero)
    if flow == 2:   # A - X X
        return sub(A, mm(X, X, zero))
    raise ValueError(flow)


def euler(flow, X, A, dT, m, one, zero):
    dt = dT / m
    for _ in range(m):
        X = add(X, scale(dt, rhs(flow, X, A, one, zero)))
    return X


def rk4(flow, X, A, dT, J, one, zero):
    h = dT / J
    two = one + one
    six = two + two + two
    for _ in range(J):
        k1 = rhs(flow, X, A, one, zero)
        k2 = rhs(flow, add(X, scale(h / two, k1)), A, one, zero)
        k3 = rhs(flow, add(X, scale(h / two, k2)), A, one, zero)
        k4 = rhs(flow, add(X, scale(h, k3)), A, one, zero)
        s = add(add(k1, scale(two, k2)), add(scale(two, k3), k4))
        X = add(X, scale(h / six, s))
    return X


def parareal(A, flow, T, N, m, J, K, one, zero):
    """K iterations of Algorithm 1 (no early stop); returns [U^k_n for n] for k = 0..K."""
    n = len(A)
    dT = T / N
    X0 = eye(n, one, zero)
    U = [X0]
    G_old = []
    for s in range(N):
        g = euler(flow, U[s], A, dT, m, one, zero)
        G_old.append(g)
        U.append(g)
    history = [U]
    for _ in range(K):
        F_old = [rk4(flow, U[s], A, dT, J, one, zero) for s in range(N)]
        V = [X0]
        G_new = []
        for s in range(N):
            g = euler(flow, V[s], A, dT, m, one, zero)
            G_new.append(g)
            V.append(add(g, sub(F_old[s], G_old[s])))
        U, G_old = V, G_new
        history.append(U)
    return history


def parareal_fraction(A_rows, flow, T, N, m, J, K):
    A = [[Fraction(x) for x in r] for r in A_rows]
    return parareal(A, flow, Fraction(T), N, m, J, K, Fraction(1), Fraction(0))


def parareal_decimal(A_rows, flow, T, N, m, J, K, digits=50):
    with localcontext() as ctx:
        ctx.prec = digits
        A = [[Decimal(float(x)) if not isinstance(x, Decimal) else x for x in r] for r in A_rows]
        return parareal(A, flow, Decimal(T), N, m, J, K, Decimal(1), Decimal(0))


def to_float(X):
    return [[float(a) for a in r] for r in X]
