"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks the oracle against something the paper or mathematics fixes:
closed-form solutions of the flows, the order of RK4, the exact polynomial form
of RK4 and Euler on a linear flow, the finite-termination property of
Algorithm 1, the G = F special case, an exact rational (Fraction) and a
50-digit (Decimal) re-computation, and the eigenvalue-space reduction.  The
mutation tests at the end plant mistakes in the oracle and check that the pins
catch them.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import brute, closed, parareal as P, scalar as S
from paper_1505_07959_gb300 import inputs

FLOWS = [P.FLOW_INV, P.FLOW_EXP, P.FLOW_SQRT]
T_OF = {P.FLOW_INV: 1.0, P.FLOW_EXP: 1.0, P.FLOW_SQRT: 4.0}
KIND_OF = {P.FLOW_INV: "inv", P.FLOW_EXP: "exp", P.FLOW_SQRT: "sqrt"}


def _nonsym(n, seed, scale=0.3):
    """A general (non-symmetric) matrix close to I, so that I + t(A - I) stays invertible."""
    rng = np.random.default_rng(seed)
    return np.eye(n) + scale * rng.standard_normal((n, n)) / math.sqrt(n)


# --- closed forms -------------------------------------------------------------------------


@pytest.mark.parametrize("flow", FLOWS)
def test_scalar_rk4_matches_closed_form_with_fourth_order(flow):
    """Sequential RK4 on one eigenvalue vs the exact scalar solution; error ratio ~16 per halving."""
    lam = inputs.spectrum(64, KIND_OF[flow], inputs.rng_for(3))
    T = T_OF[flow]
    exact = closed.scalar_solution(flow, lam, T)
    errs = []
    for N, J in [(4, 8), (4, 16), (4, 32)]:
        x = S.sequential_fine(lam, flow, T, N, J)
        errs.append(np.max(np.abs(x - exact) / np.abs(exact)))
    assert errs[-1] < 1e-7
    for e0, e1 in zip(errs, errs[1:]):
        assert 12.0 < e0 / e1 < 20.0, errs


def test_inverse_flow_reaches_lu_inverse():
    """Example 1: Q(1) = A^{-1}.  The tiny inverse workload (n=64, N=8, J=16) vs LU."""
    w = inputs.INV_N64
    sm = inputs.sym_matrix(w.n, w.kind, w.seed)
    X = P.sequential_fine(sm.A, P.FLOW_INV, w.T, w.N, w.J)
    assert P.rel_fro(X, closed.inv_lu(sm.A)) < 1e-10


def test_inverse_flow_nonsymmetric_reaches_lu_inverse():
    """The homotopy inverse flow holds for any A with I + t(A - I) invertible on [0, 1]."""
    A = _nonsym(12, 7)
    X = P.sequential_fine(A, P.FLOW_INV, 1.0, 8, 32)
    assert P.rel_fro(X, closed.inv_lu(A)) < 1e-10


def test_exp_flow_reaches_expm_symmetric_and_general():
    """Example 2: Q(1) = exp(A), vs eigh (symmetric) and scipy.linalg.expm (general)."""
    sm = inputs.sym_matrix(48, "exp", 5)
    X = P.sequential_fine(sm.A, P.FLOW_EXP, 1.0, 8, 64)
    assert P.rel_fro(X, closed.expm_sym(sm.A)) < 1e-11
    A = _nonsym(10, 11, scale=1.0) - np.eye(10)
    X = P.sequential_fine(A, P.FLOW_EXP, 1.0, 8, 64)
    assert P.rel_fro(X, scipy.linalg.expm(A)) < 1e-11


def test_sqrt_flow_tracks_scalar_solution_and_steady_state():
    """dX/dt = A - X^2 from I: at time T each eigen-component equals x(T); as T grows X -> A^{1/2}."""
    rng = inputs.rng_for(9)
    q = inputs.haar_orthogonal(32, rng)
    lam = rng.uniform(0.25, 1.0, 32)
    A = (q * lam) @ q.T
    A = 0.5 * (A + A.T)
    X = P.sequential_fine(A, P.FLOW_SQRT, 4.0, 8, 16)
    ref = S.to_matrix(q, closed.scalar_solution(P.FLOW_SQRT, lam, 4.0))
    assert P.rel_fro(X, ref) < 1e-9
    X = P.sequential_fine(A, P.FLOW_SQRT, 40.0, 40, 16)
    assert P.rel_fro(X, closed.sqrtm_spd(A)) < 1e-9


def test_exp_rk4_and_euler_are_the_taylor_polynomials():
    """On dX/dt = AX one RK4 step is T4(hA) X and Euler is (I + dt A) X, exactly."""
    A = _nonsym(16, 3, scale=1.0) - np.eye(16)
    N, J, m, T = 4, 8, 3, 1.0
    h = T / (N * J)
    hA = h * A
    T4 = np.eye(16) + hA + hA @ hA / 2 + hA @ hA @ hA / 6 + hA @ hA @ hA @ hA / 24
    X = P.sequential_fine(A, P.FLOW_EXP, T, N, J)
    assert P.rel_fro(X, np.linalg.matrix_power(T4, N * J)) < 1e-13
    G = P.euler(P.FLOW_EXP, np.eye(16), A, T / N, m)
    assert P.rel_fro(G, np.linalg.matrix_power(np.eye(16) + (T / N / m) * A, m)) < 1e-14


# --- properties of Algorithm 1 ------------------------------------------------------------


@pytest.mark.parametrize("flow", FLOWS)
def test_finite_termination(flow):
    """After k iterations, U^k_n equals the sequential fine solution for n <= k; K = N gives it everywhere."""
    sm = inputs.sym_matrix(12, KIND_OF[flow], 21)
    T, N, J, m = T_OF[flow], 6, 4, 2
    seq = P.sequential_fine(sm.A, flow, T, N, J, all_slices=True)
    res = P.parareal(sm.A, flow, T, N, m, J, K_max=N, tol=0.0, keep_all=True)
    assert res.iterations == N
    for k, Uk in enumerate(res.all_U):
        for n in range(0, min(k, N) + 1):
            assert P.rel_fro(Uk[n], seq[n]) < 1e-13, (k, n)
    assert P.rel_fro(res.U[N], seq[N]) < 1e-13


@pytest.mark.parametrize("flow", FLOWS)
def test_coarse_equal_fine_converges_in_one_iteration(flow):
    """With G replaced by F the correction makes every slice exact after one sweep."""
    sm = inputs.sym_matrix(10, KIND_OF[flow], 4)
    T, N, J = T_OF[flow], 5, 3
    seq = P.sequential_fine(sm.A, flow, T, N, J, all_slices=True)
    res = P.parareal(sm.A, flow, T, N, 1, J, K_max=3, tol=1e-14, coarse="fine")
    assert res.iterations <= 2
    assert res.dx_history[0] < 1e-14
    for n in range(N + 1):
        assert P.rel_fro(res.U[n], seq[n]) < 1e-14


def test_exp_fine_sweep_is_linear():
    """For the linear flow F(aX + bY) = aF(X) + bF(Y) (the affine identity of Section 3)."""
    A = _nonsym(9, 2) - np.eye(9)
    rng = np.random.default_rng(0)
    X, Y = rng.standard_normal((9, 9)), rng.standard_normal((9, 9))
    F = lambda Z: P.rk4(P.FLOW_EXP, Z, A, 0.25, 5)
    assert P.rel_fro(F(2.0 * X - 3.0 * Y), 2.0 * F(X) - 3.0 * F(Y)) < 1e-14


def test_coarse_sweep_and_fine_sweep_compose_algorithm_1():
    """One iteration assembled from fine_sweep + coarse_sweep equals Algorithm 1's first iteration."""
    sm = inputs.sym_matrix(8, "inv", 1)
    T, N, m, J = 1.0, 4, 1, 4
    U0, G0 = P.coarse_sweep(sm.A, P.FLOW_INV, T, N, m, np.eye(8))
    Fs = P.fine_sweep(sm.A, P.FLOW_INV, T, N, J, U0)
    D = [Fs[n] - G0[n] for n in range(N)]
    U1, _ = P.coarse_sweep(sm.A, P.FLOW_INV, T, N, m, np.eye(8), D)
    res = P.parareal(sm.A, P.FLOW_INV, T, N, m, J, K_max=1, tol=0.0)
    for n in range(N + 1):
        assert np.array_equal(U1[n], res.U[n])


# --- independent re-computations ----------------------------------------------------------


def test_exact_fraction_parareal_exp_nonsymmetric():
    """Exact rational Algorithm 1 on a non-symmetric rational A (exp flow) vs the float64 oracle."""
    A_rows = [[-1, 0.5, 0.25], [0.125, -2, 0.5], [-0.25, 0.75, -0.5]]
    hist = brute.parareal_fraction(A_rows, 1, 1, 3, 2, 2, 2)
    A = np.array(A_rows, dtype=float)
    res = P.parareal(A, P.FLOW_EXP, 1.0, 3, 2, 2, K_max=2, tol=0.0, keep_all=True)
    for k in range(3):
        for n in range(4):
            ex = np.array(brute.to_float(hist[k][n]))
            assert P.rel_fro(res.all_U[k][n], ex) < 1e-14, (k, n)


@pytest.mark.parametrize("flow", FLOWS)
def test_exact_fraction_parareal_nonlinear_tiny(flow):
    """Exact rational Algorithm 1 for every flow on a tiny non-symmetric A (1 RK4 step per slice)."""
    A_rows = [[1.5, 0.25], [-0.125, 0.75]] if flow != P.FLOW_EXP else [[-1, 0.5], [0.25, -2]]
    T = 1 if flow != P.FLOW_SQRT else 2
    hist = brute.parareal_fraction(A_rows, flow, T, 2, 1, 1, 2)
    A = np.array(A_rows, dtype=float)
    res = P.parareal(A, flow, float(T), 2, 1, 1, K_max=2, tol=0.0, keep_all=True)
    for k in range(3):
        for n in range(3):
            ex = np.array(brute.to_float(hist[k][n]))
            assert P.rel_fro(res.all_U[k][n], ex) < 1e-14, (k, n)


@pytest.mark.parametrize("flow", FLOWS)
def test_decimal_50_digit_parareal(flow):
    """50-digit Algorithm 1 with every flow, m = 2 Euler substeps, non-symmetric A, vs float64."""
    A = _nonsym(4, 13 + flow, scale=0.4)
    if flow == P.FLOW_EXP:
        A = A - 2.0 * np.eye(4)
    T = T_OF[flow]
    hist = brute.parareal_decimal(A.tolist(), flow, T, 3, 2, 2, 3)
    res = P.parareal(A, flow, T, 3, 2, 2, K_max=3, tol=0.0, keep_all=True)
    for k in range(4):
        for n in range(4):
            ex = np.array(brute.to_float(hist[k][n]))
            assert P.rel_fro(res.all_U[k][n], ex) < 1e-13, (k, n)


@pytest.mark.parametrize("flow", FLOWS)
def test_matrix_oracle_equals_eigenvalue_recurrence(flow):
    """With X0 = I every iterate is Q diag(u) Q^T: the two oracles agree iterate by iterate."""
    n = 24
    sm = inputs.sym_matrix(n, KIND_OF[flow], 31)
    T, N, J, m = T_OF[flow], 6, 8, 1
    res = P.parareal(sm.A, flow, T, N, m, J, K_max=6, tol=1e-12)
    sres = S.parareal(sm.lam, flow, T, N, m, J, K_max=6, tol=1e-12)
    assert res.iterations == sres.iterations
    for k in range(res.iterations):
        a, b = res.dx_history[k], sres.dx_history[k]
        assert abs(a - b) <= 1e-9 * max(b, 1e-6), (k, a, b)
    for s in range(N + 1):
        assert P.rel_fro(res.U[s], S.to_matrix(sm.Q, sres.u[s])) < 1e-12


def test_tiny_inverse_workload_iterations_and_accuracy():
    """The n=64 inverse workload: converges within K <= 8 and matches A^{-1} to 1e-10."""
    w = inputs.INV_N64
    sm = inputs.sym_matrix(w.n, w.kind, w.seed)
    res = P.parareal(sm.A, w.flow, w.T, w.N, w.m, w.J, w.K_max, w.tol)
    assert res.iterations <= 8
    assert P.rel_fro(res.U[w.N], closed.inv_lu(sm.A)) < 1e-10
    seq = P.sequential_fine(sm.A, w.flow, w.T, w.N, w.J)
    assert P.rel_fro(res.U[w.N], seq) < 1e-12


# --- refinement ----------------------------------------------------------------------------


def test_newton_schulz_converges_quadratically_to_inverse():
    from oracle import refine
    sm = inputs.sym_matrix(40, "inv", 8)
    Ainv = closed.inv_lu(sm.A)
    rng = np.random.default_rng(1)
    E = rng.standard_normal((40, 40)) * 1e-3
    X = Ainv @ (np.eye(40) + 0.5 * (E + E.T))
    e0 = P.rel_fro(X, Ainv)
    e1 = P.rel_fro(refine.newton_schulz_inv(sm.A, X, 1), Ainv)
    e3 = P.rel_fro(refine.newton_schulz_inv(sm.A, X, 3), Ainv)
    assert e1 < 10 * e0 * e0 * 40 and e1 < e0 / 10
    assert e3 < 1e-13


def test_newton_sylvester_sqrt_converges():
    from oracle import refine
    sm = inputs.sym_matrix(48, "sqrt", 2)
    R = closed.sqrtm_spd(sm.A)
    rng = np.random.default_rng(2)
    E = rng.standard_normal((48, 48)) * 1e-3
    X = R + 0.5 * (E + E.T) * np.abs(R).max()
    errs = [P.rel_fro(refine.newton_sylvester_sqrt(sm.A, X, s), R) for s in range(5)]
    assert errs[4] < 1e-11
    assert errs[2] < errs[1] < errs[0]


# --- planted mistakes: the pins above must catch each of these -----------------------------


def _pins_pass():
    """A small battery of the pins above, run against the (possibly mutated) oracle."""
    ok = True
    try:
        test_inverse_flow_reaches_lu_inverse()
        test_exp_flow_reaches_expm_symmetric_and_general()
        test_sqrt_flow_tracks_scalar_solution_and_steady_state()
        test_inverse_flow_nonsymmetric_reaches_lu_inverse()
        for f in FLOWS:
            test_finite_termination(f)
            test_decimal_50_digit_parareal(f)
    except AssertionError:
        ok = False
    return ok


def test_unmutated_oracle_passes_battery():
    assert _pins_pass()


@pytest.mark.parametrize("mutation", [
    "rk4_weight", "rk4_node", "inv_sign", "exp_transpose", "sqrt_order", "euler_step",
    "correction_sign", "correction_reuse_new",
])
def test_planted_mistakes_are_caught(monkeypatch, mutation):
    real_rhs, real_rk4, real_euler = P.rhs, P.rk4, P.euler

    if mutation == "rk4_weight":
        def rk4(flow, X, A, dT, J):
            h = dT / J
            for _ in range(J):
                k1 = real_rhs(flow, X, A); k2 = real_rhs(flow, X + h / 2 * k1, A)
                k3 = real_rhs(flow, X + h / 2 * k2, A); k4 = real_rhs(flow, X + h * k3, A)
                X = X + h / 6 * (k1 + 2 * k2 + k3 + 2 * k4)
            return X
        monkeypatch.setattr(P, "rk4", rk4)
    elif mutation == "rk4_node":
        def rk4(flow, X, A, dT, J):
            h = dT / J
            for _ in range(J):
                k1 = real_rhs(flow, X, A); k2 = real_rhs(flow, X + h / 2 * k1, A)
                k3 = real_rhs(flow, X + h / 2 * k2, A); k4 = real_rhs(flow, X + h / 2 * k3, A)
                X = X + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            return X
        monkeypatch.setattr(P, "rk4", rk4)
    elif mutation == "inv_sign":
        monkeypatch.setattr(P, "rhs", lambda f, X, A: (X @ (A - np.eye(A.shape[0])) @ X) if f == 0
                            else real_rhs(f, X, A))
    elif mutation == "exp_transpose":
        monkeypatch.setattr(P, "rhs", lambda f, X, A: (A.T @ X) if f == 1 else real_rhs(f, X, A))
    elif mutation == "sqrt_order":
        monkeypatch.setattr(P, "rhs", lambda f, X, A: (A - X @ X @ X) if f == 2 else real_rhs(f, X, A))
    elif mutation == "euler_step":
        monkeypatch.setattr(P, "euler", lambda f, X, A, dT, m: real_euler(f, X, A, dT, 1)
                            if m > 1 else X + dT * real_rhs(f, X, A) * 0.9)
    elif mutation in ("correction_sign", "correction_reuse_new"):
        real_generic = P.parareal_generic

        def generic(X0, N, G, F, K_max, tol, keep_all=False):
            U = [X0]; G_old = []
            for n in range(N):
                g = G(n, U[n]); G_old.append(g); U.append(g)
            all_U = [list(U)] if keep_all else None
            hist, last, it = [], [], 0
            for _ in range(K_max):
                F_old = [F(n, U[n]) for n in range(N)]
                V = [X0]; G_new = []
                for n in range(N):
                    g = G(n, V[n]); G_new.append(g)
                    if mutation == "correction_sign":
                        V.append(g - (F_old[n] - G_old[n]))
                    else:
                        V.append(g + (F_old[n] - g))
                r = [P.fro(V[n] - U[n]) / P.fro(V[n]) for n in range(1, N + 1)]
                U, G_old = V, G_new
                it += 1; hist.append(max(r)); last.append(r[-1])
                if keep_all:
                    all_U.append(list(U))
                if max(r) < tol:
                    break
            return P.PararealResult(U=U, iterations=it, dx_history=hist, dx_last_slice=last, all_U=all_U)
        monkeypatch.setattr(P, "parareal_generic", generic)
        assert real_generic is not generic
    assert not _pins_pass(), mutation


def test_convergence_measure_propagates_non_finite_slices():
    """A slice whose iterate is not finite makes the stopping test's maximum not finite (the
    maximum over n of ||dU_n|| / ||U_n||), so a diverging run is never reported converged."""
    def F(_n, x):
        return x * np.inf if _n == 2 else 2.0 * x
    r = P.parareal_generic(np.eye(2), 4, lambda _n, x: x, F, 2, 1e-10)
    assert not np.isfinite(r.dx_history[0])


def test_sign_iteration_solves_the_sylvester_equation():
    """The block Newton-Schulz sign iteration reaches the eigenbasis solution of X E + E X = R
    (the plain definition) and the identity P -> I; dropping the P Q P term breaks it."""
    from oracle import refine as RF
    sm = inputs.sym_matrix(60, "sqrt", 12)
    X = S.to_matrix(sm.Q, np.sqrt(sm.lam)) + 1e-3 * inputs.sym_matrix(60, "exp", 13).A
    X = 0.5 * (X + X.T)
    R = sm.A - X @ X
    mu, V = np.linalg.eigh(X)
    E_exact = V @ ((V.T @ R @ V) / (mu[:, None] + mu[None, :])) @ V.T
    E, Pm = RF.sylvester_sign(X, R, 16)
    assert P.rel_fro(E, E_exact) < 1e-11
    assert np.max(np.abs(Pm - np.eye(60))) < 1e-12
    assert P.rel_fro(X @ E + E @ X, R) < 1e-11
    # a scale below lambda_max / sqrt(3) leaves the convergence region
    E_bad, _ = RF.sylvester_sign(X, R, 16, mu=float(mu[-1]) / 2.0)
    assert not (P.rel_fro(E_bad, E_exact) < 1e-3)


def test_newton_sign_sqrt_matches_eigen_newton():
    from oracle import refine as RF
    sm = inputs.sym_matrix(48, "sqrt", 14)
    X0 = S.to_matrix(sm.Q, closed.scalar_solution(2, sm.lam, 20.0))
    X0 = X0 + 1e-3 * inputs.sym_matrix(48, "exp", 15).A
    exact = S.to_matrix(sm.Q, np.sqrt(sm.lam))
    Xa = RF.newton_sylvester_sqrt(sm.A, X0, 4)
    Xb = RF.newton_sign_sqrt(sm.A, X0, 4, 18)
    assert P.rel_fro(Xa, exact) < 1e-10 and P.rel_fro(Xb, exact) < 1e-10


# --- the paper's own propagators: explicit Euler F and Crank-Nicolson (Section 2) ------------


def test_crank_nicolson_is_the_cayley_step_per_eigenvalue():
    """On a symmetric A every CN step multiplies eigencomponent i by (1 + h l_i / 2) /
    (1 - h l_i / 2), so J steps from I give Q diag(r_i^J) Q^T; the scheme is second order."""
    sm = inputs.sym_matrix(12, "exp", 21)
    dT, J = 0.25, 5
    h = dT / J
    X = P.crank_nicolson(P.FLOW_EXP, np.eye(12), sm.A, dT, J)
    r = (1 + h * sm.lam / 2) / (1 - h * sm.lam / 2)
    assert P.rel_fro(X, S.to_matrix(sm.Q, r ** J)) < 1e-14
    exact = scipy.linalg.expm(sm.A)
    e1 = P.rel_fro(P.crank_nicolson(P.FLOW_EXP, np.eye(12), sm.A, 1.0, 16), exact)
    e2 = P.rel_fro(P.crank_nicolson(P.FLOW_EXP, np.eye(12), sm.A, 1.0, 32), exact)
    assert 3.5 < e1 / e2 < 4.5


def test_explicit_euler_fine_propagator_is_the_euler_polynomial():
    """F with the explicit Euler scheme is (I + h A)^J on the linear flow; first order."""
    sm = inputs.sym_matrix(10, "exp", 22)
    f = P.propagator("euler", P.FLOW_EXP, sm.A, 0.5, 8)
    want = np.linalg.matrix_power(np.eye(10) + (0.5 / 8) * sm.A, 8)
    assert P.rel_fro(f(np.eye(10)), want) < 1e-14
    exact = scipy.linalg.expm(sm.A)
    e1 = P.rel_fro(P.sequential_fine(sm.A, P.FLOW_EXP, 1.0, 4, 64, fine="euler"), exact)
    e2 = P.rel_fro(P.sequential_fine(sm.A, P.FLOW_EXP, 1.0, 4, 128, fine="euler"), exact)
    assert 1.8 < e1 / e2 < 2.2


@pytest.mark.parametrize("ex", [inputs.PAPER_EX1, inputs.PAPER_EX2])
def test_paper_examples_converge_to_the_fine_solution_and_the_matrix_function(ex):
    """Section 2, Examples 1 and 2 (n = 80 Laplacian / 2^10, N = 25, J = 200): parareal with the
    paper's propagators terminates on the sequential fine solution (finite termination at
    K = N) and its error measure max|E| / max|A| against the function is the fine scheme's."""
    A = inputs.paper_example_matrix(ex.example)
    r = P.parareal(A, ex.flow, ex.T, ex.N, 1, ex.J, ex.N, 0.0, coarse=ex.coarse, fine=ex.fine)
    seq = P.sequential_fine(A, ex.flow, ex.T, ex.N, ex.J, fine=ex.fine)
    assert P.paper_norm(r.U[ex.N] - seq, A) < 1e-12
    ref = closed.inv_lu(A) if ex.flow == P.FLOW_INV else scipy.linalg.expm(A)
    # explicit Euler with h = 2e-4 on the inverse flow: O(h) error; Crank-Nicolson: O(h^2)
    assert P.paper_norm(r.U[ex.N] - ref, A if ex.flow == P.FLOW_INV else ref) < (
        5e-2 if ex.flow == P.FLOW_INV else 1e-6)
    assert r.dx_history[-1] < 1e-12
    assert r.dx_history[0] > r.dx_history[min(5, len(r.dx_history) - 1)]
