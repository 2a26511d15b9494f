"""Pins of the modified-parareal oracle (Section 3: the diamond product, globalQR, the projection
and Algorithms 3 and 4) against facts that do not come from the oracle itself."""
import numpy as np
import pytest

from oracle import modified as M, parareal as P
from paper_1505_07959_gb300 import inputs


def _blocks(k, n, s, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((n, s)) for _ in range(k)]


def test_diamond_product_properties():
    """Section 3's proposition: s = 1 gives A^T B; Q is F-orthonormal iff Q^T <> Q = I;
    X^T <> X = ||X||_F^2; and <A, B>_F = tr(B^T A) on a hand-computed pair."""
    A, B = _blocks(3, 5, 1, 0), _blocks(2, 5, 1, 1)
    Am, Bm = np.hstack(A), np.hstack(B)
    assert np.allclose(M.diamond(A, B), Am.T @ Bm, rtol=1e-14, atol=1e-14)
    X = _blocks(1, 4, 3, 2)[0]
    assert np.isclose(M.diamond([X], [X])[0, 0], np.sum(X * X), rtol=1e-14)
    assert M.fro_inner(np.array([[1.0, 2.0], [3.0, 4.0]]), np.array([[0.0, 1.0], [-1.0, 2.0]])) == 7.0
    # column blocks of an orthogonal matrix, scaled, are F-orthonormal
    Qm = inputs.haar_orthogonal(6, inputs.rng_for(3))
    Qb = [Qm[:, 2 * i:2 * i + 2] / np.sqrt(2.0) for i in range(3)]
    assert np.allclose(M.diamond(Qb, Qb), np.eye(3), atol=1e-14)


@pytest.mark.parametrize("passes", [1, 2])
def test_global_qr_reconstructs_and_orthonormalises(passes):
    """Proposition of Algorithm 2: Z = Q (R kron I_s) and Q^T <> Q = I (independent blocks)."""
    Z = _blocks(5, 6, 4, 4)
    Q, R, kept = M.global_qr(Z, passes=passes)
    assert kept == list(range(5))
    assert np.allclose(M.diamond(Q, Q), np.eye(5), atol=1e-13)
    Zm, Qm = np.hstack(Z), np.hstack(Q)
    assert np.allclose(Qm @ np.kron(R, np.eye(4)), Zm, atol=1e-13)
    assert np.allclose(R, np.triu(R))                          # upper triangular
    assert np.all(np.diag(R) > 0)


def test_global_qr_removes_dependent_blocks():
    """A block that is a combination of earlier ones reduces to exactly zero (exact binary
    arithmetic here) and is removed with its row of R; it is still reconstructed."""
    E = np.zeros((3, 3))
    E[0, 0] = 1.0
    F = np.zeros((3, 3))
    F[1, 2] = 2.0
    Z = [E, 2.0 * E, F, E + 0.5 * F]
    Q, R, kept = M.global_qr(Z)
    assert kept == [0, 2]
    assert np.array_equal(Q[0], E) and np.array_equal(Q[1], F / 2.0)
    assert np.allclose(np.hstack(Q) @ np.kron(R, np.eye(3)), np.hstack(Z), atol=0)


def test_projection_properties():
    Z = _blocks(4, 5, 5, 6)
    Q, _, _ = M.global_qr(Z, passes=2)
    Y = _blocks(1, 5, 5, 7)[0]
    PY = M.project(Q, Y)
    assert P.rel_fro(M.project(Q, PY), PY) < 1e-14             # idempotent
    for q in Q:
        assert abs(M.fro_inner(Y - PY, q)) < 1e-13             # residual orthogonal to the span
    c = np.array([0.3, -1.0, 2.0, 0.5])
    inside = sum(ci * z for ci, z in zip(c, Z))
    assert P.rel_fro(M.project(Q, inside), inside) < 1e-14     # identity on the span


def _exp_setup(n, N, J, seed=0):
    sm = inputs.sym_matrix(n, "exp", seed)
    return sm, P.sequential_fine(sm.A, P.FLOW_EXP, 1.0, N, J, all_slices=True)


def test_finite_termination_of_the_modified_algorithm():
    """As in Algorithm 1, U^k_n equals the sequential fine solution for n <= k: U^k_n lies in
    S^k, where the update is F(U^k_n) exactly (up to rounding)."""
    n, N, J = 12, 6, 4
    sm, seq = _exp_setup(n, N, J, 1)
    r = M.modified_parareal(sm.A, P.FLOW_EXP, 1.0, N, 1, J, N, 0.0, drop=1e-14, keep_all=True)
    for k, Uk in enumerate(r.all_U):
        for nn in range(min(k, N) + 1):
            assert P.rel_fro(Uk[nn], seq[nn]) < 1e-12, (k, nn)


def test_full_span_gives_the_fine_solution_after_one_iteration():
    """X0 = I: every iterate is a polynomial in A, a space of dimension n.  With N + 1 > n
    Step-0 blocks the first basis spans it, P = I on every iterate, and the first update is the
    sequential fine solution at every slice; the second changes nothing."""
    n, N, J = 4, 8, 3
    sm, seq = _exp_setup(n, N, J, 2)
    r = M.modified_parareal(sm.A, P.FLOW_EXP, 1.0, N, 1, J, 2, 0.0, drop=1e-13, keep_all=True)
    assert r.new_blocks[0] == n and r.new_blocks[1] == 0
    for nn in range(N + 1):
        assert P.rel_fro(r.all_U[1][nn], seq[nn]) < 1e-12, nn
    assert r.dx_history[1] < 1e-13


def test_empty_space_leaves_the_coarse_solution():
    """With nothing kept (P = 0) the update is U_{n+1} = G(U_n): the Step-0 coarse sweep."""
    n, N, J = 6, 5, 3
    sm = inputs.sym_matrix(n, "exp", 3)
    r = M.modified_parareal(sm.A, P.FLOW_EXP, 1.0, N, 1, J, 3, 0.0, drop=np.inf)
    V = [np.eye(n)]
    for _ in range(N):
        V.append(V[-1] + (1.0 / N) * sm.A @ V[-1])           # forward Euler, written out
    assert r.new_blocks == [0, 0, 0]
    for a, b in zip(r.U, V):
        assert P.rel_fro(a, b) < 1e-15


def test_modified_converges_much_faster_than_classical():
    """Section 3, Example 3's observation on a linear flow: the exponential flow at n = 64 with
    N = 16, J = 16 reaches 1e-10 in at most 3 iterations (classical: 9), and its result is the
    sequential fine solution."""
    n, N, J = 64, 16, 16
    sm, seq = _exp_setup(n, N, J, 0)
    cl = P.parareal(sm.A, P.FLOW_EXP, 1.0, N, 1, J, N, 1e-10)
    r = M.modified_parareal(sm.A, P.FLOW_EXP, 1.0, N, 1, J, N, 1e-10, drop=1e-12)
    assert cl.iterations >= 8
    assert r.iterations <= 3
    assert P.rel_fro(r.U[N], seq[N]) < 1e-12
    assert sum(r.new_blocks) <= N + 1      # at most one sweep's worth of fine propagations (classical: 9 sweeps)


def test_affine_algorithm_4_on_an_inhomogeneous_flow():
    """Algorithm 4 on U' = B U + C (RK4 F, Euler G, both affine): finite termination and the
    sequential fine solution; with C = 0 it is Algorithm 3."""
    n, N, J = 5, 6, 4
    rng = np.random.default_rng(9)
    B = -np.eye(n) + 0.3 * rng.standard_normal((n, n))
    C = rng.standard_normal((n, n))
    dT = 1.0 / N

    def rhs(X):
        return B @ X + C

    def rk4(X):
        h = dT / J
        for _ in range(J):
            k1 = rhs(X); k2 = rhs(X + h / 2 * k1); k3 = rhs(X + h / 2 * k2); k4 = rhs(X + h * k3)
            X = X + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        return X

    def euler(X):
        return X + dT * rhs(X)

    X0 = np.eye(n)
    seq = [X0]
    for _ in range(N):
        seq.append(rk4(seq[-1]))
    r = M.modified_parareal_generic(X0, N, euler, rk4, N, 0.0, drop=1e-13, keep_all=True,
                                    affine=True)
    for k, Uk in enumerate(r.all_U):
        for nn in range(min(k, N) + 1):
            assert P.rel_fro(Uk[nn], seq[nn]) < 1e-12, (k, nn)
    sm = inputs.sym_matrix(n, "exp", 4)
    a = M.modified_parareal(sm.A, P.FLOW_EXP, 1.0, N, 1, J, 3, 0.0, drop=1e-13)
    b = M.modified_parareal_generic(np.eye(n), N, lambda x: P.euler(1, x, sm.A, dT, 1),
                                    lambda x: P.rk4(1, x, sm.A, dT, J), 3, 0.0, 1e-13, affine=True)
    for x, y in zip(a.U, b.U):
        assert P.rel_fro(x, y) < 1e-13


def _battery() -> bool:
    checks = [test_diamond_product_properties,
              lambda: [test_global_qr_reconstructs_and_orthonormalises(p) for p in (1, 2)],
              test_global_qr_removes_dependent_blocks, test_projection_properties,
              test_finite_termination_of_the_modified_algorithm,
              test_full_span_gives_the_fine_solution_after_one_iteration,
              test_empty_space_leaves_the_coarse_solution,
              test_modified_converges_much_faster_than_classical,
              test_affine_algorithm_4_on_an_inhomogeneous_flow]
    try:
        for c in checks:
            c()
    except AssertionError:
        return False
    return True


def test_unmutated_modified_oracle_passes_battery():
    assert _battery()


@pytest.mark.parametrize("mutation", ["inner_transposed", "classical_gs_coefficient",
                                      "no_reorthogonalisation", "coarse_on_full_state",
                                      "alpha_from_images", "normalise_skipped"])
def test_planted_mistakes_in_modified_oracle_are_caught(monkeypatch, mutation):
    real_fi, real_qr, real_gen = M.fro_inner, M.global_qr, M.modified_parareal_generic
    if mutation == "inner_transposed":          # tr(A B) instead of tr(B^T A)
        monkeypatch.setattr(M, "fro_inner", lambda A, B: (float(np.trace(A @ B))
                                                          if A.shape[0] == A.shape[1]
                                                          else real_fi(A, B)))
    elif mutation == "classical_gs_coefficient":    # r_ji from Z_i, not from the reduced Q
        def qr(Z, passes=1, drop=0.0):
            Q, cols, kept = [], [], []
            for i, z in enumerate(Z):
                q = z.copy()
                for j in range(len(Q)):
                    q = q - real_fi(z, Q[j]) * Q[j] - 0.0
                rii = P.fro(q)
                if rii > drop * P.fro(z) and rii > 0:
                    Q.append(q / rii)
                    kept.append(i)
            return Q, np.zeros((len(Q), len(Z))), kept
        monkeypatch.setattr(M, "global_qr", qr)
    elif mutation == "no_reorthogonalisation":
        monkeypatch.setattr(M, "global_qr", lambda Z, passes=1, drop=0.0: real_qr(Z, 1, drop))
    elif mutation in ("coarse_on_full_state", "alpha_from_images"):
        def gen(X0, N, G, F, K_max, tol, drop, passes=2, keep_all=False, affine=False):
            if affine:
                return real_gen(X0, N, G, F, K_max, tol, drop, passes, keep_all, affine)
            U = [X0]
            for n in range(N):
                U.append(G(U[n]))
            all_U = [list(U)] if keep_all else None
            Q, FQ, hist, added = [], [], [], []
            for _ in range(K_max):
                Qk, _, _ = M.global_qr(Q + U, passes=passes, drop=drop)
                new = Qk[len(Q):]
                FQ.extend(F(q) for q in new)
                Q = Qk
                added.append(len(new))
                V = [X0]
                for n in range(N):
                    basis = FQ if mutation == "alpha_from_images" else Q
                    a = np.array([M.fro_inner(V[n], q) for q in basis])
                    PV = sum((ai * q for ai, q in zip(a, Q)), np.zeros_like(X0))
                    FPV = sum((ai * f for ai, f in zip(a, FQ)), np.zeros_like(X0))
                    arg = V[n] if mutation == "coarse_on_full_state" else V[n] - PV
                    V.append(FPV + G(arg))
                dx = max(P.fro(V[n] - U[n]) / P.fro(V[n]) for n in range(1, N + 1))
                U = V
                hist.append(dx)
                if keep_all:
                    all_U.append(list(U))
                if dx < tol:
                    break
            return M.ModifiedResult(U=U, iterations=len(hist), dx_history=hist, new_blocks=added,
                                    basis=Q, all_U=all_U)
        monkeypatch.setattr(M, "modified_parareal_generic", gen)
    elif mutation == "normalise_skipped":       # Q_i = Q instead of Q / r_ii
        def qr(Z, passes=1, drop=0.0):
            Q, R, kept = real_qr(Z, passes, drop)
            return [q * R[j, kept[j]] for j, q in enumerate(Q)], R, kept
        monkeypatch.setattr(M, "global_qr", qr)
    assert not _battery(), mutation
