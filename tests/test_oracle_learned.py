"""Pins of the learned-coarse-propagator oracle against facts independent of it."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import learned as L, parareal as P
from paper_1505_07959_gb300 import inputs

FLOWS = [0, 1, 2]
KIND = {0: "inv", 1: "exp", 2: "sqrt"}


def test_taylor_terms_match_exact_one_slice_maps():
    """inverse: X (I - t B X)^{-1} (Neumann); exp: expm(tA) X; sqrt: the scalar solution."""
    sm = inputs.sym_matrix(20, "inv", 1)
    X = np.eye(20) + 0.05 * inputs.sym_matrix(20, "exp", 2).A
    B = np.eye(20) - sm.A
    for t in (0.05, 0.025):
        exact = X @ np.linalg.inv(np.eye(20) - t * B @ X)
        T = L.taylor_terms(0, sm.A, X, 4)
        approx = X + sum(t ** (j + 1) * T[j] for j in range(4))
        assert P.rel_fro(approx, exact) < 40 * t ** 5
    A = inputs.sym_matrix(20, "exp", 3).A
    for t in (0.05, 0.025):
        T = L.taylor_terms(1, A, X, 4)
        approx = X + sum(t ** (j + 1) * T[j] for j in range(4))
        assert P.rel_fro(approx, scipy.linalg.expm(t * A) @ X) < 10 * t ** 5
    # sqrt: from X = I the solution is Q diag(x(t)) Q^T with the scalar closed form
    sq = inputs.sym_matrix(16, "sqrt", 4)
    from oracle import closed, scalar as S
    t = 0.05
    T = L.taylor_terms(2, sq.A, np.eye(16), 4)
    approx = np.eye(16) + sum(t ** (j + 1) * T[j] for j in range(4))
    exact = S.to_matrix(sq.Q, closed.scalar_solution(2, sq.lam, t))
    assert P.rel_fro(approx, exact) < 1e-6


@pytest.mark.parametrize("flow", FLOWS)
def test_euler_and_taylor_coefficients(flow):
    """c = (1,0,0,0) is the paper's forward-Euler step; the first term is Fl(X)."""
    sm = inputs.sym_matrix(12, KIND[flow], 5)
    X = np.eye(12) + 0.01 * sm.A
    dT = 0.1
    assert np.allclose(L.g_theta(flow, sm.A, X, dT, [1, 0, 0, 0]), P.euler(flow, X, sm.A, dT, 1),
                       rtol=0, atol=1e-14)
    assert np.allclose(L.taylor_terms(flow, sm.A, X, 1)[0], P.rhs(flow, X, sm.A), atol=1e-14)


def test_pair_record_gives_the_residual_as_a_quadratic():
    sm = inputs.sym_matrix(14, "inv", 6)
    X0 = np.eye(14) + 0.02 * sm.A
    X1 = P.rk4(0, X0, sm.A, 0.1, 4)
    M, b, dd = L.pair_record(0, sm.A, X0, X1, 0.1)
    c = np.array([0.9, 1.1, 0.7, 0.3])
    direct = np.sum((L.g_theta(0, sm.A, X0, 0.1, c) - X1) ** 2) / dd
    assert abs((c @ M @ c - 2 * c @ b + dd) / dd - direct) < 1e-12


def test_gelu_and_backprop_against_finite_differences():
    assert abs(L.gelu(np.array([1.0]))[0] - 0.5 * (1 + math.erf(1 / math.sqrt(2)))) < 1e-15
    rng = np.random.default_rng(0)
    p = L.init_params(1)
    p["W3"] = rng.standard_normal(p["W3"].shape) * 0.1
    x = rng.standard_normal((5, 8))
    M = np.array([np.eye(4) + 0.1 * rng.standard_normal((4, 4)) for _ in range(5)])
    M = np.einsum("bij,bkj->bik", M, M)
    bv = rng.standard_normal((5, 4))
    dd = rng.uniform(1, 2, 5)
    loss, g = L.loss_and_grad(p, x, M, bv, dd)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        idx = tuple(rng.integers(0, s) for s in p[k].shape)
        eps = 1e-6
        q = {kk: vv.copy() for kk, vv in p.items()}
        q[k][idx] += eps
        lp, _ = L.loss_and_grad(q, x, M, bv, dd)
        q[k][idx] -= 2 * eps
        lm, _ = L.loss_and_grad(q, x, M, bv, dd)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[k][idx]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k][idx])


def test_untrained_network_is_euler_and_blob_round_trips():
    p = L.init_params(3)
    c, _ = L.forward(p, np.random.default_rng(1).standard_normal((3, 8)))
    assert np.array_equal(c, np.tile([1.0, 0.0, 0.0, 0.0], (3, 1)))
    q = L.from_blob(L.to_blob(p))
    for k in L.BLOB_ORDER:
        assert np.allclose(q[k], p[k], rtol=1e-6, atol=1e-7)


def test_adam_decreases_the_loss_on_a_fixed_batch():
    rng = np.random.default_rng(2)
    p = L.init_params(4)
    x = rng.standard_normal((16, 8))
    target = np.array([1.0, 0.5, 0.2, 0.05])
    M = np.tile(np.eye(4), (16, 1, 1))
    bv = np.tile(target, (16, 1))
    dd = np.full(16, target @ target)          # loss = |c - target|^2 / |target|^2, minimum 0
    st = {}
    l0, _ = L.loss_and_grad(p, x, M, bv, dd)
    for _ in range(200):
        _, g = L.loss_and_grad(p, x, M, bv, dd)
        p = L.adam(p, g, st, lr=3e-3)
    l1, _ = L.loss_and_grad(p, x, M, bv, dd)
    assert l1 < 0.05 * l0


def test_taylor_coarse_step_cuts_parareal_iterations_on_the_wide_inverse_family():
    """The fixed Taylor-4 step (c = 1,1,1,1) already beats Euler on the wide-spectrum inverse
    family, so there is something for a learned step to recover."""
    sm = inputs.sym_matrix(48, "inv_wide", 7)
    T, N, J = 1.0, 16, 16
    dT = T / N
    F = lambda _n, x: P.rk4(0, x, sm.A, dT, J)
    Ge = lambda _n, x: P.euler(0, x, sm.A, dT, 1)
    Gt = lambda _n, x: L.g_theta(0, sm.A, x, dT, [1, 1, 1, 1])
    re = P.parareal_generic(np.eye(48), N, Ge, F, N, 1e-8)
    rt = P.parareal_generic(np.eye(48), N, Gt, F, N, 1e-8)
    assert rt.iterations < re.iterations
    assert P.rel_fro(rt.U[N], re.U[N]) < 1e-7


def test_splitmix64_matches_the_published_stream():
    """Seed 0: the reference generator's first outputs are 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4."""
    assert L.splitmix64(0, 2) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_hutchinson_is_exact_on_diagonals_and_unbiased():
    Z = L.probes(300)
    assert set(np.unique(Z)) == {-1.0, 1.0}
    assert abs(Z.mean()) < 4.0 / math.sqrt(Z.size)
    d = np.random.default_rng(3).standard_normal(300)
    assert abs(L.hutchinson(np.diag(d), Z) - d.sum()) < 1e-12          # z_i^2 = 1
    A = inputs.sym_matrix(300, "exp", 8).A
    sigma = math.sqrt(2 * (np.sum(A * A) - np.sum(np.diag(A) ** 2)) / Z.shape[0])
    assert abs(L.hutchinson(A, Z) - np.trace(A)) < 5 * sigma


def test_bf16_rounding_ties_to_even():
    e = 2.0 ** -8
    x = np.array([1.0, 1 + e, 1 + 3 * e, 1 + e * 1.01, -1 - 3 * e, 3.0e38])
    want = np.array([1.0, 1.0, 1 + 4 * e, 1 + 2 * e, -1 - 4 * e, None], dtype=object)
    got = L.bf16_round(x)
    for g, w in zip(got[:5], want[:5]):
        assert g == w
    assert np.isfinite(got[5]) or np.isinf(got[5])
    q = L.deployed(L.init_params(0))
    for k in ("W1", "W2", "W3"):
        assert np.array_equal(L.bf16_round(q[k]), q[k])


def test_constant_networks_reproduce_euler_and_taylor_parareal():
    """W3 = 0 makes c = b3: (1,0,0,0) must give the paper's Euler-G parareal iterate for
    iterate (up to the grouping of X (I - A) X), (1,1,1,1) the Taylor-4 G; and parareal with
    any G meets the sequential fine solution after N iterations (finite termination)."""
    sm = inputs.sym_matrix(10, "inv_wide", 9)
    T, N, J = 1.0, 4, 4
    p = L.init_params(1)
    r_l = L.parareal_learned(p, sm.A, 0, T, N, J, N, 0.0)
    r_e = P.parareal(sm.A, 0, T, N, 1, J, N, 0.0)
    for a, b in zip(r_l.U, r_e.U):
        assert P.rel_fro(a, b) < 1e-14
    p["b3"] = np.array([1.0, 1.0, 1.0, 1.0])
    r_t = L.parareal_learned(p, sm.A, 0, T, N, J, N, 0.0)
    seq = P.sequential_fine(sm.A, 0, T, N, J)
    assert P.rel_fro(r_t.U[N], seq) < 1e-14
    Gt = lambda _n, x: L.g_theta(0, sm.A, x, T / N, [1, 1, 1, 1])
    F = lambda _n, x: P.rk4(0, x, sm.A, T / N, J)
    r_g = P.parareal_generic(np.eye(10), N, Gt, F, 1, 0.0)
    r_t1 = L.parareal_learned(p, sm.A, 0, T, N, J, 1, 0.0)
    assert all(np.array_equal(a, b) for a, b in zip(r_g.U, r_t1.U))


def _learned_battery() -> bool:
    """A battery of the pins above, run against the (possibly mutated) learned oracle."""
    checks = [test_taylor_terms_match_exact_one_slice_maps, test_pair_record_gives_the_residual_as_a_quadratic,
              test_gelu_and_backprop_against_finite_differences, test_hutchinson_is_exact_on_diagonals_and_unbiased,
              test_splitmix64_matches_the_published_stream, test_bf16_rounding_ties_to_even,
              test_constant_networks_reproduce_euler_and_taylor_parareal,
              lambda: [test_euler_and_taylor_coefficients(f) for f in FLOWS]]
    try:
        for c in checks:
            c()
    except AssertionError:
        return False
    return True


def test_unmutated_learned_oracle_passes_battery():
    assert _learned_battery()


@pytest.mark.parametrize("mutation", ["inv_power", "exp_factorial", "sqrt_cauchy", "gelu_grad",
                                      "backprop_transpose", "splitmix_shift", "bf16_truncate",
                                      "dd_residual"])
def test_planted_mistakes_in_learned_oracle_are_caught(monkeypatch, mutation):
    real_tt, real_gg, real_lg, real_sm = L.taylor_terms, L.gelu_grad, L.loss_and_grad, L.splitmix64
    real_pr = L.pair_record
    if mutation == "inv_power":          # X (BX)^j with the powers off by one
        monkeypatch.setattr(L, "taylor_terms", lambda f, A, X, q=4: (
            [X @ np.linalg.matrix_power((np.eye(A.shape[0]) - A) @ X, j) for j in range(q)]
            if f == 0 else real_tt(f, A, X, q)))
    elif mutation == "exp_factorial":    # A^j X without 1/j!
        monkeypatch.setattr(L, "taylor_terms", lambda f, A, X, q=4: (
            [np.linalg.matrix_power(A, j) @ X for j in range(1, q + 1)]
            if f == 1 else real_tt(f, A, X, q)))
    elif mutation == "sqrt_cauchy":      # missing the 1/(j+1) of the recursion
        def tt(f, A, X, q=4):
            if f != 2:
                return real_tt(f, A, X, q)
            c = [X]
            for j in range(q):
                s = sum(c[i] @ c[j - i] for i in range(j + 1))
                c.append((A if j == 0 else 0.0) - s)
            return c[1:]
        monkeypatch.setattr(L, "taylor_terms", tt)
    elif mutation == "gelu_grad":        # drops the x phi(x) term
        from scipy.special import erf
        monkeypatch.setattr(L, "gelu_grad", lambda x: 0.5 * (1.0 + erf(x / math.sqrt(2.0))))
    elif mutation == "backprop_transpose":
        def lg(p, x, M, b, dd):
            loss, g = real_lg(p, x, M, b, dd)
            g["W2"] = g["W2"].T.copy()
            return loss, g
        monkeypatch.setattr(L, "loss_and_grad", lg)
    elif mutation == "splitmix_shift":
        def sm(seed, count):
            out = []
            for c in range(count):
                z = (seed + (c + 1) * 0x9E3779B97F4A7C15) & L._M64
                z = ((z ^ (z >> 31)) * 0xBF58476D1CE4E5B9) & L._M64
                z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & L._M64
                out.append(z ^ (z >> 31))
            return out
        monkeypatch.setattr(L, "splitmix64", sm)
    elif mutation == "bf16_truncate":
        monkeypatch.setattr(L, "bf16_round", lambda x: (np.asarray(x, dtype=np.float32).view(np.uint32)
                                                        & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64))
    elif mutation == "dd_residual":      # b taken against X_{n+1} instead of D = X_{n+1} - X_n
        def pr(flow, A, X0, X1, dT):
            M, b, dd = real_pr(flow, A, X0, X1, dT)
            Z = [dT ** (j + 1) * T for j, T in enumerate(real_tt(flow, A, X0, 4))]
            return M, np.array([np.sum(z * X1) for z in Z]), dd
        monkeypatch.setattr(L, "pair_record", pr)
    assert not _learned_battery(), mutation
