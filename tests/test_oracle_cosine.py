"""Pins of the cosine oracle (Example 3, eq. eqB, Algorithm 5) against closed forms."""
import numpy as np
import pytest
import scipy.linalg

from oracle import cosine as C, parareal as P
from paper_1505_07959_gb300 import inputs


def _sym(n, seed, scale):
    sm = inputs.sym_matrix(n, "exp", seed)      # eigenvalues in [-4, 0]
    return sm.A * scale, sm.Q, sm.lam * scale


def test_block_flow_is_sine_and_cosine():
    """exp(B) (0; I) = (sin A0; cos A0) for B of eq. eqB (scipy's expm, eigendecomposition)."""
    A0, Q, lam = _sym(9, 1, 0.2)
    U = scipy.linalg.expm(C.block_matrix(A0)) @ C.start_state(9)
    assert P.rel_fro(U[:9], (Q * np.sin(lam)) @ Q.T) < 1e-13
    assert P.rel_fro(U[9:], (Q * np.cos(lam)) @ Q.T) < 1e-13


@pytest.mark.parametrize("norm,m", [(0.3, 0), (1.0, 0), (1.5, 1), (5.0, 3), (8.0, 3), (8.5, 4)])
def test_scaling_exponent(norm, m):
    """Smallest m >= 0 with 2^-m ||A||_inf <= 1; ||A||_inf of a diagonal matrix is its largest |entry|."""
    A = np.diag([norm, -0.5 * norm, 0.1])
    assert C.scaling_exponent(A) == m


def test_double_angle_recovery_is_exact_on_exact_input():
    A, Q, lam = _sym(11, 2, 2.0)                 # ||A|| up to 8: m = 3 or so
    m = C.scaling_exponent(A)
    C0 = (Q * np.cos(lam * 2.0 ** -m)) @ Q.T
    assert m >= 2
    assert P.rel_fro(C.double_angle(C0, m), (Q * np.cos(lam)) @ Q.T) < 1e-13


def test_schemes_reach_the_cosine():
    """RK4 on eq. eqB with J = 40 per slice: cos(A) to the scheme's error; explicit Euler is first
    order (halving h halves the error)."""
    A, Q, lam = _sym(8, 3, 1.5)
    want = (Q * np.cos(lam)) @ Q.T
    c, s0, m, r = C.cos_algorithm5(A, 4, 40, 4, 0.0, method="classical", fine="rk4")
    assert r.iterations == 4 and P.rel_fro(c, want) < 1e-9
    e1 = P.rel_fro(C.cos_algorithm5(A, 4, 100, 4, 0.0, method="classical")[0], want)
    e2 = P.rel_fro(C.cos_algorithm5(A, 4, 200, 4, 0.0, method="classical")[0], want)
    assert 1.7 < e1 / e2 < 2.3


def test_example_3_modified_converges_faster_than_classical():
    """Example 3's setup (N = 10, J = 100, explicit Euler G and F): the modified algorithm reaches
    the sequential fine solution in fewer iterations than the classical one."""
    A, Q, lam = _sym(30, 4, 1.0)
    c_m, _, m, rm = C.cos_algorithm5(A, 10, 100, 10, 1e-10, method="modified")
    c_c, _, _, rc = C.cos_algorithm5(A, 10, 100, 10, 1e-10, method="classical")
    assert rm.iterations < rc.iterations
    assert P.rel_fro(c_m, c_c) < 1e-9


def _battery():
    try:
        test_block_flow_is_sine_and_cosine()
        for nm, m in [(0.3, 0), (1.0, 0), (1.5, 1), (5.0, 3), (8.0, 3), (8.5, 4)]:
            test_scaling_exponent(nm, m)
        test_double_angle_recovery_is_exact_on_exact_input()
        test_schemes_reach_the_cosine()
    except AssertionError:
        return False
    return True


def test_unmutated_cosine_oracle_passes_battery():
    assert _battery()


@pytest.mark.parametrize("mutation", ["double_angle_sign", "start_state", "scaling_fro",
                                      "block_transposed"])
def test_planted_mistakes_in_cosine_oracle_are_caught(monkeypatch, mutation):
    n_eye = np.eye
    if mutation == "double_angle_sign":
        def da(C0, m):
            Cm = C0
            for _ in range(m):
                Cm = 2.0 * (Cm @ Cm) + n_eye(C0.shape[0])
            return Cm
        monkeypatch.setattr(C, "double_angle", da)
    elif mutation == "start_state":
        monkeypatch.setattr(C, "start_state", lambda n: np.vstack([np.eye(n), np.zeros((n, n))]))
    elif mutation == "scaling_fro":
        def se(A):
            a, m = float(np.linalg.norm(A)), 0
            while a > 1.0:
                a *= 0.5
                m += 1
            return m
        monkeypatch.setattr(C, "scaling_exponent", se)
    else:
        real = C.block_matrix
        monkeypatch.setattr(C, "block_matrix", lambda A0: real(A0).T)
    assert not _battery(), mutation
