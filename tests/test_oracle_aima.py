"""Pins of the accelerated inverse-matrix oracle (Algorithm 8, Section 4) against closed forms of
the iteration on a symmetric matrix, and the acceleration the paper reports (Example 5)."""
import numpy as np
import pytest

from oracle import aima as AI
from paper_1505_07959_gb300 import inputs


def _spd(n, seed):
    sm = inputs.sym_matrix(n, "inv", seed)
    return sm.A, sm.Q, sm.lam


def test_without_control_it_is_euler_on_the_steady_state_flow():
    """u = 0: X^(k) = A^{-1} + (I - dt A)^k (X0 - A^{-1}) (explicit Euler for dX/dt = I - A X)."""
    A, Q, lam = _spd(12, 1)
    X0 = 0.1 * np.eye(12)
    dt, k = 0.3, 7
    X, res = AI.aima(A, X0, np.zeros((12, 12)), dt, k)
    Ainv = (Q / lam) @ Q.T
    want = Ainv + (Q * (1 - dt * lam) ** k) @ Q.T @ (X0 - Ainv)
    assert np.allclose(X, want, rtol=0, atol=1e-13)
    assert len(res) == k + 1 and abs(res[0] - np.linalg.norm(np.eye(12) - A @ X0)) < 1e-13


def test_exact_initial_error_closed_form():
    """e = A^{-1} - X0 exactly: E^(k) = X^(k) - A^{-1} = (I - dt A)^(k-1) (I - dt A - k dt I) E^(0)
    (from E^(k+1) = (I - dt A) E^(k) - dt (I - dt A)^k E^(0))."""
    A, Q, lam = _spd(10, 2)
    Ainv = (Q / lam) @ Q.T
    X0 = np.zeros((10, 10))
    dt = 0.05
    for k in (1, 5, 20):
        X, _ = AI.aima(A, X0, Ainv - X0, dt, k)
        f = (1 - dt * lam) ** (k - 1) * (1 - dt * lam - k * dt)
        want = Ainv + (Q * f) @ Q.T @ (X0 - Ainv)
        assert np.allclose(X, want, rtol=0, atol=1e-12), k


def test_acceleration_on_example_5():
    """Example 5 (grid Laplacian scaled by its Frobenius norm, X0 = 0, dt = 0.1): after t = 1
    (10 steps) the residual ||I - A X|| with the exact initial error is far below the one without
    control, and the thresholded estimate (entries of A^{-1} below 1 % dropped) also gains."""
    A, X0, e_thr = inputs.aima_example(m=15, threshold=0.01)
    _, _, e_ex = inputs.aima_example(m=15, threshold=0.0)
    dt, k = 0.1, 10
    _, r0 = AI.aima(A, X0, np.zeros_like(A), dt, k)
    _, rt = AI.aima(A, X0, e_thr, dt, k)
    _, rx = AI.aima(A, X0, e_ex, dt, k)
    assert rx[-1] < 1e-2 * r0[-1]
    assert rt[-1] < 0.5 * r0[-1]


def _battery():
    try:
        test_without_control_it_is_euler_on_the_steady_state_flow()
        test_exact_initial_error_closed_form()
        test_acceleration_on_example_5()
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("mutation", ["control_sign", "control_not_decayed", "residual_sign"])
def test_planted_mistakes_in_aima_oracle_are_caught(monkeypatch, mutation):
    def aima(A, X0, e, dt, steps):
        n = A.shape[0]
        I = np.eye(n)
        X, u = X0.copy(), e.copy()
        res = [float(np.linalg.norm(I - A @ X))]
        for _ in range(steps):
            if mutation == "control_sign":
                X, u = X + dt * (I - A @ X - u), u - dt * (A @ u)
            elif mutation == "control_not_decayed":
                X, u = X + dt * (I - A @ X + u), u
            else:
                X, u = X + dt * (I + A @ X + u), u - dt * (A @ u)
            res.append(float(np.linalg.norm(I - A @ X)))
        return X, res
    monkeypatch.setattr(AI, "aima", aima)
    assert not _battery(), mutation


def test_unmutated_aima_oracle_passes_battery():
    assert _battery()
