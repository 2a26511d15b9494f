"""Algorithm 8 (accelerated inverse-matrix approximation, Section 4) on the GPU through fa_aima,
against the oracle (oracle.aima): the iterate and the residual history ||I - A X^(k)||_F.
Float64 products: 1e-12; BF16x6 products: the split form's bound.  Example 5's matrix (the
63 x 63 grid Laplacian over its Frobenius norm, order 3969) runs at full size."""
import time

import numpy as np
import pytest

from gpu_helpers import cuda_or_fail, dev, fa, host, rel, torch
from oracle import aima as AI
from paper_1505_07959_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    cuda_or_fail()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("bf16x6", 1e-6)])
@pytest.mark.parametrize("n", [100, 257])
def test_aima_matches_oracle(n, dtype, tol):
    sm = inputs.sym_matrix(n, "inv", 70 + n)
    A = sm.A
    Ainv = np.linalg.inv(A)
    e = np.where(np.abs(Ainv) >= 0.05 * np.abs(Ainv).max(), Ainv, 0.0)
    X0 = np.zeros((n, n))
    dt, steps = 0.3, 25
    Xr, rr = AI.aima(A, X0, e, dt, steps)
    ai = fa.Aima(n, dtype)
    X, res = ai.run(A, X0, e, dt, steps)
    ai.close()
    X = host(X)
    assert rel(X, Xr) < tol, rel(X, Xr)
    np.testing.assert_allclose(res, rr, rtol=max(tol, 1e-10) * 100, atol=tol * 10)
    assert res[-1] < 0.5 * res[0]


def test_aima_without_control_is_the_euler_iteration():
    n = 64
    sm = inputs.sym_matrix(n, "inv", 3)
    X0 = 0.2 * np.eye(n)
    ai = fa.Aima(n, "f64")
    X, res = ai.run(sm.A, X0, np.zeros((n, n)), 0.25, 9)
    ai.close()
    Ainv = (sm.Q / sm.lam) @ sm.Q.T
    want = Ainv + (sm.Q * (1 - 0.25 * sm.lam) ** 9) @ sm.Q.T @ (X0 - Ainv)
    assert rel(host(X), want) < 1e-12


def test_aima_rejects_bad_arguments():
    ai = fa.Aima(16, "f64")
    z = np.zeros((16, 16))
    with pytest.raises(fa.FaError):
        ai.run(np.eye(16), z, z, -0.1, 3)
    with pytest.raises(fa.FaError):
        ai.run(np.eye(16), z, z, 0.1, 16 * 16)
    ai.close()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("bf16x6", 1e-5)])
def test_aima_example_5_full_size(dtype, tol):
    """Example 5 (m = 63, order 3969, dt = 0.1, X0 = 0, e from A^{-1} thresholded at 1 %): 10
    steps (t = 1) against the oracle, and the acceleration over the uncontrolled iteration.  As
    printed, Algorithm 8 never switches the control off, so the residual is smallest at t = 1
    (with the exact e: E_k = (I - dt A)^(k-1) (I - dt A - k dt) E_0) and grows afterwards."""
    A, X0, e = inputs.aima_example(63, 0.01)
    steps, dt = 10, 0.1
    t_o = time.perf_counter()
    Xr, rr = AI.aima(A, X0, e, dt, steps)
    t_o = time.perf_counter() - t_o
    ai = fa.Aima(A.shape[0], dtype)
    X, res = ai.run(A, X0, e, dt, steps)          # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, res = ai.run(A, X0, e, dt, steps)
    torch.cuda.synchronize()
    dtm = time.perf_counter() - t0
    _, res0 = ai.run(A, X0, np.zeros_like(A), dt, steps)
    ai.close()
    X = host(X)
    print(f"AIMA example 5 ({dtype}): {dtm / steps * 1e3:.2f} ms per step (oracle on the host "
          f"{t_o / steps * 1e3:.0f} ms), residual "
          f"{res[0]:.3e} -> {res[-1]:.3e} (uncontrolled {res0[-1]:.3e}), X vs oracle {rel(X, Xr):.2e}")
    assert rel(X, Xr) < tol
    assert abs(res[-1] - rr[-1]) <= tol * 100 * rr[0]
    assert res[-1] < 0.5 * res0[-1]
