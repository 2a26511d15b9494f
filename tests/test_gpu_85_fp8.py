"""E4M3 fine sweeps of the square-root flow (per-tile delayed scaling) against the oracle, and
whole E4M3 solves refined to A^{1/2}."""
import numpy as np
import pytest

from oracle import closed, parareal as P, scalar as S
from paper_1505_07959_gb300 import fa, inputs
from tests.gpu_helpers import cuda_or_fail, dev, host

pytestmark = pytest.mark.gpu

# E4M3 keeps 3 mantissa bits: each operand entry carries up to 2^-4 relative rounding, so a
# stage product A - Y^2 is off by ~1e-2 of |Y|^2 and an RK4 step by ~h * 1e-2 of the state's
# rate of change; over one slice (dT = T / N) the state is off by a few 1e-3 relative.  The
# bound below is 2^-5.
SWEEP_TOL_FP8 = 2.0 ** -5


@pytest.mark.parametrize("n", [136, 256])
def test_fp8_fine_sweep_matches_oracle(n):
    cuda_or_fail()
    T, N, J = 20.0, 8, 8
    sm = inputs.sym_matrix(n, "sqrt", 31 + n)
    dT = T / N
    # states on the flow (the scalar solution at the slice times): finite, SPD, realistic
    U = np.array([S.to_matrix(sm.Q, closed.scalar_solution(2, sm.lam, b * dT)) for b in range(N)])
    plan = fa.Plan(n, fa.FA_FLOW_SQRT, T, N, J, coarse_steps=2, fine_dtype="fp8e4m3",
                   coarse_dtype="bf16x6")
    plan.set_matrix(dev(sm.A))
    F = host(plan.fine_sweep(dev(U)))
    for b in range(N):
        want = P.rk4(2, U[b], sm.A, dT, J)
        err = P.rel_fro(F[b], want)
        assert err < SWEEP_TOL_FP8, (b, err)
    # the E4M3 operands are in use: the result differs from the BF16x6 sweep's
    plan2 = fa.Plan(n, fa.FA_FLOW_SQRT, T, N, J, coarse_steps=2, fine_dtype="bf16x6")
    plan2.set_matrix(dev(sm.A))
    F2 = host(plan2.fine_sweep(dev(U)))
    assert P.rel_fro(F, F2) > 1e-5
    plan.close()
    plan2.close()


def test_fp8_sweep_is_deterministic():
    cuda_or_fail()
    n, T, N, J = 200, 20.0, 2, 2
    sm = inputs.sym_matrix(n, "sqrt", 3)
    plan = fa.Plan(n, fa.FA_FLOW_SQRT, T, N, J, coarse_steps=8, fine_dtype="fp8e4m3",
                   coarse_dtype="bf16x6")
    plan.set_matrix(dev(sm.A))
    U = dev(np.array([np.eye(n), 0.5 * np.eye(n) + 0.1 * sm.A]))
    a = host(plan.fine_sweep(U))
    b = host(plan.fine_sweep(U))
    assert np.array_equal(a, b)
    plan.close()


@pytest.mark.parametrize("coarse", ["bf16x6", "f64"])
def test_fp8_solve_with_refinement_reaches_the_square_root(coarse):
    cuda_or_fail()
    n, T, N, J = 256, 20.0, 16, 8
    sm = inputs.sym_matrix(n, "sqrt", 11)
    exact = S.to_matrix(sm.Q, np.sqrt(sm.lam))
    plan = fa.Plan(n, fa.FA_FLOW_SQRT, T, N, J, coarse_steps=2, fine_dtype="fp8e4m3",
                   coarse_dtype=coarse, max_iters=6, tol=0.0, refine_steps=5)
    X, rep = plan.solve(dev(sm.A))
    assert rep["iters"] == 6
    # the flow state alone: the transient of the smallest eigenvalues (~2e-2) plus E4M3 error
    x20 = S.to_matrix(sm.Q, closed.scalar_solution(2, sm.lam, T))
    assert P.rel_fro(host(X), exact) < 1e-10
    plan.close()
    plan0 = fa.Plan(n, fa.FA_FLOW_SQRT, T, N, J, coarse_steps=2, fine_dtype="fp8e4m3",
                    coarse_dtype=coarse, max_iters=6, tol=0.0)
    X0, _ = plan0.solve(dev(sm.A))
    assert P.rel_fro(host(X0), x20) < 5e-2
    plan0.close()


def test_fp8_is_square_root_only():
    cuda_or_fail()
    with pytest.raises(fa.FaError) as e:
        fa.Plan(64, fa.FA_FLOW_INV, 1.0, 2, 2, fine_dtype="fp8e4m3", coarse_dtype="bf16x6")
    assert e.value.status == 7
    with pytest.raises(fa.FaError) as e:
        fa.Plan(64, fa.FA_FLOW_SQRT, 20.0, 16, 2, coarse_steps=2, fine_dtype="fp8e4m3",
                coarse_dtype="fp8e4m3")
    assert e.value.status == 1
