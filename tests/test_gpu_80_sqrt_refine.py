"""Square-root refinement on the GPU: Newton steps whose Sylvester equations are solved by the
tensor-core sign iteration, against the oracle's Newton step (exact Sylvester solve in the
eigenbasis) and against A^{1/2}."""
import numpy as np
import pytest

from oracle import closed, parareal as P, refine as RF, scalar as S
from paper_1505_07959_gb300 import fa, inputs
from tests.gpu_helpers import cuda_or_fail, dev, host

pytestmark = pytest.mark.gpu


def _flow_state(n, seed, noise):
    """The exact flow state X(20) from X(0) = I (not yet A^{1/2} for small eigenvalues), plus a
    symmetric perturbation of relative size `noise` (a BF16-level flow error)."""
    sm = inputs.sym_matrix(n, "sqrt", seed)
    X = S.to_matrix(sm.Q, closed.scalar_solution(2, sm.lam, 20.0))
    E = inputs.sym_matrix(n, "exp", seed + 1).A
    X = X + noise * np.linalg.norm(X) / np.linalg.norm(E) * E
    return sm, X


@pytest.mark.parametrize("n", [64, 200])
def test_refinement_matches_oracle_newton(n):
    cuda_or_fail()
    sm, X0 = _flow_state(n, 7 + n, 1e-3)
    exact = S.to_matrix(sm.Q, np.sqrt(sm.lam))
    assert P.rel_fro(X0, exact) > 1e-2                 # far from A^{1/2} before refinement
    for steps in (1, 2, 4):
        plan = fa.Plan(n, fa.FA_FLOW_SQRT, 20.0, 4, 2, coarse_steps=2, fine_dtype="bf16x6",
                       refine_steps=steps)
        plan.set_matrix(dev(sm.A))
        X = plan.refine(dev(X0))
        want = RF.newton_sylvester_sqrt(sm.A, X0, steps)
        err_o = P.rel_fro(want, exact)
        got = host(X)
        # each Newton step's Sylvester solution is accurate to ~1e-7 relative (BF16x6 products),
        # which adds ~1e-7 of the step's correction (at most ~2e-2 of X) to the oracle's step
        assert P.rel_fro(got, want) <= 1e-6, (steps, P.rel_fro(got, want), err_o)
        assert np.array_equal(got, got.T)
        if steps == 4:
            assert P.rel_fro(got, exact) < 1e-10
        plan.close()


def test_refinement_is_deterministic():
    cuda_or_fail()
    n = 136
    sm, X0 = _flow_state(n, 3, 1e-2)
    plan = fa.Plan(n, fa.FA_FLOW_SQRT, 20.0, 4, 2, coarse_steps=2, fine_dtype="bf16", refine_steps=3)
    plan.set_matrix(dev(sm.A))
    a = host(plan.refine(dev(X0)))
    b = host(plan.refine(dev(X0)))
    assert np.array_equal(a, b)
    plan.close()


@pytest.mark.parametrize("dtype", ["bf16", "bf16x6"])
def test_mixed_sqrt_solve_with_refinement_reaches_the_square_root(dtype):
    """The square-root flow to T = 20 with BF16-term products, then five Newton steps: the
    flow's own error (~1e-2 from the unfinished transient of small eigenvalues, plus the BF16
    error) goes to <= 1e-10 against A^{1/2}."""
    cuda_or_fail()
    n, T, N, J = 256, 20.0, 32, 8
    sm = inputs.sym_matrix(n, "sqrt", 11)
    exact = S.to_matrix(sm.Q, np.sqrt(sm.lam))
    plan = fa.Plan(n, fa.FA_FLOW_SQRT, T, N, J, coarse_steps=2, fine_dtype=dtype, max_iters=6,
                   tol=0.0, refine_steps=5)
    X, rep = plan.solve(dev(sm.A))
    assert rep["iters"] == 6 and rep["t_refine_ms"] > 0
    assert P.rel_fro(host(X), exact) < 1e-10
    plan.close()


def test_exp_flow_has_no_refinement():
    cuda_or_fail()
    plan = fa.Plan(32, fa.FA_FLOW_EXP, 1.0, 2, 2, refine_steps=1)
    plan.set_matrix(dev(inputs.sym_matrix(32, "exp", 1).A))
    with pytest.raises(fa.FaError) as e:
        plan.refine(dev(np.eye(32)))
    assert e.value.status == 7
    plan.close()


def test_refinement_at_the_square_root_workloads_order():
    """n = 4096 (the square-root workload: lam log-U[1e-3, 1], the flow state at T = 20 from
    X(0) = I, plus BF16-level symmetric noise): one Newton step against the oracle's exact-
    Sylvester Newton step, and four steps against A^{1/2}."""
    cuda_or_fail()
    n = 4096
    sm, X0 = _flow_state(n, 0, 1e-3)
    exact = S.to_matrix(sm.Q, np.sqrt(sm.lam))
    for steps in (1, 4):
        plan = fa.Plan(n, fa.FA_FLOW_SQRT, 20.0, 1, 1, coarse_steps=2, fine_dtype="bf16",
                       refine_steps=steps)
        plan.set_matrix(dev(sm.A))
        got = host(plan.refine(dev(X0)))
        plan.close()
        assert np.array_equal(got, got.T)
        if steps == 1:
            want = RF.newton_sylvester_sqrt(sm.A, X0, 1)
            assert P.rel_fro(got, want) <= 1e-6, P.rel_fro(got, want)
        else:
            assert P.rel_fro(got, exact) < 1e-10, P.rel_fro(got, exact)
