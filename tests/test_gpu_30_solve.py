"""fa_parareal_solve against the oracle's Algorithm 1: same inputs, same iteration count,
element-by-element agreement (float64: 1e-12; mixed forms: their stated bound), plus the
invariants (finite termination, determinism) and the error paths."""
import numpy as np
import pytest

from gpu_helpers import cuda_or_fail, dev, fa, host, rel, torch
from oracle import closed, parareal as orc
from paper_1505_07959_gb300 import inputs

pytestmark = pytest.mark.gpu

FLOWS = [(fa.FA_FLOW_INV, "inv", 1.0, 1), (fa.FA_FLOW_EXP, "exp", 1.0, 1),
         (fa.FA_FLOW_SQRT, "sqrt", 8.0, 2)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    cuda_or_fail()


def test_tiny_inverse_workload_f64():
    """n=64 inverse flow, lam~U[0.5,2], N=8, J=16, K<=8, float64: oracle parity and A^{-1}."""
    w = inputs.INV_N64
    sm = inputs.sym_matrix(w.n, w.kind, w.seed)
    ref = orc.parareal(sm.A, w.flow, w.T, w.N, w.m, w.J, w.K_max, w.tol)
    plan = fa.Plan(w.n, w.flow, w.T, w.N, fine_steps=w.J, coarse_steps=w.m, max_iters=w.K_max,
                   tol=w.tol, fine_dtype="f64")
    X, rep = plan.solve(dev(sm.A))
    X = host(X)
    assert rep["iters"] == ref.iterations
    assert rel(X, ref.U[w.N]) < 1e-12
    assert rel(X, closed.inv_lu(sm.A)) < 1e-10
    # the paper's own error measure (Section 2, Example 1): max_ij |E_ij| / max_ij |A_ij|
    assert orc.paper_norm(X - ref.U[w.N], sm.A) < 1e-12
    assert orc.paper_norm(X - closed.inv_lu(sm.A), sm.A) < 1e-10
    for a, b in zip(rep["dx_history"], ref.dx_history):
        assert abs(a - b) <= 1e-8 * b + 1e-15


@pytest.mark.parametrize("flow,kind,T,m", FLOWS)
def test_solve_f64_ragged(flow, kind, T, m):
    n, N, J = 100, 4, 8
    sm = inputs.sym_matrix(n, kind, 11)
    ref = orc.parareal(sm.A, flow, T, N, m, J, 4, 0.0)
    plan = fa.Plan(n, flow, T, N, fine_steps=J, coarse_steps=m, max_iters=4, tol=0.0,
                   fine_dtype="f64")
    X, rep = plan.solve(dev(sm.A))
    assert rep["iters"] == 4
    assert rel(host(X), ref.U[N]) < 1e-12


@pytest.mark.parametrize("flow,kind,T,m", FLOWS)
def test_finite_termination_f64(flow, kind, T, m):
    """K = N iterations reproduce the sequential fine solution."""
    n, N, J = 40, 5, 6
    sm = inputs.sym_matrix(n, kind, 12)
    seq = orc.sequential_fine(sm.A, flow, T, N, J)
    plan = fa.Plan(n, flow, T, N, fine_steps=J, coarse_steps=m, max_iters=N, tol=0.0,
                   fine_dtype="f64")
    X, rep = plan.solve(dev(sm.A))
    assert rep["iters"] == N
    assert rel(host(X), seq) < 1e-12


# Relative error of a mixed solve vs the oracle.  BF16X6 keeps both operands to float32
# precision and drains the main product every k-block, so the solve stays near the
# float32 level (bound 1e-6).  BF16X4 keeps the right operand to two BF16 terms
# (~2^-18 = 3.8e-6 per element); over T ||Fl'|| <= 8 (square root, T = 8) that allows
# up to ~3e-5, bound 1e-5 on these inputs.
SOLVE_TOL = {"bf16x4": 1e-5, "bf16x6": 1e-6}


@pytest.mark.parametrize("dtype", ["bf16x4", "bf16x6"])
@pytest.mark.parametrize("flow,kind,T,m", FLOWS)
def test_solve_mixed(dtype, flow, kind, T, m):
    n, N, J = 200, 8, 16
    sm = inputs.sym_matrix(n, kind, 13)
    ref = orc.parareal(sm.A, flow, T, N, m, J, 8, 1e-10)
    plan = fa.Plan(n, flow, T, N, fine_steps=J, coarse_steps=m, max_iters=8, tol=1e-10,
                   fine_dtype=dtype)
    X, rep = plan.solve(dev(sm.A))
    e = rel(host(X), ref.U[N])
    print(f"solve {dtype} flow={kind}: iters {rep['iters']} (oracle {ref.iterations}) err {e:.2e}")
    assert e < SOLVE_TOL[dtype]
    assert abs(rep["iters"] - ref.iterations) <= 1


def test_mixed_coarse_f64_fine_bf16():
    n, N, J = 128, 6, 8
    sm = inputs.sym_matrix(n, "exp", 14)
    ref = orc.parareal(sm.A, fa.FA_FLOW_EXP, 1.0, N, 1, J, 6, 1e-10)
    plan = fa.Plan(n, fa.FA_FLOW_EXP, 1.0, N, fine_steps=J, max_iters=6, tol=1e-10,
                   fine_dtype="bf16x6", coarse_dtype="f64")
    X, rep = plan.solve(dev(sm.A))
    assert rel(host(X), ref.U[N]) < 1e-6


def test_solve_is_bitwise_deterministic_and_host_equals_device():
    n, N, J = 256, 4, 8
    sm = inputs.sym_matrix(n, "exp", 15)
    plan = fa.Plan(n, fa.FA_FLOW_EXP, 1.0, N, fine_steps=J, max_iters=4, tol=0.0,
                   fine_dtype="bf16x4")
    X1, _ = plan.solve(dev(sm.A))
    X2, _ = plan.solve(dev(sm.A))
    X3, rep = plan.solve_host(sm.A)
    X1, X2 = host(X1), host(X2)
    assert np.array_equal(X1, X2)
    assert np.array_equal(X1, X3)
    assert rep["iters"] == 4


def test_newton_schulz_refinement_recovers_inverse_from_bf16():
    """One-term BF16 products leave ~1e-3 error; three float64 Newton-Schulz steps fix it."""
    n, N, J = 160, 4, 8
    sm = inputs.sym_matrix(n, "inv", 16)
    plan0 = fa.Plan(n, fa.FA_FLOW_INV, 1.0, N, fine_steps=J, max_iters=4, tol=0.0,
                    fine_dtype="bf16")
    X0, _ = plan0.solve(dev(sm.A))
    e0 = rel(host(X0), closed.inv_lu(sm.A))
    plan = fa.Plan(n, fa.FA_FLOW_INV, 1.0, N, fine_steps=J, max_iters=4, tol=0.0,
                   fine_dtype="bf16", refine_steps=3)
    X, rep = plan.solve(dev(sm.A))
    e3 = rel(host(X), closed.inv_lu(sm.A))
    print(f"bf16 inverse: before refinement {e0:.2e}, after 3 Newton-Schulz steps {e3:.2e}")
    assert e0 > 1e-5
    assert e3 < 1e-12
    # the float64 refinement alone, through fa_refine, on the same start
    plan.set_matrix(dev(sm.A))
    from oracle import refine as oref
    Xr = host(plan.refine(X0))
    assert rel(Xr, oref.newton_schulz_inv(sm.A, host(X0), 3)) < 1e-12


def test_nonfinite_input_is_reported():
    n = 32
    A = np.eye(n)
    A[3, 5] = np.nan
    plan = fa.Plan(n, fa.FA_FLOW_EXP, 1.0, 2, fine_steps=2, max_iters=2, tol=0.0,
                   fine_dtype="bf16x4")
    with pytest.raises(fa.FaError) as ei:
        plan.solve(dev(A))
    assert ei.value.status == 4


def test_not_converged_is_reported_with_output():
    n = 48
    sm = inputs.sym_matrix(n, "inv", 17)
    plan = fa.Plan(n, fa.FA_FLOW_INV, 1.0, 6, fine_steps=4, max_iters=1, tol=1e-14,
                   fine_dtype="f64")
    X, rep = plan.solve(dev(sm.A))
    assert rep["status"] == fa.FA_ERR_NOT_CONVERGED and not rep["converged"]
    ref = orc.parareal(sm.A, fa.FA_FLOW_INV, 1.0, 6, 1, 4, 1, 0.0)
    assert rel(host(X), ref.U[6]) < 1e-12
