"""cos(A) by Algorithm 5 (Section 3, Example 3) on the GPU (FA_FLOW_COS): the block flow of
eq. eqB by classical or modified parareal, then the double-angle recovery, against the oracle's
statement (oracle.cosine) and against cos(A) from the eigendecomposition."""
import time

import numpy as np
import pytest

from gpu_helpers import cuda_or_fail, dev, fa, host, rel, torch
from oracle import cosine as C
from paper_1505_07959_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    cuda_or_fail()


def _sym(n, seed, scale):
    sm = inputs.sym_matrix(n, "exp", seed)       # eigenvalues in [-4 scale, 0]
    return sm.A * scale, sm.Q, sm.lam * scale


def _plan(n, N, J, K, tol, dtype, method, fine="euler", **kw):
    return fa.Plan(n, fa.FA_FLOW_COS, 1.0, N, fine_steps=J, coarse_steps=1, max_iters=K, tol=tol,
                   fine_dtype=dtype, method=method, fine_scheme=fine, **kw)


@pytest.mark.parametrize("method", [fa.FA_METHOD_CLASSICAL, fa.FA_METHOD_MODIFIED])
def test_example_3_setup_float64_matches_oracle(method):
    """Example 3's setup (N = 10, J = 100, explicit Euler G and F) on a ragged n: the same
    iterations, double-angle steps and result as the oracle (1e-12)."""
    n = 50
    A, Q, lam = _sym(n, 5, 1.2)
    name = "modified" if method == fa.FA_METHOD_MODIFIED else "classical"
    t_o = time.perf_counter()
    c_ref, _, m, r = C.cos_algorithm5(A, 10, 100, 10, 1e-10, method=name, drop=1e-12)
    t_o = time.perf_counter() - t_o
    plan = _plan(n, 10, 100, 10, 1e-10, "f64", method, span_drop=1e-12, max_basis=44)
    dA = dev(A)
    plan.solve(dA)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, rep = plan.solve(dA)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    plan.close()
    X = host(X)
    print(f"cos Example 3 setup n={n} {name}: {rep['iters']} iterations, {dt * 1e3:.1f} ms "
          f"(oracle on the host {t_o * 1e3:.0f} ms)")
    assert rep["double_angle_steps"] == m >= 1
    assert rep["iters"] == r.iterations
    assert rel(X, c_ref) < 1e-12
    assert rel(X, (Q * np.cos(lam)) @ Q.T) < 5e-3          # explicit Euler (h = 1e-3), amplified by the recovery


def test_modified_needs_fewer_iterations_on_example_3():
    n = 64
    A, Q, lam = _sym(n, 6, 1.0)
    reps = {}
    for method in (fa.FA_METHOD_CLASSICAL, fa.FA_METHOD_MODIFIED):
        plan = _plan(n, 10, 100, 10, 1e-10, "f64", method)
        X, reps[method] = plan.solve(dev(A))
        plan.close()
    assert reps[fa.FA_METHOD_MODIFIED]["iters"] < reps[fa.FA_METHOD_CLASSICAL]["iters"]


@pytest.mark.parametrize("dtype,tol", [("bf16x6", 1e-6)])
def test_cosine_rk4_mixed_at_scale(dtype, tol):
    """n = 1024, ||A|| up to 8 (three double-angle steps), RK4 F with the modified method: cos(A)
    from the eigendecomposition within the split products' bound (the recovery amplifies the
    error of C_0 by about 4^m)."""
    n = 1024
    A, Q, lam = _sym(n, 7, 2.0)
    plan = _plan(n, 16, 16, 6, 1e-8, dtype, fa.FA_METHOD_MODIFIED, fine="rk4")
    dA = dev(A)
    X, rep = plan.solve(dA)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, rep = plan.solve(dA)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    plan.close()
    err = rel(host(X), (Q * np.cos(lam)) @ Q.T)
    print(f"cos n=1024 {dtype}: {dt * 1e3:.0f} ms, m = {rep['double_angle_steps']}, "
          f"iterations {rep['iters']}, space {rep['basis_dim']}, err vs cos(A) {err:.2e}")
    assert rep["double_angle_steps"] == C.scaling_exponent(A)
    assert err < 64 * tol


def test_cosine_plan_rejects_other_calls():
    plan = _plan(16, 2, 2, 2, 0.0, "f64", fa.FA_METHOD_CLASSICAL)
    with pytest.raises(fa.FaError) as e:
        plan.fine_sweep(np.zeros((2, 16, 16)))
    assert e.value.status == 7
    plan.close()
