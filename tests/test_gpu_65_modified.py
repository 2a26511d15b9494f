"""The modified parareal (Algorithm 3, Section 3) on the GPU against the oracle's statement of it
(oracle.modified), against the sequential fine solution, and against exp(A).

Float64: the same iterations and space as the oracle, the result within 1e-12.  BF16x6: the
result within 1e-6 of exp(A) (the bound of the split products).  The full-size case is the
exponential workload (n = 2048, N = 64, J = 64) with the modified method."""
import time

import numpy as np
import pytest

from gpu_helpers import cuda_or_fail, dev, fa, host, rel, torch
from oracle import modified as M, parareal as orc, scalar as S
from paper_1505_07959_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    cuda_or_fail()


def _plan(n, N, J, m, K, tol, dtype, **kw):
    return fa.Plan(n, fa.FA_FLOW_EXP, 1.0, N, fine_steps=J, coarse_steps=m, max_iters=K, tol=tol,
                   fine_dtype=dtype, method=fa.FA_METHOD_MODIFIED, **kw)


@pytest.mark.parametrize("n,N,J,m", [(64, 16, 16, 1), (100, 7, 4, 2), (33, 5, 3, 1)])
def test_modified_f64_matches_oracle(n, N, J, m):
    sm = inputs.sym_matrix(n, "exp", 50 + n)
    t_o = time.perf_counter()
    ref = M.modified_parareal(sm.A, 1, 1.0, N, m, J, N, 1e-10, drop=1e-12)
    t_o = time.perf_counter() - t_o
    seq = orc.sequential_fine(sm.A, 1, 1.0, N, J)
    plan = _plan(n, N, J, m, N, 1e-10, "f64", span_drop=1e-12, max_basis=(N + 1) * N)
    X, rep = plan.solve(dev(sm.A))
    X = host(X)
    plan.close()
    print(f"modified f64 n={n} N={N} J={J}: {rep['iters']} iterations, space {rep['basis_dim']}, "
          f"device {rep['t_init_ms'] + rep['t_fine_ms'] + rep['t_coarse_ms']:.1f} ms "
          f"(oracle on the host {t_o * 1e3:.0f} ms)")
    assert rep["converged"]
    assert rep["iters"] == ref.iterations
    assert rep["basis_dim"] == len(ref.basis)
    assert rep["fine_blocks"] == sum(ref.new_blocks)
    assert rel(X, ref.U[N]) < 1e-12
    assert rel(X, seq) < 1e-12
    for a, b in zip(rep["dx_history"][:-1], ref.dx_history[:-1]):
        assert abs(a - b) <= 1e-6 * b


def test_modified_finite_termination_f64():
    """K iterations make slices 0..K exact (as in Algorithm 1): with the tolerance off and
    K = N the result is the sequential fine solution."""
    n, N, J = 40, 5, 6
    sm = inputs.sym_matrix(n, "exp", 12)
    seq = orc.sequential_fine(sm.A, 1, 1.0, N, J)
    plan = _plan(n, N, J, 1, N, 0.0, "f64", max_basis=(N + 1) * N)
    X, rep = plan.solve(dev(sm.A))
    assert rep["iters"] == N
    assert rel(host(X), seq) < 1e-12
    plan.close()


@pytest.mark.parametrize("dtype", ["bf16x6", "bf16x4"])
def test_modified_mixed_reaches_exp(dtype):
    n, N, J = 256, 16, 16
    sm = inputs.sym_matrix(n, "exp", 7)
    ex = (sm.Q * np.exp(sm.lam)) @ sm.Q.T
    plan = _plan(n, N, J, 1, N, 1e-8, dtype)
    X, rep = plan.solve(dev(sm.A))
    plan.close()
    cl = orc.parareal(sm.A, 1, 1.0, N, 1, J, N, 1e-10)
    assert rep["converged"]
    assert rep["iters"] <= 4
    assert rep["fine_blocks"] < cl.iterations * N / 4
    bound = 1e-6 if dtype == "bf16x6" else 2e-5
    assert rel(host(X), ex) < bound, rel(host(X), ex)


def test_modified_is_bitwise_deterministic():
    n, N, J = 130, 8, 4
    sm = inputs.sym_matrix(n, "exp", 3)
    plan = _plan(n, N, J, 1, N, 1e-9, "bf16x6")
    a, ra = plan.solve(dev(sm.A))
    a = host(a).copy()
    b, rb = plan.solve(dev(sm.A))
    assert np.array_equal(a, host(b))
    assert ra["basis_dim"] == rb["basis_dim"]
    plan.close()


def test_modified_space_capacity_is_respected():
    n, N, J = 64, 8, 4
    sm = inputs.sym_matrix(n, "exp", 4)
    plan = _plan(n, N, J, 1, N, 0.0, "f64", max_basis=3)
    X, rep = plan.solve(dev(sm.A))
    assert rep["basis_dim"] == 3 and rep["fine_blocks"] == 3
    # slices the capped space still covers converge; the iteration stays finite and bounded
    assert np.all(np.isfinite(host(X)))
    plan.close()


def test_modified_rejects_nonlinear_flows():
    with pytest.raises(fa.FaError) as e:
        fa.Plan(16, fa.FA_FLOW_INV, 1.0, 2, fine_steps=2, method=fa.FA_METHOD_MODIFIED)
    assert e.value.status == 7


def test_modified_exp_workload_full_size():
    """The exponential workload (n = 2048, lam ~ U[-4, 0], N = 64, J = 64, Euler G) with the
    modified method and BF16x6 products: error vs exp(A) <= 1e-6, against the oracle's RK4 fine
    solution evaluated in the eigenbasis (exact for X0 = I) on the whole matrix."""
    w = inputs.EXP_N2048
    sm = inputs.sym_matrix(w.n, w.kind, w.seed)
    plan = _plan(w.n, w.N, w.J, w.m, 8, w.mixed_tol, "bf16x6")
    A = dev(sm.A)
    X, rep = plan.solve(A)                       # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, rep = plan.solve(A)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    Xh = host(X)
    ex = (sm.Q * np.exp(sm.lam)) @ sm.Q.T
    seq = S.to_matrix(sm.Q, S.sequential_fine(sm.lam, w.flow, w.T, w.N, w.J))
    print(f"modified exp n=2048: {dt * 1e3:.0f} ms/solve, iterations {rep['iters']}, "
          f"space {rep['basis_dim']}, fine blocks {rep['fine_blocks']}, "
          f"err vs exp {rel(Xh, ex):.2e}, vs fine {rel(Xh, seq):.2e}, dx {rep['dx_history']}")
    plan.close()
    assert rep["converged"]
    assert rel(Xh, ex) < 1e-6
    assert rel(Xh, seq) < 1e-6
