"""The propagators' time-stepping schemes on the GPU: explicit-Euler F (Section 2, Example 1)
and Crank-Nicolson F and G (Example 2), against the oracle's statement of each (float64: 1e-12;
BF16x6: the split products' bound), and the paper's own example setups end to end (n = 80
Laplacian / 2^10, N = 25, J = 200) with the paper's error measure."""
import time

import numpy as np
import pytest
import scipy.linalg

from gpu_helpers import cuda_or_fail, dev, fa, host, rel, torch
from oracle import closed, modified as M, parareal as orc
from paper_1505_07959_gb300 import inputs

pytestmark = pytest.mark.gpu

KIND = {0: "inv", 1: "exp", 2: "sqrt"}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    cuda_or_fail()


@pytest.mark.parametrize("flow,T", [(0, 1.0), (1, 1.0), (2, 4.0)])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("bf16x6", 2e-6)])
def test_explicit_euler_fine_sweep(flow, T, dtype, tol):
    n, N, J = 100, 3, 7
    sm = inputs.sym_matrix(n, KIND[flow], 60 + flow)
    U = np.stack([np.eye(n) + 0.05 * k * sm.A for k in range(N)])
    plan = fa.Plan(n, flow, T, N, fine_steps=J, fine_dtype=dtype, fine_scheme="euler")
    plan.set_matrix(dev(sm.A))
    F = host(plan.fine_sweep(dev(U)))
    plan.close()
    f = orc.propagator("euler", flow, sm.A, T / N, J)
    for b in range(N):
        assert rel(F[b], f(U[b])) < tol, (b, rel(F[b], f(U[b])))


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("bf16x6", 2e-6)])
def test_crank_nicolson_fine_and_coarse_sweeps(dtype, tol):
    n, N, J, m = 130, 4, 6, 2
    sm = inputs.sym_matrix(n, "exp", 61)
    A = 3.0 * sm.A                                  # a stiffer spectrum, [-12, 0]
    U = np.stack([np.eye(n) + 0.1 * k * A / 12 for k in range(N)])
    plan = fa.Plan(n, 1, 1.0, N, fine_steps=J, coarse_steps=m, fine_dtype=dtype,
                   fine_scheme="cn", coarse_scheme="cn")
    plan.set_matrix(dev(A))
    F = host(plan.fine_sweep(dev(U)))
    f = orc.propagator("cn", 1, A, 1.0 / N, J)
    for b in range(N):
        assert rel(F[b], f(U[b])) < tol, (b, rel(F[b], f(U[b])))
    V, G, _ = plan.coarse_sweep(dev(np.eye(n)))
    V = host(V)
    ref_V, _ = np.eye(n), None
    g = orc.propagator("cn", 1, A, 1.0 / N, m)
    x = np.eye(n)
    for b in range(N):
        x = g(x)
        assert rel(V[b + 1], x) < tol * (b + 1), (b, rel(V[b + 1], x))
    plan.close()


@pytest.mark.parametrize("ex", [inputs.PAPER_EX1, inputs.PAPER_EX2], ids=["example1", "example2"])
def test_paper_example_setups_float64(ex):
    """Section 2's examples as the paper ran them: parareal to 1e-12 with its propagators, the
    same iterations as the oracle, the same result (1e-12), and the paper's error measure
    max|E| / max|ref| against the matrix function (Example 1 normalises by max|A|)."""
    A = inputs.paper_example_matrix(ex.example)
    t_o = time.perf_counter()
    ref = orc.parareal(A, ex.flow, ex.T, ex.N, 1, ex.J, ex.N, 1e-12, coarse=ex.coarse,
                       fine=ex.fine)
    t_o = time.perf_counter() - t_o
    plan = fa.Plan(80, ex.flow, ex.T, ex.N, fine_steps=ex.J, coarse_steps=1, max_iters=ex.N,
                   tol=1e-12, fine_dtype="f64", fine_scheme=ex.fine, coarse_scheme=ex.coarse)
    dA = dev(A)
    X, rep = plan.solve(dA)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, rep = plan.solve(dA)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    X = host(X)
    plan.close()
    fref = closed.inv_lu(A) if ex.flow == 0 else scipy.linalg.expm(A)
    scale = A if ex.flow == 0 else fref
    e_gpu, e_orc = orc.paper_norm(X - fref, scale), orc.paper_norm(ref.U[ex.N] - fref, scale)
    print(f"{ex.name}: {rep['iters']} iterations ({ref.iterations} oracle), {dt * 1e3:.1f} ms "
          f"(oracle on the host {t_o * 1e3:.0f} ms), paper error vs f(A) {e_gpu:.3e} "
          f"(oracle {e_orc:.3e})")
    assert abs(rep["iters"] - ref.iterations) <= 1
    assert rel(X, ref.U[ex.N]) < 1e-12
    # the results agree to 1e-12 in Frobenius norm, so the max-abs measures to ~n x that
    assert abs(e_gpu - e_orc) <= 1e-10


def test_paper_example_2_with_the_modified_method():
    """Example 2 with the modified parareal (Section 3) and the same Crank-Nicolson propagators:
    the oracle's Algorithm 3 with those propagators, iteration for iteration."""
    ex = inputs.PAPER_EX2
    A = inputs.paper_example_matrix(2)
    dT = ex.T / ex.N
    ref = M.modified_parareal_generic(np.eye(80), ex.N, orc.propagator("cn", 1, A, dT, 1),
                                      orc.propagator("cn", 1, A, dT, ex.J), ex.N, 1e-12, 1e-12)
    plan = fa.Plan(80, 1, ex.T, ex.N, fine_steps=ex.J, coarse_steps=1, max_iters=ex.N, tol=1e-12,
                   fine_dtype="f64", fine_scheme="cn", coarse_scheme="cn",
                   method=fa.FA_METHOD_MODIFIED, span_drop=1e-12, max_basis=(ex.N + 1) * 4)
    X, rep = plan.solve(dev(A))
    plan.close()
    classical = orc.parareal(A, 1, ex.T, ex.N, 1, ex.J, ex.N, 1e-12, coarse="cn", fine="cn")
    assert rep["iters"] == ref.iterations < classical.iterations
    assert rel(host(X), ref.U[ex.N]) < 1e-12
