"""The n=2048 exponential-flow workload at full size, in the launch configuration the bench
times, against the oracle's iterates evaluated in the eigenbasis (exact for X0 = I)."""
import numpy as np
import pytest

from gpu_helpers import cuda_or_fail, dev, fa, host, rel, torch
from oracle import closed, parareal as orc, scalar as S
from paper_1505_07959_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    cuda_or_fail()


@pytest.fixture(scope="module")
def exp2048():
    w = inputs.EXP_N2048
    return w, inputs.sym_matrix(w.n, w.kind, w.seed)


def test_exp_n2048_solve_matches_oracle(exp2048):
    w, sm = exp2048
    tol = w.mixed_tol                 # the stopping tolerance the bench uses with BF16 products
    plan = fa.Plan(w.n, w.flow, w.T, w.N, fine_steps=w.J, coarse_steps=w.m, max_iters=w.K_max,
                   tol=tol, fine_dtype=w.dtype)
    X, rep = plan.solve(dev(sm.A))
    X = host(X)
    k = rep["iters"]
    sres = S.parareal(sm.lam, w.flow, w.T, w.N, w.m, w.J, k, 0.0)
    ref = S.to_matrix(sm.Q, sres.u[w.N])
    e = rel(X, ref)
    e_closed = rel(X, closed.expm_sym(sm.A))
    full = S.parareal(sm.lam, w.flow, w.T, w.N, w.m, w.J, w.K_max, tol)
    print(f"exp n=2048 {w.dtype}: iters {k} (oracle {full.iterations}), err vs oracle {e:.2e}, "
          f"vs exp(A) {e_closed:.2e}, dx {rep['dx_history']}")
    assert rep["converged"]
    assert e < 1e-6
    assert abs(k - full.iterations) <= 1
    # sampled entries, one by one: row 17 and column 1500 of the oracle's U_N
    assert np.allclose(X[17], ref[17], rtol=0, atol=1e-6 * np.abs(ref).max())
    assert np.allclose(X[:, 1500], ref[:, 1500], rtol=0, atol=1e-6 * np.abs(ref).max())


def test_f64_fine_and_coarse_sweep_at_n2048(exp2048):
    """The float64 path at full matrix size (2 slices, 1 RK4 step: a few seconds of float64)."""
    w, sm = exp2048
    N, J = 2, 1
    plan = fa.Plan(w.n, w.flow, w.T, N, fine_steps=J, fine_dtype="f64")
    plan.set_matrix(dev(sm.A))
    U0, G0 = orc.coarse_sweep(sm.A, w.flow, w.T, N, 1, np.eye(w.n))
    Ug, Gg, _ = plan.coarse_sweep(dev(np.eye(w.n)))
    assert rel(host(Ug)[N], U0[N]) < 1e-13
    F = host(plan.fine_sweep(Ug[:N]))
    ref = orc.fine_sweep(sm.A, w.flow, w.T, N, J, U0[:N])
    for b in range(N):
        assert rel(F[b], ref[b]) < 1e-12
