"""Batched solves (fa_batch_*): many problems of mixed order and flow in shared persistent
launches, against the oracle and against single-problem solves of the same problems."""
import numpy as np
import pytest

from gpu_helpers import cuda_or_fail, dev, fa, host, rel, torch
from oracle import parareal as orc
from paper_1505_07959_gb300 import inputs

pytestmark = pytest.mark.gpu

KIND = {0: "inv", 1: "exp", 2: "sqrt"}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    cuda_or_fail()


def _problems():
    ns = [16, 40, 64, 100, 130, 200, 24, 150, 96]
    flows = [i % 3 for i in range(len(ns))]
    Ts = [4.0 if f == 2 else 1.0 for f in flows]
    ms = [2 if f == 2 else 1 for f in flows]
    mats = [inputs.sym_matrix(n, KIND[f], 40 + i) for i, (n, f) in enumerate(zip(ns, flows))]
    return ns, flows, Ts, ms, mats


def test_batch_matches_oracle_and_single_solves():
    ns, flows, Ts, ms, mats = _problems()
    N, J, K = 4, 4, 3
    b = fa.Batch(ns, flows, Ts, ms, N, J, K, tol=0.0, dtype="bf16x6")
    Xs, iters, dxs, st = b.solve([dev(m.A) for m in mats])
    assert iters == [K] * len(ns)
    for i, (n, f, T, m, sm) in enumerate(zip(ns, flows, Ts, ms, mats)):
        ref = orc.parareal(sm.A, f, T, N, m, J, K, 0.0)
        X = host(Xs[i])
        e = rel(X, ref.U[N])
        assert e < 1e-6, (i, n, f, e)
        plan = fa.Plan(n, f, T, N, fine_steps=J, coarse_steps=m, max_iters=K, tol=0.0,
                       fine_dtype="bf16x6")
        Xp, rep = plan.solve(dev(sm.A))
        assert np.array_equal(host(Xp), X), (i, n, f)     # same arithmetic, element by element
        plan.close()
    b.close()


def test_batch_stops_per_problem_at_tolerance_and_repeats_bitwise():
    ns, flows, Ts, ms, mats = _problems()
    N, J = 6, 4
    b = fa.Batch(ns, flows, Ts, ms, N, J, N, tol=1e-7, dtype="bf16x6")
    As = [dev(m.A) for m in mats]
    X1, it1, dx1, st1 = b.solve(As)
    X2, it2, dx2, st2 = b.solve(As)          # second solve replays the captured iteration graph
    assert it1 == it2
    for a, c in zip(X1, X2):
        assert np.array_equal(host(a), host(c))
    for i, (n, f, T, m, sm) in enumerate(zip(ns, flows, Ts, ms, mats)):
        solo = orc.parareal(sm.A, f, T, N, m, J, N, 1e-7)
        assert abs(it1[i] - solo.iterations) <= 1, (i, it1[i], solo.iterations)
        assert dx1[i] < 1e-7 or it1[i] == N     # converged, or ran every iteration
        # a converged problem leaves the batch: its result is its iterate at convergence
        ref = orc.parareal(sm.A, f, T, N, m, J, it1[i], 0.0)
        assert rel(host(X1[i]), ref.U[N]) < 1e-6
        plan = fa.Plan(n, f, T, N, fine_steps=J, coarse_steps=m, max_iters=N, tol=1e-7,
                       fine_dtype="bf16x6")
        Xp, rep = plan.solve(dev(sm.A))
        assert rep["iters"] == it1[i]
        assert np.array_equal(host(Xp), host(X1[i])), (i, n, f)   # same iterations, same bits
        plan.close()
    assert len(set(it1)) > 1            # the problems converge at different iterations
    b.close()
