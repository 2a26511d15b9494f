"""The slice-partitioned parareal driver (paper_1505_07959_gb300.slices) with the library's fine
and coarse sweeps as propagators, against the library's single-plan solve.  The ranks are
emulated in one process (threads handing states over through queues; each rank's launches are
complete and synchronised before its state is passed on, so no kernel waits on another rank)."""
import queue
import threading

import numpy as np
import pytest

from gpu_helpers import cuda_or_fail, dev, fa, host, rel, torch
from paper_1505_07959_gb300 import inputs, slices

pytestmark = pytest.mark.gpu


class ThreadComm:
    """`size` ranks as threads of one process: queues for the boundary states, a barrier-based
    maximum for the stopping test."""

    def __init__(self, rank, size, links, red):
        self.rank, self.size, self.links, self.red = rank, size, links, red

    def send(self, t, dst):
        torch.cuda.synchronize()
        self.links[(self.rank, dst)].put(t.clone())

    def recv(self, t, src):
        t.copy_(self.links[(src, self.rank)].get(timeout=120))
        torch.cuda.synchronize()

    def max(self, x, device):
        vals, bar = self.red
        vals[self.rank] = x
        bar.wait(timeout=120)
        m = max(vals)
        bar.wait(timeout=120)
        return m


def _run_ranks(size, n, flow, T, N, J, m, dtype, A, K, tol):
    links = {(a, b): queue.Queue() for a in range(size) for b in range(size) if a != b}
    red = ([0.0] * size, threading.Barrier(size))
    results, errors = [None] * size, []

    def work(r):
        try:
            plan = slices.library_plan(n, flow, T, N, r, size, fine_steps=J, coarse_steps=m,
                                       fine_dtype=dtype)
            plan.set_matrix(A)
            props = slices.LibraryPropagators(plan)
            X0 = torch.eye(n, dtype=torch.float64, device="cuda")
            results[r] = slices.parareal_sliced(X0, N, props.fine, props.coarse, K, tol,
                                                ThreadComm(r, size, links, red))
            torch.cuda.synchronize()
            plan.close()
        except Exception as e:           # surface rank failures in the test
            errors.append(e)

    threads = [threading.Thread(target=work, args=(r,)) for r in range(size)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(300)
    assert not errors, errors
    return results


@pytest.mark.parametrize("size,dtype,flow,kind,T,m", [(1, "f64", 0, "inv", 1.0, 1),
                                                        (2, "f64", 1, "exp", 1.0, 1),
                                                        (3, "bf16x6", 2, "sqrt", 6.0, 2)])
def test_sliced_driver_matches_single_plan_solve(size, dtype, flow, kind, T, m):
    cuda_or_fail()
    n, N, J = 96, 7, 4
    sm = inputs.sym_matrix(n, kind, 31)
    A = dev(sm.A)
    plan = fa.Plan(n, flow, T, N, fine_steps=J, coarse_steps=m, max_iters=N, tol=1e-9,
                   fine_dtype=dtype)
    X, rep = plan.solve(A)
    X = host(X)
    plan.close()
    res = _run_ranks(size, n, flow, T, N, J, m, dtype, A, N, 1e-9)
    assert {r.iterations for r in res} == {rep["iters"]}
    np.testing.assert_allclose(res[0].dx_history, rep["dx_history"], rtol=1e-6)
    assert res[-1].hi == N
    assert rel(host(res[-1].final(N)), X) < 1e-12
