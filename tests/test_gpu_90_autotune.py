"""Autotuned launch schedules: the tuned batch and plan give bitwise the same results, and the
tuning cache round-trips."""
import numpy as np
import pytest
import torch

from paper_1505_07959_gb300 import fa, inputs
from tests.gpu_helpers import cuda_or_fail, host

pytestmark = pytest.mark.gpu


def _batch(ns, flows, dtype="bf16x6"):
    Ts = [20.0 if f == 2 else 1.0 for f in flows]
    ms = [2 if f == 2 else 1 for f in flows]
    # N = 16 with two Euler substeps keeps the square-root coarse step stable at T = 20
    return fa.Batch(ns, flows, Ts, ms, N=16, fine_steps=2, max_iters=3, tol=0.0, dtype=dtype)


def test_tuned_batch_is_bitwise_equal_and_cache_round_trips(tmp_path):
    cuda_or_fail()
    ns = [40, 70, 100, 150, 200, 260, 300, 520, 90]
    flows = [0, 1, 2, 0, 1, 2, 0, 1, 2]
    kinds = {0: "inv", 1: "exp", 2: "sqrt"}
    As = [torch.from_numpy(inputs.sym_matrix(n, kinds[f], 500 + i).A).cuda()
          for i, (n, f) in enumerate(zip(ns, flows))]
    b = _batch(ns, flows)
    X0, it0, dx0, _ = b.solve(As)
    cache = str(tmp_path / "tune.txt")
    acct = b.autotune(As, cache)
    assert acct.startswith("tuned:"), acct
    X1, it1, dx1, _ = b.solve(As)
    for a, c in zip(X0, X1):
        assert torch.equal(a, c)
    assert it0 == it1 and dx0 == dx1
    # a second batch of the same problems takes the schedule from the cache
    b2 = _batch(ns, flows)
    acct2 = b2.autotune(As, cache)
    assert acct2.startswith("from cache:"), acct2
    assert acct2.split("from cache: ")[1] == acct.split("; ")[1]
    X2, _, _, _ = b2.solve(As)
    for a, c in zip(X0, X2):
        assert torch.equal(a, c)
    # a different batch does not match the cached entry
    b3 = _batch(ns[:-1], flows[:-1])
    assert b3.autotune(As[:-1], cache).startswith("tuned:")
    b.close(); b2.close(); b3.close()


@pytest.mark.parametrize("flow,dtype", [(0, "bf16x6"), (2, "bf16")])
def test_tuned_plan_is_bitwise_equal(flow, dtype):
    cuda_or_fail()
    n = 300
    kind = {0: "inv", 2: "sqrt"}[flow]
    A = torch.from_numpy(inputs.sym_matrix(n, kind, 7).A).cuda()
    T, m = (20.0, 2) if flow == 2 else (1.0, 1)
    plan = fa.Plan(n, flow, T, 16, 2, coarse_steps=m, fine_dtype=dtype, max_iters=3, tol=0.0)
    X0, r0 = plan.solve(A)
    acct = plan.autotune()
    assert acct.startswith("chose prefetch="), acct
    X1, r1 = plan.solve(A)
    assert torch.equal(X0, X1) and r0["dx_history"] == r1["dx_history"]
    plan.close()
