"""The mixed batch at full size: 512 problems, n log-uniform in [32, 512], flows cycling
inverse / exponential / square root, N = 16 slices, 32 RK4 steps per slice, tolerance 1e-6,
BF16x6 products.  Sampled problems are checked against the oracle's iterates evaluated in
the eigenbasis (exact for X0 = I)."""
import time

import numpy as np
import pytest

from gpu_helpers import cuda_or_fail, dev, fa, host, rel, torch
from oracle import scalar as S
from paper_1505_07959_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_mixed_batch_of_512_problems():
    cuda_or_fail()
    probs = inputs.batched_problems(512)
    ws = [w for w, _ in probs]
    N, J, K = 16, 32, 16
    b = fa.Batch([w.n for w in ws], [w.flow for w in ws], [w.T for w in ws], [w.m for w in ws],
                 N, J, K, tol=1e-6, dtype="bf16x6")
    As = [dev(sm.A) for _, sm in probs]
    b.solve(As)                                   # warm-up (captures the iteration graph)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xs, iters, dxs, st = b.solve(As)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(f"512-problem batch: {dt * 1e3:.0f} ms, {512 / dt:.1f} solves/s, "
          f"iterations run {max(iters)}, per-problem {np.bincount(iters)}")
    assert st == fa.FA_OK
    rng = np.random.default_rng(0)
    for i in sorted(rng.choice(512, 24, replace=False)):
        w, sm = probs[i]
        # a problem leaves the batch once it converged: its result is its iterate then
        ref = S.to_matrix(sm.Q, S.parareal(sm.lam, w.flow, w.T, N, w.m, J, iters[i], 0.0).u[N])
        e = rel(host(Xs[i]), ref)
        assert e < 1e-6, (i, w.n, w.flow, e)
    b.close()
