"""Failure detection of the tensor-core kernel: a device-side wait that runs out.

The diagnostic switch fa_debug_set_wait_fault makes CTA 0 of every tensor-core launch issue no
operand loads and shortens every wait to about a millisecond.  Nothing is ever in flight in
that CTA, so its MMA warp's wait on the operand tiles runs out: the kernel raises its abort
flag (the other warps of the CTA leave their waits), records FA_ERR_TIMEOUT in the plan's error
word, releases its tensor memory and returns.  No fault, trap or hang is involved.  The solve
reports the status at its end, and the next solve on the same plan, with the switch off, is
bitwise equal to the one before."""
import numpy as np
import pytest

from gpu_helpers import cuda_or_fail, dev, fa, host, torch
from paper_1505_07959_gb300 import inputs

pytestmark = pytest.mark.gpu

FA_ERR_TIMEOUT = 6


@pytest.mark.parametrize("dtype", ["bf16x6", "bf16"])
def test_wait_that_runs_out_reports_timeout_and_the_plan_recovers(dtype):
    cuda_or_fail()
    n, N = 256, 2
    sm = inputs.sym_matrix(n, "exp", 21)
    plan = fa.Plan(n, fa.FA_FLOW_EXP, 1.0, N, fine_steps=1, max_iters=2, tol=0.0,
                   fine_dtype=dtype)
    A = dev(sm.A)
    try:
        X0, rep0 = plan.solve(A)
        ref = host(X0).copy()
        assert rep0["iters"] == 2
        fa.fa_debug_set_wait_fault(2_000_000, 0)
        try:
            with pytest.raises(fa.FaError) as ei:
                plan.solve(A)
            assert ei.value.status == FA_ERR_TIMEOUT
            assert "timed out" in fa.fa_last_error()
        finally:
            fa.fa_debug_set_wait_fault(0, -1)
        X1, rep1 = plan.solve(A)
        assert rep1["iters"] == 2
        assert np.array_equal(host(X1), ref)
    finally:
        plan.close()
