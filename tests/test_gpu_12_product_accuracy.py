"""Accuracy of single tensor-core products against float64, per BF16 form (seeded Gaussian
n x n operands), at the orders the workloads use.

    python -m pytest tests/test_gpu_12_product_accuracy.py -m gpu -s

err = ||C - L R||_F / ||L R||_F, bias = sum((C - L R) sign(L R)) / sum |L R|.  For the one-term
form the accumulation is separated from the operands' rounding: C_rep is the float64 product of
the BF16-rounded operands (each BF16 x BF16 product is exact, so C_rep is what an exact
accumulator returns); acc_err / acc_bias compare C with C_rep, and f32_rn_err is numpy's
round-to-nearest float32 sum of the same products, for scale.  The tensor core truncates while it
accumulates, so the one-term form (accumulated over the whole k extent in TMEM) shows a bias
toward zero that grows with the number of MMA instructions, still far below its operands'
rounding; the multi-term forms drain the main product every 64-wide k-block (float32 round to
nearest) and stay at the split's level."""
import json

import numpy as np
import pytest

from gpu_helpers import cuda_or_fail, dev, fa, host
from product_accuracy import bf16_rn, bias, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [256, 1024, 2048, 4096])
def test_product_accuracy_per_form(n):
    cuda_or_fail()
    rng = np.random.default_rng(n)
    L, R = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    ref = L @ R
    out = {"n": n}
    for dt in ("bf16", "bf16x4", "bf16x6"):
        plan = fa.Plan(n, fa.FA_FLOW_SQRT, 1.0, 1, fine_steps=1, fine_dtype=dt)
        C = host(plan.debug_product(dev(L), dev(R)))
        plan.close()
        out[dt] = {"err": rel(C, ref), "bias": bias(C, ref)}
        if dt == "bf16":
            Lb, Rb = bf16_rn(L), bf16_rn(R)
            rep = Lb @ Rb
            f32 = (Lb.astype(np.float32) @ Rb.astype(np.float32)).astype(np.float64)
            out[dt].update(acc_err=rel(C, rep), acc_bias=bias(C, rep), f32_rn_err=rel(f32, rep))
    print(json.dumps(out))
    # one term: the operands' rounding (2^-9 each, ~2.4e-3 in Frobenius norm) dominates; the
    # accumulator's truncation is a bias toward zero of at most ~2.5e-8 per MMA instruction
    # (k / 16 instructions)
    assert 1.5e-3 < out["bf16"]["err"] < 4e-3
    assert -2.5e-8 * n / 16 < out["bf16"]["acc_bias"] <= 0.0
    assert out["bf16"]["acc_err"] < 2.5e-8 * n / 16 + 5e-7
    # split forms: no growth with k (per-k-block drains)
    assert out["bf16x4"]["err"] < 1e-5
    assert out["bf16x6"]["err"] < 3e-7
    assert abs(out["bf16x6"]["bias"]) < 1e-7
