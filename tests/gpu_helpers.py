"""Shared set-up for the GPU parity tests (imported by the test_gpu_* modules)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1505_07959_gb300 import build, fa  # noqa: E402

# Bound on ||C - L R||_F / (||L||_F ||R||_F) for one product in each arithmetic.
# BF16 rounding of both operands costs up to 2^-9 each (bound 2^-7).  With a
# two-term split each operand keeps ~18 bits, and the dropped cross term x1 y1
# and the two residuals are ~2^-18 each (bound 2^-15).  BF16X4 splits the left
# operand into three terms, which changes nothing at this level.  With three
# terms on both sides everything dropped is ~2^-27, and float32 accumulation
# (~2^-24 relative to ||L|| ||R||) dominates (bound 2^-21).
PRODUCT_TOL = {"f64": 1e-14, "bf16": 2 ** -7, "bf16x3": 2 ** -15, "bf16x4": 2 ** -15,
               "bf16x6": 2 ** -21}
MIXED = ["bf16", "bf16x3", "bf16x4", "bf16x6"]


def cuda_or_fail():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    build.build_library()
    fa.load_library()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(x, ref):
    return float(np.linalg.norm(np.asarray(x) - np.asarray(ref)) / np.linalg.norm(ref))
