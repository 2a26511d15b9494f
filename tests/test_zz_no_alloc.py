"""The allocation-free product (fa_product_noalloc), for callers that cannot allocate device
memory, against the planned product (fa_debug_product, which runs in a caller-bound
workspace).  Collected last so that a run stopping at the first failure has run every other
test before it."""
import numpy as np
import pytest

from gpu_helpers import PRODUCT_TOL, cuda_or_fail, dev, fa, host, torch

pytestmark = pytest.mark.gpu


def test_no_alloc_product_matches_planned_product_on_two_calls():
    cuda_or_fail()
    stream = torch.cuda.current_stream().cuda_stream
    dtype = "bf16x6"
    for call, n in enumerate((384, 200)):          # two calls in a row, sharing the scratch
        rng = np.random.default_rng(100 + call)
        L, R = rng.standard_normal((n, n)), rng.standard_normal((n, n))
        plan = fa.Plan(n, fa.FA_FLOW_SQRT, 1.0, 1, fine_steps=1, fine_dtype=dtype)
        ref = host(plan.debug_product(dev(L), dev(R)))
        plan.close()
        C = torch.empty((n, n), dtype=torch.float64, device="cuda")
        fa.fa_product_noalloc(n, fa.DTYPES[dtype], dev(L), dev(R), C, stream)
        out = host(C)
        scale = np.linalg.norm(L) * np.linalg.norm(R)
        assert np.linalg.norm(out - ref) / scale < PRODUCT_TOL[dtype], call
        assert np.linalg.norm(out - L @ R) / scale < PRODUCT_TOL[dtype], call


@pytest.mark.parametrize("n", [197, 1024])
def test_no_alloc_product_padded_rows_and_the_array_limit(n):
    """n = 197 pads each operand row to 200 elements (ldp > n); n = 1024 fills the array."""
    cuda_or_fail()
    stream = torch.cuda.current_stream().cuda_stream
    dtype = "bf16x6"
    rng = np.random.default_rng(300 + n)
    L, R = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    plan = fa.Plan(n, fa.FA_FLOW_SQRT, 1.0, 1, fine_steps=1, fine_dtype=dtype)
    ref = host(plan.debug_product(dev(L), dev(R)))
    plan.close()
    scale = np.linalg.norm(L) * np.linalg.norm(R)
    for call in range(2):
        C = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        fa.fa_product_noalloc(n, fa.DTYPES[dtype], dev(L), dev(R), C, stream)
        out = host(C)
        assert np.all(np.isfinite(out)), call
        assert np.linalg.norm(out - ref) / scale < PRODUCT_TOL[dtype], call
        assert np.linalg.norm(out - L @ R) / scale < PRODUCT_TOL[dtype], call


def test_no_alloc_rejects_sizes_beyond_its_array():
    cuda_or_fail()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(fa.FaError) as ei:
        fa.fa_product_noalloc(1025, fa.FA_BF16X6, x, x, x, 0)
    assert ei.value.status == 1
    assert "1024" in fa.fa_last_error()
