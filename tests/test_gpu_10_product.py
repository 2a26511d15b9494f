"""One matrix product through each arithmetic of the library (tcgen05 BF16 term products and
float64 SIMT), against numpy.  This isolates the GEMM from the RK4 and parareal epilogues."""
import numpy as np
import pytest

from gpu_helpers import MIXED, PRODUCT_TOL, cuda_or_fail, dev, fa, host, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    cuda_or_fail()


@pytest.mark.parametrize("n", [8, 64, 130, 256, 300])
@pytest.mark.parametrize("dtype", ["f64"] + MIXED)
def test_product(n, dtype):
    rng = np.random.default_rng(n)
    L = rng.standard_normal((n, n))
    R = rng.standard_normal((n, n))
    plan = fa.Plan(n, fa.FA_FLOW_SQRT, 1.0, 1, fine_steps=1, fine_dtype=dtype)
    C = host(plan.debug_product(dev(L), dev(R)))
    ref = L @ R
    err = np.linalg.norm(C - ref) / (np.linalg.norm(L) * np.linalg.norm(R))
    print(f"product n={n} {dtype}: rel err {err:.3e}")
    assert err < PRODUCT_TOL[dtype], err
    # element-wise: every entry within the same bound scaled by its row/column norms
    bound = PRODUCT_TOL[dtype] * np.outer(np.linalg.norm(L, axis=1), np.linalg.norm(R, axis=0))
    assert np.all(np.abs(C - ref) <= 4 * bound + 1e-300)


@pytest.mark.parametrize("dtype", ["f64", "bf16x4"])
def test_product_is_bitwise_reproducible(dtype):
    rng = np.random.default_rng(1)
    n = 384
    L, R = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    plan = fa.Plan(n, fa.FA_FLOW_INV, 1.0, 1, fine_steps=1, fine_dtype=dtype)
    a = host(plan.debug_product(dev(L), dev(R)))
    b = host(plan.debug_product(dev(L), dev(R)))
    assert np.array_equal(a, b)
