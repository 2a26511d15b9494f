"""Host logic of the product-accuracy test: the BF16 rounding of its exact reference."""
import numpy as np

from product_accuracy import bf16_rn, bias, rel


def test_bf16_rn_is_nearest_with_eight_significant_bits():
    x = np.random.default_rng(3).standard_normal(200_000) * 10.0 ** np.random.default_rng(4).uniform(-5, 5, 200_000)
    b = bf16_rn(x)
    m, e = np.frexp(b)
    assert np.array_equal(m * 256.0, np.round(m * 256.0))          # 8 significant bits
    half_ulp = np.ldexp(1.0, np.frexp(x)[1] - 9)
    assert np.all(np.abs(b - x) <= half_ulp)                       # nearest


def test_bf16_rn_ties_go_to_even():
    ties = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 3 * 2.0 ** -10 + 2.0 ** -17])
    assert np.array_equal(bf16_rn(ties), [1.0, 1 + 2.0 ** -6, -1.0, 3 * 2.0 ** -10])


def test_bf16_rn_rounds_once_from_float64():
    # 1 + 2^-8 + 2^-30 is just above the tie: direct rounding goes up, while rounding to float32
    # first lands on the tie (1 + 2^-8) and then goes to even (1.0)
    x = np.array([1 + 2.0 ** -8 + 2.0 ** -30])
    assert bf16_rn(x)[0] == 1 + 2.0 ** -7
    assert bf16_rn(x.astype(np.float32).astype(np.float64))[0] == 1.0


def test_error_measures():
    b = np.array([1.0, -2.0, 4.0])
    assert rel(b, b) == 0.0
    assert np.isclose(bias(b * (1 - 1e-3), b), -1e-3)              # shrinking toward zero
