"""Host helpers of the product-accuracy test: the exact reference of a one-term BF16 product
and the error measures (no method arithmetic)."""
import numpy as np


def bf16_rn(x: np.ndarray) -> np.ndarray:
    """x rounded to BF16 (8 significant bits, ties to even) directly from float64, as the
    library rounds its float64 operands; normal range only (enough for Gaussian inputs).  A
    conversion through float32 first rounds twice and differs on a few elements per million."""
    m, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def rel(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def bias(a: np.ndarray, b: np.ndarray) -> float:
    """sum((a - b) sign(b)) / sum|b|: negative when a is shrunk toward zero."""
    return float(np.sum((a - b) * np.sign(b)) / np.sum(np.abs(b)))
