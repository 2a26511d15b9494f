"""Accuracy of single tensor-core products through the library, against float64.

    python -m paper_1505_07959_gb300.product_case --n 256 1024 2048 4096 --dtype bf16 bf16x6

For seeded Gaussian L, R (n x n), C = L R through fa_debug_product.  Prints one JSON line per
(n, dtype): err = ||C - L R||_F / ||L R||_F against the float64 product, and its bias toward
zero, sum((C - L R) sign(L R)) / sum|L R| (negative: toward zero).  For the one-term form it
also separates the accumulation: C_rep = the float64 product of the BF16-rounded operands (every
BF16 x BF16 product is exact in float32, so C_rep is what an exact accumulator would return);
acc_err and acc_bias compare C with C_rep, and f32_rn_err is the same BF16 product summed by
numpy in float32 (round-to-nearest), for scale.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import build, fa


def bf16_rn(x: np.ndarray) -> np.ndarray:
    """x rounded to BF16 (8 significant bits, ties to even) directly from float64, as the
    library rounds its float64 operands; normal range only (enough for Gaussian inputs).  A
    conversion through float32 first rounds twice and differs on a few elements per million."""
    m, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def rel(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def bias(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.sum((a - b) * np.sign(b)) / np.sum(np.abs(b)))


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[256, 1024, 2048])
    ap.add_argument("--dtype", nargs="+", default=["bf16", "bf16x6"])
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()

    import torch

    build.build_library()
    fa.load_library()
    for n in args.n:
        rng = np.random.default_rng(args.seed + n)
        L = rng.standard_normal((n, n))
        R = rng.standard_normal((n, n))
        ref = L @ R
        for dt in args.dtype:
            plan = fa.Plan(n, fa.FA_FLOW_SQRT, 1.0, 1, fine_steps=1, fine_dtype=dt)
            C = plan.debug_product(torch.from_numpy(L).cuda(),
                                   torch.from_numpy(R).cuda()).cpu().numpy()
            plan.close()
            out = {"n": n, "dtype": dt, "err": rel(C, ref), "bias": bias(C, ref)}
            if dt == "bf16":
                Lb, Rb = bf16_rn(L), bf16_rn(R)
                rep = Lb @ Rb
                f32 = (Lb.astype(np.float32) @ Rb.astype(np.float32)).astype(np.float64)
                out.update({"acc_err": rel(C, rep), "acc_bias": bias(C, rep),
                            "f32_rn_err": rel(f32, rep)})
            print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
