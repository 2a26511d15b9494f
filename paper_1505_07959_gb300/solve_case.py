"""Run whole solves of one workload on the GPU and report iterations, timings and accuracy.

    python -m paper_1505_07959_gb300.solve_case --flow sqrt --n 4096 --N 128 --J 32 --T 20 \\
        --m 1 --dtype bf16 --iters 8 --refine 4
    python -m paper_1505_07959_gb300.solve_case --flow inv_wide --n 1024 --N 64 --J 64 --T 1 \\
        --dtype bf16x6 --coarse-dtype f64 --coarse taylor4 --iters 20 --tol 1e-8

Builds the library if needed and solves A = Q diag(lam) Q^T of the flow's family (seed
`--seed`) from X0 = I.  The error is the relative Frobenius distance of the result to f(A)
formed from the generating eigen-decomposition (A^{-1}, exp(A) or A^{1/2}); the solve itself
never sees that decomposition.  Prints one JSON line per solve.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import build, fa, inputs, learned

FLOWS = {"inv": (fa.FA_FLOW_INV, "inv"), "inv_wide": (fa.FA_FLOW_INV, "inv_wide"),
         "exp": (fa.FA_FLOW_EXP, "exp"), "sqrt": (fa.FA_FLOW_SQRT, "sqrt")}


def f_of_A(flow: int, sm) -> np.ndarray:
    if flow == fa.FA_FLOW_INV:
        f = 1.0 / sm.lam
    elif flow == fa.FA_FLOW_EXP:
        f = np.exp(sm.lam)
    else:
        f = np.sqrt(sm.lam)
    return (sm.Q * f[None, :]) @ sm.Q.T


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--flow", default="sqrt", choices=sorted(FLOWS))
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--J", type=int, default=32)
    ap.add_argument("--T", type=float, default=20.0)
    ap.add_argument("--m", type=int, default=1)
    ap.add_argument("--dtype", default="bf16")
    ap.add_argument("--coarse-dtype", default=None)
    ap.add_argument("--iters", type=int, default=8)
    ap.add_argument("--tol", type=float, default=0.0)
    ap.add_argument("--refine", type=int, default=0)
    ap.add_argument("--coarse", default="euler", choices=["euler", "taylor4", "learned"],
                    help="coarse propagator: forward Euler, the Taylor-4 step, or the network")
    ap.add_argument("--weights", default=learned.DEFAULT_WEIGHTS)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--repeats", type=int, default=1)
    ap.add_argument("--method", default="classical", choices=["classical", "modified"],
                    help="Algorithm 1, or the modified parareal of Section 3 (exp flow)")
    ap.add_argument("--max-basis", type=int, default=0, help="modified: capacity of the space")
    args = ap.parse_args()

    import torch

    build.build_library()
    fa.load_library()
    flow, kind = FLOWS[args.flow]
    sm = inputs.sym_matrix(args.n, kind, args.seed)
    ref = f_of_A(flow, sm)
    kind_c = fa.FA_COARSE_EULER if args.coarse == "euler" else fa.FA_COARSE_LEARNED
    plan = fa.Plan(args.n, flow, args.T, args.N, args.J, coarse_steps=args.m,
                   fine_dtype=args.dtype, coarse_dtype=args.coarse_dtype, max_iters=args.iters,
                   tol=args.tol, refine_steps=args.refine, coarse_kind=kind_c,
                   method=fa.FA_METHOD_MODIFIED if args.method == "modified"
                   else fa.FA_METHOD_CLASSICAL, max_basis=args.max_basis)
    if args.coarse == "taylor4":
        plan.set_learned(learned.constant_blob((1.0, 1.0, 1.0, 1.0)))
    elif args.coarse == "learned":
        plan.set_learned(np.fromfile(args.weights, dtype=np.float32))
    A = torch.from_numpy(sm.A).cuda()
    for r in range(args.repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        X, rep = plan.solve(A)
        e1.record()
        torch.cuda.synchronize()
        err = float(np.linalg.norm(X.cpu().numpy() - ref) / np.linalg.norm(ref))
        out = {"flow": args.flow, "n": args.n, "N": args.N, "J": args.J, "T": args.T, "m": args.m,
               "dtype": args.dtype, "coarse_dtype": args.coarse_dtype or args.dtype,
               "refine": args.refine, "coarse": args.coarse, "repeat": r, "iters": rep["iters"],
               "converged": rep["converged"], "last_dx": rep["last_dx"],
               "dx_history": ["%.3e" % d for d in rep["dx_history"]],
               "solve_ms": e0.elapsed_time(e1), "t_init_ms": rep["t_init_ms"],
               "t_fine_ms": rep["t_fine_ms"], "t_coarse_ms": rep["t_coarse_ms"],
               "t_refine_ms": rep["t_refine_ms"], "rel_err": err, "method": args.method,
               "basis_dim": rep["basis_dim"], "fine_blocks": rep["fine_blocks"]}
        print(json.dumps(out), flush=True)
    plan.close()


if __name__ == "__main__":
    main()
