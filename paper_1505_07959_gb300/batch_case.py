"""Solve the mixed batch workload (512 problems by default) and report time and accuracy.

    python -m paper_1505_07959_gb300.batch_case --count 512 [--autotune] [--cache tune.txt]

Problems as `inputs.batched_problems` (n log-uniform in [32, 512], flows cycling inverse /
exponential / square root, tol 1e-6, N = 16, J = 32).  With --autotune the launch schedule is
tuned (or read from --cache) before the timed solves.  Errors are relative Frobenius distances
to f(A) formed from each problem's generating eigen-decomposition, on every --sample-th problem,
per flow (the square-root problems integrate to T = 20 only, where the transient of the
smallest eigenvalues is still ~2e-2 away from A^{1/2}).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import build, fa, inputs
from .solve_case import f_of_A


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--dtype", default="bf16x6")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--cache", default=None)
    ap.add_argument("--repeats", type=int, default=2)
    ap.add_argument("--sample", type=int, default=16)
    args = ap.parse_args()

    import torch

    build.build_library()
    fa.load_library()
    probs = inputs.batched_problems(args.count)
    ws = [w for w, _ in probs]
    b = fa.Batch([w.n for w in ws], [w.flow for w in ws], [w.T for w in ws], [w.m for w in ws],
                 N=ws[0].N, fine_steps=ws[0].J, max_iters=ws[0].K_max, tol=ws[0].tol,
                 dtype=args.dtype)
    As = [torch.from_numpy(sm.A).cuda() for _, sm in probs]
    acct = ""
    if args.autotune:
        t0 = time.time()
        acct = b.autotune(As, args.cache)
        acct += f" ({time.time() - t0:.2f} s)"
    for r in range(args.repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        Xs, iters, dx, st = b.solve(As)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        errs = {0: [], 1: [], 2: []}
        for i in range(0, args.count, args.sample):
            for k in range(3):
                w, sm = probs[min(i + k, args.count - 1)]
                ref = f_of_A(w.flow, sm)
                errs[w.flow].append(float(np.linalg.norm(Xs[i + k if i + k < args.count else args.count - 1].cpu().numpy() - ref) / np.linalg.norm(ref)))
        print(json.dumps({"count": args.count, "dtype": args.dtype, "autotune": args.autotune,
                          "repeat": r, "batch_ms": ms, "solves_per_s": args.count / ms * 1e3,
                          "iters_max": max(iters), "status": st,
                          "err_max_sampled": {["inv", "exp", "sqrt"][k]: max(v) for k, v in errs.items() if v},
                          "tuning": acct}), flush=True)
    b.close()


if __name__ == "__main__":
    main()
