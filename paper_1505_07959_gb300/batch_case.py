"""Solve the mixed batch workload (512 problems by default) and report time and accuracy.

    python -m paper_1505_07959_gb300.batch_case --count 512 [--autotune] [--cache tune.txt]
    python -m paper_1505_07959_gb300.batch_case --count 512 --fp64-every 16

Problems as `inputs.batched_problems` (n log-uniform in [32, 512], flows cycling inverse /
exponential / square root, tol 1e-6, N = 16, J = 32).  With --autotune the launch schedule is
tuned (or read from --cache) before the timed solves.  Errors are relative Frobenius distances
to f(A) formed from each problem's generating eigen-decomposition, on every --sample-th problem,
per flow (the square-root problems integrate to T = 20 only, where the transient of the
smallest eigenvalues is still ~2e-2 away from A^{1/2}).  With --fp64-every k, every k-th
problem is instead solved alone by a float64 plan (the plain float64 GPU parareal, same N, J,
m and tolerance) and the batch's float64 time is extrapolated from that sample (sum x k).
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
    ap.add_argument("--fp64-every", type=int, default=0)
    args = ap.parse_args()

    import torch

    build.build_library()
    fa.load_library()
    probs = inputs.batched_problems(args.count)
    ws = [w for w, _ in probs]
    if args.fp64_every:
        total_ms, iters, errs, k = 0.0, [], [], 0
        for i in range(0, args.count, args.fp64_every):
            w, sm = probs[i]
            plan = fa.Plan(w.n, w.flow, w.T, w.N, w.J, coarse_steps=w.m, fine_dtype="f64",
                           max_iters=w.K_max, tol=w.tol)
            A = torch.from_numpy(sm.A).cuda()
            X, rep = plan.solve(A)
            total_ms += rep["t_init_ms"] + rep["t_fine_ms"] + rep["t_coarse_ms"]
            iters.append(rep["iters"])
            if w.flow != 2:
                ref = f_of_A(w.flow, sm)
                errs.append(float(np.linalg.norm(X.cpu().numpy() - ref) / np.linalg.norm(ref)))
            plan.close()
            k += 1
        est = total_ms * args.fp64_every
        print(json.dumps({"count": args.count, "dtype": "f64", "sampled": k,
                          "sample_ms": total_ms, "batch_ms_extrapolated": est,
                          "solves_per_s_extrapolated": args.count / est * 1e3,
                          "iters_max": max(iters), "err_max_inv_exp": max(errs)}), flush=True)
        return
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
